// mcwf_c128_drive.cu -- complex128 instantiations of the trajectory kernel with the
// time-dependent terms a_k cos(omega_k t + phi_k) (-i H_k) compiled into every
// right-hand-side evaluation, for every lane layout.  The plain instantiations
// carry none of that code.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128_drive(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return a.G <= 32 ? launch_small<ArF64, kFeatDrive>(a, stream, info) : launch_large<ArF64, kFeatDrive>(a, stream, info);
}

}  // namespace qtm
