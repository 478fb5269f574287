// mcwf_df64_drive.cu -- double-float instantiations of the trajectory kernel with the
// time-dependent terms a_k cos(omega_k t + phi_k) (-i H_k) compiled into every
// right-hand-side evaluation, for every lane layout.  The plain instantiations
// carry none of that code.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_df64_drive(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return a.G <= 32 ? launch_small<ArDF, kFeatDrive>(a, stream, info) : launch_large<ArDF, kFeatDrive>(a, stream, info);
}

}  // namespace qtm
