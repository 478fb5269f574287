// mcwf_c64.cu -- complex64 instantiations of the trajectory kernel (FP32 state and
// stage products, double-float norms and inner products, FP64 time and root find).
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c64(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_for_dim<ArF32>(a, stream, info);
}

}  // namespace qtm
