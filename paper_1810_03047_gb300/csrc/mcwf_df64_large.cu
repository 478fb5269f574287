// mcwf_df64_large.cu -- double-float (FP64-class precision on the FP32 pipe) instantiations of the trajectory kernel
// for the large lane layouts (one translation unit each, so they compile in parallel).
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_df64_large(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_large<ArDF>(a, stream, info);
}

}  // namespace qtm
