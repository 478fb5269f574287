// mcwf_df64.cu -- double-float instantiations of the trajectory kernel: FP64-class
// precision (each real an FP32 pair hi + lo) computed on the FP32 pipe.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_df64(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_for_dim<ArDF>(a, stream, info);
}

}  // namespace qtm
