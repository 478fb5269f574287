// mcwf_c64_small.cu -- complex64 (FP32 state, double-float norms) instantiations of the trajectory kernel
// for the small lane layouts (one translation unit each, so they compile in parallel).
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c64_small(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_small<ArF32>(a, stream, info);
}

}  // namespace qtm
