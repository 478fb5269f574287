// mcwf_c128_small.cu -- complex128 (FP64 throughout) instantiations of the trajectory kernel
// for the small lane layouts (one translation unit each, so they compile in parallel).
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128_small(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_small<ArF64>(a, stream, info);
}

}  // namespace qtm
