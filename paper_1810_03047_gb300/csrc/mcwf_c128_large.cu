// mcwf_c128_large.cu -- complex128 (FP64 throughout) instantiations of the trajectory kernel
// for the large lane layouts (one translation unit each, so they compile in parallel).
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128_large(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_large<ArF64>(a, stream, info);
}

}  // namespace qtm
