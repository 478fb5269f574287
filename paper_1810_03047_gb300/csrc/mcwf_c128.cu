// mcwf_c128.cu -- complex128 (FP64 throughout) instantiations of the trajectory kernel.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_for_dim<ArF64>(a, stream, info);
}

}  // namespace qtm
