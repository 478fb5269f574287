// mcwf_c128_expo_prop.cu -- complex128 instantiations of the exponential-propagation
// trajectory kernel (mcwf_expo.cuh) with the learned proposal compiled in
// (single-warp lane layouts, dimension <= 64).
#include "mcwf_expo.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128_expo_prop(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_expo_prop<ArF64>(a, stream, info);
}

}  // namespace qtm
