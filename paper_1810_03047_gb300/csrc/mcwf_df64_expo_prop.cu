// mcwf_df64_expo_prop.cu -- double-float instantiations of the exponential-propagation
// trajectory kernel (mcwf_expo.cuh) with the learned proposal compiled in
// (single-warp lane layouts, dimension <= 64).
#include "mcwf_expo.cuh"

namespace qtm {

cudaError_t launch_mcwf_df64_expo_prop(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_expo_prop<ArDF>(a, stream, info);
}

}  // namespace qtm
