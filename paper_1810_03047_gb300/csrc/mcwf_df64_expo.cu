// mcwf_df64_expo.cu -- double-float instantiations of the exponential-propagation
// trajectory kernel (mcwf_expo.cuh) for every lane layout up to dimension 256.
#include "mcwf_expo.cuh"

namespace qtm {

cudaError_t launch_mcwf_df64_expo(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_expo<ArDF>(a, stream, info);
}

}  // namespace qtm
