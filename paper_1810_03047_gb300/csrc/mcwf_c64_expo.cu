// mcwf_c64_expo.cu -- complex64 instantiations of the exponential-propagation
// trajectory kernel (mcwf_expo.cuh) for every lane layout up to dimension 256:
// FP32 state and propagators, double-float norms and inner products.
#include "mcwf_expo.cuh"

namespace qtm {

cudaError_t launch_mcwf_c64_expo(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_expo<ArF32>(a, stream, info);
}

}  // namespace qtm
