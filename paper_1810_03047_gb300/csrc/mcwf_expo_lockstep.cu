// mcwf_expo_lockstep.cu -- the lock-step exponential method's per-interval kernel
// (mcwf_expo.cuh) for the layouts the tensor-core path packs its operators in:
// 32 x 2 (dimension <= 64), 64 x 2 (<= 128) and 128 x 2 (<= 256).
#include "mcwf_expo.cuh"

namespace qtm {

cudaError_t launch_expo_lockstep(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    if (a.G == 32 && a.R == 2) return launch_expo_lockstep_instance<32, 2>(a, stream, info);
    if (a.G == 64 && a.R == 2) return launch_expo_lockstep_instance<64, 2>(a, stream, info);
    if (a.G == 128 && a.R == 2) return launch_expo_lockstep_instance<128, 2>(a, stream, info);
    return cudaErrorInvalidValue;
}

}  // namespace qtm
