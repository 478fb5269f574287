// mcwf_c128_prop.cu -- complex128 instantiations of the trajectory kernel with the
// learned jump-time proposal compiled in (feature tracking, training records and
// the network's inference), for the single-warp lane layouts (N <= 64).  The
// plain instantiations carry none of that code.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128_prop(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    return launch_small<ArF64, kFeatProposal>(a, stream, info);
}

}  // namespace qtm
