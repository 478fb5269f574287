// mcwf_c128.cu -- complex128 (FP64 throughout) instantiations of the trajectory
// kernel and the choice of lanes per trajectory for a given dimension.
#include "mcwf_kernel.cuh"

namespace qtm {

cudaError_t launch_mcwf_c128(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    // G lanes per trajectory, R rows per lane: N <= G * R.  One lane per
    // trajectory for the smallest systems, otherwise a power-of-two slice of a
    // warp with two rows per lane (the register budget of the FP64 state).
    if (a.n <= 2) return launch_instance<double, 1, 2>(a, stream, info);
    if (a.n <= 8) return launch_instance<double, 4, 2>(a, stream, info);
    if (a.n <= 16) return launch_instance<double, 8, 2>(a, stream, info);
    if (a.n <= 32) return launch_instance<double, 16, 2>(a, stream, info);
    if (a.n <= 64) return launch_instance<double, 32, 2>(a, stream, info);
    return cudaErrorInvalidValue;
}

}  // namespace qtm
