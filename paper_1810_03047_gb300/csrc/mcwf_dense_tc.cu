// mcwf_dense_tc.cu -- the tensor-core engine's entry point: dispatch on the
// padded dimension to the instantiation compiled in mcwf_dense_tc_<NP>.cu.
#include "dense_tc.h"

namespace qtm {

template <int NP>
cudaError_t launch_dense_tc_np(const DenseArgs &a, const CUtensorMap &map, cudaStream_t stream, LaunchInfo *info);

cudaError_t launch_dense_tc(const DenseArgs &a, const CUtensorMap &op_map, cudaStream_t stream, LaunchInfo *info)
{
    switch (a.np) {
    case 64: return launch_dense_tc_np<64>(a, op_map, stream, info);
    case 128: return launch_dense_tc_np<128>(a, op_map, stream, info);
    case 192: return launch_dense_tc_np<192>(a, op_map, stream, info);
    case 256: return launch_dense_tc_np<256>(a, op_map, stream, info);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qtm
