// mcwf_dense_tc_64.cu -- the tensor-core engine for padded dimension 64.
#include "dense_tc_kernel.cuh"

namespace qtm {

template cudaError_t launch_dense_tc_np<64>(const DenseArgs &, const CUtensorMap &, cudaStream_t, LaunchInfo *);

}  // namespace qtm
