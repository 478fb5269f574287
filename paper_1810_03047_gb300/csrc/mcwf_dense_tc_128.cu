// mcwf_dense_tc_128.cu -- the tensor-core engine for padded dimension 128.
#include "dense_tc_kernel.cuh"

namespace qtm {

template cudaError_t launch_dense_tc_np<128>(const DenseArgs &, const CUtensorMap &, cudaStream_t, LaunchInfo *);

}  // namespace qtm
