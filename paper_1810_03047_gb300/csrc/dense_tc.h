// dense_tc.h -- the tensor-core trajectory engine for dense operators (host view).
//
// All trajectories of a CTA advance in lock step as the 128 columns of a state
// block; the Dormand-Prince step is taken in its Krylov form, whose six products
// per attempt wt_{s+1} = 2^-e M wt_s of the real form of the scaled effective
// operator (2N x 2N) with the block's 128 vectors are computed on
// the 5th-generation tensor cores (tcgen05) with both operands split into three
// bf16 terms (M = M0 + M1 + M2, Y = Y0 + Y1 + Y2) and the six products of combined
// order <= 2 accumulated in FP32 in tensor memory: FP32-accurate products.
// State vectors are FP32 in device memory; time, step size, norms, the crossing
// root find and the outputs are FP64.  See mcwf_dense_tc.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "qtm_launch.h"

namespace qtm {

constexpr int kTcCols = 128;    // trajectory columns per CTA (the MMA's M)
constexpr int kTcMaxDim = 256;  // largest N: the 2N real rows of K_s fill the 512 tensor-memory columns

// N padded to a multiple of 64 (one 128-byte bf16 row of a K-block holds 64 values)
__host__ __device__ constexpr int tc_padded_dim(int n) { return ((n + 63) / 64) * 64; }

// Per-column record (one trajectory at a time), 128 bytes.
struct DenseCol {
    double t, h, r, c;          // time, step size, current threshold r_k and channel draw c_k
    long long il;               // trajectory index within the launch; -1 = column idle
    long long k;                // jumps so far (index of the current draws)
    long long attempts;         // attempted steps
    unsigned long long n_acc, n_rej, n_rhs, n_jump;
    int j;                      // next output index
    int sel;                    // bit 0: psi in buffer 1 (else 0)
    int flags;                  // bit 0: previous attempt rejected; bit 1: this step ends at t_end
    int root_iters;
    int round;                  // trajectories this column has taken (static assignment)
    int pad[5];
};
static_assert(sizeof(DenseCol) == 128, "DenseCol is 128 bytes");

// State vectors per column: psi buffers 0 and 1 (psi and the candidate ynew swap
// roles on acceptance), then the Krylov vectors wt_1 .. wt_7 = (2^-e M)^k psi (wt_1
// is updated in place on acceptance: first same as last).  Each vector holds
// 2 np floats: the real parts of rows 0..np-1, then the imaginary parts.
enum DenseVec { kVPsi0 = 0, kVPsi1 = 1, kVK0 = 2, kNumDenseVecs = 9 };

enum DenseMode { kDenseRun = 0, kDenseRhs = 1 };

struct DenseArgs {
    KernelArgs k;          // run description; operators packed SELL-32 with FP32 values
    // copies for the control warps' products, operator i in the order of k.op:
    // dense_off[i] >= 0: column-major [n][np] complex FP32 at dense + dense_off[i];
    // <= -2: diagonal, np complex values at dense + (-2 - dense_off[i]); -1: SELL
    const float2 *dense;
    int dense_off[kMaxOps];
    int np;                // padded dimension (multiple of 64, <= 256)
    int cols;              // resident columns = CTAs * 128 (run mode)
    float *state;          // [kNumDenseVecs][cols][2 np]
    DenseCol *col;         // [cols]
    int mode;              // DenseMode
    unsigned long long wait_limit_ns;  // bound of one device wait (0: 2 s); past it the run reports QTM_ERR_TIMEOUT
    const float *rhs_in;   // rhs mode: [rhs_n][2 np] vectors (planar as the state)
    float *rhs_out;        // rhs mode: [rhs_n][2 np] = M in
    long long rhs_n;
};

// CTAs of a run of ntraj trajectories on a device with `sms` multiprocessors.
inline int dense_tc_ctas(long long ntraj, int sms)
{
    const long long need = (ntraj + kTcCols - 1) / kTcCols;
    return (int)(need < sms ? (need < 1 ? 1 : need) : sms);
}

// Launches the engine.  op_map: 2-D tensor map over the bf16 operator splits
// [3][2 np][2 np] (inner dimension k, box 64 x 128, 128-byte swizzle).
// cudaErrorInvalidValue when np is not one of 64, 128, 192, 256.
cudaError_t launch_dense_tc(const DenseArgs &a, const CUtensorMap &op_map, cudaStream_t stream, LaunchInfo *info);

}  // namespace qtm
