// qtm_launch.h -- arguments of the trajectory kernels, shared by the host side of
// the library (qtm_api.cpp) and the CUDA translation units that launch them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qtm {

constexpr int kMaxOps = 64;        // M + collapse operators + observables + drive terms
constexpr int kMaxDrive = 8;       // time-dependent terms a_k cos(omega_k t + phi_k) H_k
constexpr int kMaxChannels = 48;   // collapse operators per problem

// One operator inside the packed operator blob.  Its real and imaginary parts are
// stored as two separate real matrices (an entry whose imaginary or real part is
// zero appears in one of them only -- the matrices of Hermitian Hamiltonians
// with real coefficients, -iH, are purely imaginary off the diagonal, so this
// halves the multiply-adds).  Each part is sliced ELLPACK with slice height G
// (SELL-G): slice r holds rows gl + G r (gl = 0..G-1) and is width_r entries
// wide; entry t of the row owned by lane gl sits at off_r + t G + gl in both the
// column and the value array, so the lanes of a group read consecutive words.
// Short rows are padded with (column 0, value 0).
struct SellPart {
    int table;  // ints[table + 2 r] = off_r, ints[table + 2 r + 1] = width_r, r < R
    int cols;   // column indices: ints[cols + off_r + t G + gl]
    int vals;   // real values: vals[vals + off_r + t G + gl]
};
struct OpOffsets {
    SellPart re, im;
};

// Lanes per trajectory G and state rows per lane R for dimension n (n <= G R);
// G = 0 when no layout fits.
struct Layout {
    int G, R;
};

// Layouts the autotuner may time for dimension n, default first.
inline int layout_candidates(int n, Layout out[2])
{
    if (n <= 2) { out[0] = Layout{1, 2}; return 1; }
    if (n <= 8) { out[0] = Layout{4, 2}; return 1; }
    if (n <= 16) { out[0] = Layout{8, 2}; out[1] = Layout{4, 4}; return 2; }
    if (n <= 32) { out[0] = Layout{16, 2}; out[1] = Layout{8, 4}; return 2; }
    if (n <= 64) { out[0] = Layout{32, 2}; out[1] = Layout{16, 4}; return 2; }
    if (n <= 128) { out[0] = Layout{64, 2}; out[1] = Layout{32, 4}; return 2; }
    if (n <= 256) { out[0] = Layout{128, 2}; out[1] = Layout{64, 4}; return 2; }
    if (n <= 512) { out[0] = Layout{256, 2}; out[1] = Layout{128, 4}; return 2; }
    if (n <= 1024) { out[0] = Layout{256, 4}; return 1; }
    return 0;
}
inline Layout layout_for_dim(int n)
{
    if (n <= 2) return Layout{1, 2};
    if (n <= 8) return Layout{4, 2};
    if (n <= 16) return Layout{8, 2};
    if (n <= 32) return Layout{16, 2};
    if (n <= 64) return Layout{32, 2};
    if (n <= 128) return Layout{64, 2};
    if (n <= 256) return Layout{128, 2};
    if (n <= 512) return Layout{256, 2};
    if (n <= 1024) return Layout{256, 4};
    return Layout{0, 0};
}

struct KernelArgs {
    int n, n_c, n_obs, n_t;
    int G, R;                 // layout the operators were packed for
    // packed operators: op[0] = M = -i H_eff, op[1..n_c] = C_n, op[1+n_c..] = A_k
    const int *ints;
    const void *vals;         // real values in the kernel's arithmetic (double, float pair or float)
    int n_ints, n_vals;
    OpOffsets op[kMaxOps];
    const double *t;          // n_t output times
    const void *psi0;         // n elements of cpx<V>, normalised
    double rtol, atol;
    long long max_steps;
    unsigned long long seed;
    long long traj0, ntraj;   // global id of local trajectory 0; trajectories in this launch
    unsigned long long *queue;     // work counter (zeroed before launch)
    double *out;              // [ntraj][n_t][n_obs]
    unsigned long long *counters;  // accepted, rejected, rhs, jumps, root iterations, failed
    int *first_error;         // first non-zero per-trajectory status (zeroed before launch)
    int max_jumps;            // jump records per trajectory (0 = none)
    int *n_jumps;             // [ntraj]
    double *jump_t;           // [ntraj][max_jumps]
    int *jump_ch;             // [ntraj][max_jumps]
    int smem_vals_offset;     // byte offset of the value array in dynamic shared memory
    int smem_coef_offset;     // byte offset of the method's coefficient tables
    int smem_scratch_offset;  // byte offset of the multi-warp groups' reduction scratch
    int smem_mlp_offset;      // byte offset of the proposal network's per-group scratch
    // learned jump-time proposal
    int rec_stride;           // > 0: record a training pair every rec_stride accepted steps
    int rec_max;              // records per trajectory
    float *rec;               // [ntraj][rec_max][8]: 6 features, time, time left to the next jump
    const float *mlp;         // proposal network (weights and feature normalisation) or null
    float prop_margin;        // a proposed step ends this fraction past the predicted crossing
    int smem_ybuf_offset;     // byte offset of the per-trajectory vector slots
    // time-dependent Hamiltonian: op[drive_op0 + k] = -i H_k, coefficient
    // a_k cos(omega_k t + phi_k) with drive[k] = {a_k, omega_k, phi_k}
    int n_drive, drive_op0;
    double drive[kMaxDrive][3];
    // exponential propagation: expo_levels propagators P_l = exp(M expo_delta 2^l),
    // each column-major [n][G R] in the kernel's complex type (rows >= n zero);
    // expo_uniform: the output grid is uniform with spacing expo_delta 2^(levels-1)
    const void *expo;
    int expo_levels, expo_uniform;
    double expo_delta;
    // Krylov form of the Dormand-Prince step: 2^krylov_shift >= ||M|| (the
    // Krylov vectors are kept as (2^-krylov_shift M)^k psi)
    int krylov_shift;
    // lock-step exponential method (tensor-core products, uniform grid): column il
    // holds psi at lock_psi + il lock_ld (lock_ld / 2 real parts, then the
    // imaginary parts), the tensor cores' product (P_L - I) psi at
    // lock_y + il lock_ld, and its record at lock_col[il]
    float *lock_psi;
    const float *lock_y;
    void *lock_col;
    int lock_j, lock_ld;
    int lock_mode;            // LockMode: interval lock_j, catch-up of the deferred columns, or finish
    int *lock_list;           // [ntraj] deferred columns (count in queue[0], catch-up position in queue[1])
    // FP32 copies of dense operators for the lock-step kernel's products
    // (operator i in the order of op): dense_off[i] >= 0: column-major, column c
    // at dense + dense_off[i] + c dense_ld; < 0: none (the packed form is used)
    const float2 *dense;
    int dense_ld;
    int dense_off[kMaxOps];
};

enum CounterIndex { kAccepted = 0, kRejected, kRhs, kJumps, kRootIters, kFailed, kPropMiss, kNumCounters };

struct LaunchInfo {
    int group, rows, grid, block;
    size_t smem;
};

// Largest dimension the trajectory kernels handle (ten state vectors of N complex
// values per trajectory must fit in shared memory).
constexpr int kMaxDimSparse = 1024;

// The trajectory kernel for the layout args.G x args.R, in complex128,
// double-float or complex64 arithmetic (single-warp layouts in *_small,
// multi-warp layouts in *_large); cudaErrorInvalidValue when no instantiation
// exists for the layout or its shared memory does not fit.
cudaError_t launch_mcwf_c128_small(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_c128_large(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_small(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_large(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_c64_small(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_c64_large(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// One launch of the lock-step exponential method (complex64 arithmetic on the
// layouts 32 x 2, 64 x 2 and 128 x 2) in mode args.lock_mode: output interval
// args.lock_j of columns 0 .. args.ntraj - 1, the catch-up of the deferred
// columns to interval args.lock_j, or the final totals.  cudaErrorInvalidValue
// for any other layout.
cudaError_t launch_expo_lockstep(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// Record of one lock-step column (device layout; zeroed storage is not needed).
constexpr int kLockColBytes = 96;
enum LockMode { kLockInterval = 0, kLockCatchUp = 1, kLockFinish = 2 };
// Instantiations with the learned proposal compiled in (single-warp layouts only).
cudaError_t launch_mcwf_c128_prop(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_prop(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// Instantiations with the time-dependent terms compiled in (every lane layout).
cudaError_t launch_mcwf_c128_drive(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_drive(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_c64_drive(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// The exponential-propagation kernel (every lane layout up to dimension 256).
cudaError_t launch_mcwf_c128_expo(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_expo(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_c64_expo(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// The exponential-propagation kernel with the learned proposal (single-warp layouts only).
cudaError_t launch_mcwf_c128_expo_prop(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
cudaError_t launch_mcwf_df64_expo_prop(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
constexpr int kMaxDimExpo = 256;
inline cudaError_t launch_mcwf_c128(const KernelArgs &a, cudaStream_t s, LaunchInfo *i)
{
    return a.G <= 32 ? launch_mcwf_c128_small(a, s, i) : launch_mcwf_c128_large(a, s, i);
}
inline cudaError_t launch_mcwf_df64(const KernelArgs &a, cudaStream_t s, LaunchInfo *i)
{
    return a.G <= 32 ? launch_mcwf_df64_small(a, s, i) : launch_mcwf_df64_large(a, s, i);
}
inline cudaError_t launch_mcwf_c64(const KernelArgs &a, cudaStream_t s, LaunchInfo *i)
{
    return a.G <= 32 ? launch_mcwf_c64_small(a, s, i) : launch_mcwf_c64_large(a, s, i);
}

// Ensemble reduction of out[ntraj][P] into sums, sums of squares, mean and
// standard error, in a fixed summation order (bitwise reproducible).
// partial must hold 2 * S * P doubles for S = reduce_segments(ntraj).
int reduce_segments(long long ntraj);
cudaError_t launch_ensemble_reduce(const double *out, long long ntraj, int P, double *partial,
                                   double *sum, double *sumsq, double *mean, double *se,
                                   cudaStream_t stream);

// Exact ensemble moments (moments.h) of out[ntraj][P], P = n_t * n_obs, with the
// per-observable scale exponents scale_exp[n_obs] (device): words[P][kMomentWords].
// partial must hold kMomentWords * S * P int64 for S = reduce_segments(ntraj).
cudaError_t launch_ensemble_moments(const double *out, long long ntraj, int P, int n_obs, const int *scale_exp,
                                    long long *partial, long long *words, cudaStream_t stream);

// Sets the message returned by qtm_last_error(NULL).
void set_last_error(const char *msg);

}  // namespace qtm
