// qtm_launch.h -- arguments of the trajectory kernels, shared by the host side of
// the library (qtm_api.cpp) and the CUDA translation units that launch them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qtm {

constexpr int kMaxOps = 64;        // M + collapse operators + observables
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
// G = 0 when no register-resident layout fits.
struct Layout {
    int G, R;
};
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
    int smem_ybuf_offset;     // byte offset of the per-trajectory vector slots
};

enum CounterIndex { kAccepted = 0, kRejected, kRhs, kJumps, kRootIters, kFailed, kNumCounters };

struct LaunchInfo {
    int group, rows, grid, block;
    size_t smem;
};

// Largest dimension the trajectory kernels handle (ten state vectors of N complex
// values per trajectory must fit in shared memory).
constexpr int kMaxDimSparse = 1024;

// FP64 (complex128) trajectory kernel, CSR operators.  Chooses lanes per
// trajectory and rows per lane from args.n; returns cudaErrorInvalidValue when
// no instantiation fits.
cudaError_t launch_mcwf_c128(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// Same kernel with double-float vectors (FP64-class precision on the FP32 pipe).
cudaError_t launch_mcwf_df64(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);
// Same kernel with complex64 vectors and double-float norms.
cudaError_t launch_mcwf_c64(const KernelArgs &args, cudaStream_t stream, LaunchInfo *info);

// Ensemble reduction of out[ntraj][P] into sums, sums of squares, mean and
// standard error, in a fixed summation order (bitwise reproducible).
// partial must hold 2 * S * P doubles for S = reduce_segments(ntraj).
int reduce_segments(long long ntraj);
cudaError_t launch_ensemble_reduce(const double *out, long long ntraj, int P, double *partial,
                                   double *sum, double *sumsq, double *mean, double *se,
                                   cudaStream_t stream);

// Sets the message returned by qtm_last_error(NULL).
void set_last_error(const char *msg);

}  // namespace qtm
