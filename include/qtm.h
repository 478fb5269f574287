/*
 * qtm.h -- C ABI of the GB300 (sm_103a) quantum-trajectory library.
 *
 * The library runs the Monte Carlo wave-function method of Sawerwain &
 * Wisniewska, "QTM: computational package using MPI protocol for quantum
 * trajectories method" (arXiv 1810.03047), Algorithm 1 of Sec. 2.2, over an
 * ensemble of trajectories on one GPU and averages the observables over the
 * ensemble (Sec. 3).  The problem statement follows the paper's mpi_main
 * (Sec. 3): a Hamiltonian H, collapse operators C_n, expectation operators A_k,
 * an initial state, a time interval with output points, a tolerance and a number
 * of trajectories.
 *
 * Conventions
 *   - hbar = 1.  Each trajectory integrates dpsi/dt = -i H_eff psi with
 *     H_eff = H - (i/2) sum_n C_n^dag C_n (Sec. 2.2, Eq. eqn:effective:hamiltonian);
 *     the library forms H_eff itself from H and the C_n.
 *   - Complex numbers are pairs of doubles (re, im), interleaved.
 *   - Matrices are square, n x n, either CSR (the storage of Sec. 3, uCSRMatrix)
 *     or dense row-major.
 *   - Output 0 is the initial state at t[0]; output j is the state at t[j].
 *   - The value recorded for observable k at output j of one trajectory is
 *     Re<psi|A_k|psi> / <psi|psi>; the ensemble mean is the plain average over
 *     trajectories (Sec. 3 averages per node and again at the master; with equal
 *     shares that equals the plain average).
 *   - Random numbers: Philox4x64-10 (Salmon et al., SC'11), key (seed, 0),
 *     counter (jump index k, global trajectory id, 0, 0); words 0 and 1 map to
 *     r_k (the norm threshold of Algorithm 1 steps (A)/(D)) and c_k (the channel
 *     draw of step (C)) by ((w >> 11) + 0.5) * 2^-53, both in (0, 1).  Results
 *     therefore depend only on (seed, trajectory id), not on how trajectories are
 *     split over launches or GPUs.
 *
 * Ownership and threading
 *   - Every pointer passed to qtm_create is a HOST pointer; the library validates
 *     and copies the data, so the caller may free its buffers when qtm_create
 *     returns.  Output pointers of qtm_expect / qtm_sums / qtm_traj_expect /
 *     qtm_jumps are HOST pointers owned by the caller.
 *   - A context owns all device memory it allocates.  Device memory comes from the
 *     allocator installed with qtm_set_allocator (the Python binding installs the
 *     PyTorch caching allocator), else from cudaMallocAsync on the context stream.
 *   - All device work of a context is issued on the CUDA stream given to
 *     qtm_create (NULL = the legacy default stream).  qtm_run is asynchronous;
 *     qtm_expect, qtm_sums, qtm_stats, qtm_traj_expect and qtm_jumps synchronise
 *     that stream.  A context must not be used from two host threads at once.
 *
 * Errors
 *   - No C++ exception crosses this ABI; every call returns a qtm_status.
 *   - Argument errors are reported by the call that receives them (QTM_ERR_ARG)
 *     and a message is available from qtm_last_error(ctx) (or qtm_last_error(NULL)
 *     when no context exists yet).
 *   - Per-trajectory failures inside qtm_run (step limit, step-size underflow,
 *     non-finite state, a jump with no channel) do not stop the other
 *     trajectories; they are counted, and the first failure's code is returned by
 *     the next synchronising call.  Outputs of a failed trajectory after the
 *     failure are NaN.  This mirrors ZVODE's negative ISTATE being turned into an
 *     error level (Sec. 3, zvode_method_for_mc).
 */
#ifndef QTM_H
#define QTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QTM_OK = 0,
    QTM_ERR_ARG = 1,          /* invalid argument (message in qtm_last_error) */
    QTM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    QTM_ERR_NOMEM = 3,        /* host or device allocation failed */
    QTM_ERR_MAXSTEPS = 4,     /* a trajectory exceeded max_steps attempted steps */
    QTM_ERR_STEPSIZE = 5,     /* step size fell below 1e-14 max(1, |t|) */
    QTM_ERR_NONFINITE = 6,    /* a non-finite error norm (NaN/Inf state) */
    QTM_ERR_NO_CHANNEL = 7,   /* the norm fell to r but every ||C_n psi|| was 0 */
    QTM_ERR_TIMEOUT = 8,      /* a bounded device wait of the tensor-core engine gave up (qtm_set_wait_limit) */
    QTM_ERR_STATE = 9,        /* call out of order (e.g. qtm_expect before qtm_run) */
    QTM_ERR_UNSUPPORTED = 10  /* the problem has no kernel in this build (e.g. dim too large) */
} qtm_status;

enum { QTM_FORMAT_DENSE = 0, QTM_FORMAT_CSR = 1 };

/* Arithmetic of the trajectory integration.  In every mode the time, step size,
 * crossing test, jump-time root find and ensemble reduction are FP64. */
enum {
    QTM_PREC_C128 = 0,  /* complex128 state, operators and stage products (FP64 throughout) */
    QTM_PREC_C64 = 1,   /* complex64 state, operators and stage products; norms and inner
                           products accumulated in double-float (about 48 bits); the
                           step-size control in FP32.  Faster, but a trajectory's jump
                           times move by about the FP32 rounding of its state */
    QTM_PREC_DF64 = 3,  /* double-float: every real is a pair of FP32 numbers hi + lo
                           (about 48 significant bits) and every product and sum is
                           error-free-transformed on the FP32 pipe; matches complex128
                           to round-off while running on GB300's much wider FP32 units */
    QTM_PREC_BF16X6 = 4 /* tensor-core engine for dense operators (dim <= 256): 128
                           trajectories per SM advance in lock step and every stage
                           product M Y (real 2N x 2N form) runs on the tcgen05 tensor
                           cores with both operands split into three bf16 terms and
                           the six products of combined order <= 2 accumulated in
                           FP32 (as accurate as an FP32 product); state vectors FP32,
                           outputs, norms and root find as complex64 with FP64
                           scalars.  No learned proposal, no layout choice.  With
                           QTM_METHOD_EXPONENTIAL: the lock-step exponential
                           method on the tensor cores (see qtm_set_method) */
};

/* Integrator of the no-jump evolution (qtm_set_method). */
enum {
    QTM_METHOD_DOPRI5 = 0,      /* Dormand-Prince 5(4) with error control and continuous extension (default) */
    QTM_METHOD_EXPONENTIAL = 1  /* exact propagation psi(t) = exp(M (t - t_k)) psi_k between jumps, for stiff
                                   problems; see qtm_set_method */
};

/* qtm_problem.flags */
enum {
    QTM_FLAG_RECORD_JUMPS = 1  /* keep the first max_jumps_recorded jump times/channels per trajectory */
};

/* A square complex operator (host memory, copied by qtm_create).
 *   CSR:   row_ptr[n + 1] (row_ptr[0] = 0, non-decreasing), col_ind[nnz] in [0, n),
 *          values[2 * nnz]; nnz = row_ptr[n].
 *   dense: values[2 * n * n] row-major; row_ptr, col_ind ignored, nnz ignored. */
typedef struct {
    int32_t n;
    int32_t format;            /* QTM_FORMAT_CSR or QTM_FORMAT_DENSE */
    const int32_t *row_ptr;
    const int32_t *col_ind;
    const double *values;      /* (re, im) interleaved */
    int64_t nnz;
} qtm_op;

/* The problem statement (host memory, copied by qtm_create). */
typedef struct {
    int32_t dim;               /* Hilbert-space dimension N >= 1 */
    qtm_op H;                  /* system Hamiltonian, Hermitian within 1e-12 (relative) */
    int32_t n_c;               /* number of collapse operators, >= 0 */
    const qtm_op *C;           /* n_c collapse operators, channel order = array order */
    int32_t n_obs;             /* number of observables, >= 0 */
    const qtm_op *A;           /* n_obs Hermitian observables */
    const double *psi0;        /* 2 * dim; normalised by the library (must be non-zero, finite) */
    int32_t n_t;               /* number of output times, >= 1 */
    const double *t;           /* n_t strictly increasing times; t[0] is the start time */
    double rtol, atol;         /* Dormand-Prince error control: rtol > 0, atol >= 0 */
    int32_t precision;         /* QTM_PREC_* */
    int64_t max_steps;         /* attempted steps per trajectory before QTM_ERR_MAXSTEPS (> 0) */
    int32_t flags;             /* QTM_FLAG_* */
    int32_t max_jumps_recorded;/* with QTM_FLAG_RECORD_JUMPS: jumps kept per trajectory (>= 1) */
} qtm_problem;

typedef struct {
    int64_t trajectories;      /* trajectories of the last qtm_run */
    int64_t accepted;          /* accepted Dormand-Prince steps (all trajectories) */
    int64_t rejected;          /* rejected steps */
    int64_t rhs_evals;         /* products M psi (one column each), rejected steps included */
    int64_t jumps;             /* quantum jumps */
    int64_t root_iters;        /* Newton/bisection iterations of the jump-time search */
    int64_t failed;            /* trajectories that stopped with an error */
    int32_t first_error;       /* qtm_status of the first failure, QTM_OK if none */
    int32_t kernel_group;      /* lanes per trajectory chosen by the library */
    int32_t kernel_rows;       /* state rows per lane chosen by the library */
    int32_t grid;              /* CTAs of the trajectory kernel */
    int32_t block;             /* threads per CTA of the trajectory kernel */
    int32_t reserved;
    double kernel_ms;          /* device time of the trajectory kernel (CUDA events on the context stream) */
    double reduce_ms;          /* device time of the ensemble reduction */
    int64_t proposal_misses;   /* exponential method with the learned proposal: crossings whose predicted
                                  bracket missed (the search then descended as without a prediction) */
    double product_ms;         /* exponential method on the tensor cores (QTM_PREC_BF16X6): device time of
                                  one tensor-core product launch, (P_L - I) applied to every trajectory (the
                                  first output interval's launch); 0 otherwise */
} qtm_stats_t;

typedef struct qtm_ctx qtm_ctx;

/* Device allocator hooks (no counterpart in the paper: device-memory plumbing).
 * alloc returns device memory usable on `stream` or
 * NULL; free releases it.  Installing NULL hooks restores cudaMallocAsync /
 * cudaFreeAsync.  Contexts keep the hooks that were installed when they were
 * created.  Not thread-safe with concurrent qtm_create calls. */
typedef void *(*qtm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*qtm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
qtm_status qtm_set_allocator(qtm_alloc_fn alloc, qtm_free_fn free_fn, void *user);

/* The problem statement of the paper's mpi_main (Sec. 3).  Validates and copies
 * the problem, forms H_eff (Sec. 2.2, Eq. eqn:effective:hamiltonian), uploads the
 * operators to the current CUDA device and returns a context bound to
 * cuda_stream (a cudaStream_t, may be NULL).  On error *out is NULL and the
 * message is available from qtm_last_error(NULL). */
qtm_status qtm_create(const qtm_problem *problem, void *cuda_stream, qtm_ctx **out);

/* Algorithm 1 (Sec. 2.2) for every trajectory: runs trajectories 0 .. ntraj-1 of
 * the ensemble keyed by seed (asynchronous), then the ensemble sums of Sec. 3.
 * ntraj >= 0.  Replaces the results of any previous run of this context. */
qtm_status qtm_run(qtm_ctx *ctx, int64_t ntraj, uint64_t seed);

/* Same for global trajectory ids first .. first+ntraj-1 (first >= 0): a shard of a
 * larger ensemble, e.g. one GPU's share (the paper's worker processes, Sec. 3).
 * Results equal those of the same ids in a single larger run. */
qtm_status qtm_run_range(qtm_ctx *ctx, int64_t first, int64_t ntraj, uint64_t seed);

/* Runs several ensembles at once (the paper runs one system per mpi_main call,
 * Sec. 3; batching systems of uneven size is this library's): context i runs global trajectory ids
 * first[i] .. first[i]+ntraj[i]-1 (first may be NULL: all zero) keyed by seed.  All runs are captured into one CUDA graph -- each system's
 * persistent kernel and reduction on its own branch -- and launched on the
 * stream of ctxs[0]; the other contexts' streams wait for that launch, so each
 * context's results are read with qtm_expect as usual.  Systems of different
 * dimension (e.g. Ising chains of several lengths) thus share the GPU in one
 * submission, and the tail of one system overlaps the others.  All contexts must
 * be on the same device and distinct.  qtm_stats of a batched run reports no
 * kernel times (kernel_ms = 0). */
qtm_status qtm_run_batch(qtm_ctx *const *ctxs, const int64_t *first, const int64_t *ntraj, int32_t n,
                         uint64_t seed);

/* No counterpart in the paper (GPU lane mapping).  Times the lane layouts
 * available for the context's dimension (threads per
 * trajectory x state rows per thread, see qtm_stats_t.kernel_group / kernel_rows)
 * on a run of `sample` trajectories keyed by seed, keeps the fastest, and returns
 * it in *group and *rows (either may be NULL).  Results of later runs do not
 * depend on the layout beyond round-off.  Synchronises; discards the sample's
 * results. */
qtm_status qtm_autotune(qtm_ctx *ctx, int64_t sample, uint64_t seed, int32_t *group, int32_t *rows);

/* No counterpart in the paper (GPU lane mapping).  Selects one of the lane
 * layouts qtm_autotune would consider for the context's
 * dimension (e.g. a layout found by an earlier qtm_autotune); QTM_ERR_UNSUPPORTED
 * for any other pair.  Synchronises; discards the results of earlier runs. */
qtm_status qtm_set_layout(qtm_ctx *ctx, int32_t group, int32_t rows);

/* The trajectory average of Sec. 3: ensemble mean (n_t * n_obs doubles,
 * output-major: [j * n_obs + k]) and, if stderr_out is not NULL, the standard
 * error sqrt(var / n) with the sample variance (n - 1 divisor; 0 when n < 2),
 * computed from the run's exact moment words (below), so the result does not
 * depend on how the trajectories were split over runs or GPUs.  NaN where a
 * trajectory failed.  Synchronises; returns the first per-trajectory failure of
 * the run, if any. */
qtm_status qtm_expect(qtm_ctx *ctx, double *mean, double *stderr_out);

/* Sums over the run's trajectories (from the same moment words):
 * sum[j * n_obs + k] = sum_i x_i, sumsq = sum_i x_i^2, *count = trajectories. */
qtm_status qtm_sums(qtm_ctx *ctx, double *sum, double *sumsq, int64_t *count);

/* ---------------------------------------------------------------------------
 * Exact ensemble moments, for combining shards (the paper's two-level average of
 * Sec. 3: each node averages its trajectories, the master averages the nodes).
 * A value x of observable k is Re<psi|A_k|psi>/<psi|psi>, bounded in magnitude by
 * max_i sum_j (|Re A_ij| + |Im A_ij|) < 2^(E_k - 1); E_k is the observable's scale
 * exponent.  The library truncates x to an integer q(x) of quanta 2^(E_k - 100)
 * and adds q(x) and q(x)^2 as integers, so the totals are exact: they do not
 * depend on the order of addition or on how the trajectories were split, and the
 * mean and standard error formed from them (the variance of the quantised values,
 * exactly) are the same bits for one run, for any set of shards, and for any
 * order in which shards are combined (an integer all-reduce across GPUs
 * included).  The truncation moves a value by less than 2^-99 of the bound.
 *
 * Moment words: QTM_MOMENT_WORDS int64 per output value j * n_obs + k, laid out
 * [n_t * n_obs][QTM_MOMENT_WORDS]:
 *   [0..2]  sum of q(x)   as d0 + d1 2^48 + d2 2^96
 *   [3..7]  sum of q(x)^2 as d0 + d1 2^48 + ... + d4 2^192
 *   [8]     count of values that cannot be represented (NaN or Inf: a failed
 *           trajectory); a non-zero count makes that output's mean and SE NaN.
 * Word sets returned by the library have every digit but the last of each sum in
 * [0, 2^48), so up to 16384 of them add word by word in int64 without overflow.
 * ------------------------------------------------------------------------- */
#define QTM_MOMENT_WORDS 9

/* Moment words of the last run (HOST buffer of n_t * n_obs * QTM_MOMENT_WORDS),
 * its trajectory count, and the n_obs scale exponents (may be NULL).  Synchronises. */
qtm_status qtm_moments(qtm_ctx *ctx, int64_t *words, int64_t *count, int32_t *scale_exp);

/* Asynchronous copy of the same words into a caller-owned DEVICE buffer, ordered
 * on the context stream: the input of an integer sum all-reduce across GPUs (one
 * shard per GPU), which is exact and therefore independent of the collective's
 * reduction order. */
qtm_status qtm_moments_device(qtm_ctx *ctx, int64_t *words_dev);

/* Scale exponents E_k of the problem's n_obs observables (HOST output, n_obs
 * int32); reads only dim, n_obs and A.  Needs no GPU. */
qtm_status qtm_scale_exponents(const qtm_problem *problem, int32_t *scale_exp);

/* Moment words of per-trajectory values held on the HOST, [ntraj][n_values] with
 * n_values = n_t * n_obs (value p belongs to observable p % n_obs), by the same
 * rule as a run: for shards computed elsewhere (or checking).  Needs no GPU. */
qtm_status qtm_moments_of_values(const double *values, int64_t ntraj, int32_t n_values, int32_t n_obs,
                                 const int32_t *scale_exp, int64_t *words);

/* The master's average: adds the moment words of n_shards shards
 * (words: HOST, [n_shards][n_values][QTM_MOMENT_WORDS], in rank order, although
 * the integer sums make the order immaterial), counts[n_shards] trajectories each
 * (total <= 2^40), and writes the ensemble mean and, where not NULL, the standard
 * error (sample variance, n - 1 divisor), the sum and the sum of squares
 * (HOST, n_values doubles each).  Equal, bit for bit, to qtm_expect / qtm_sums of
 * one run over all the shards' trajectories.  Needs no GPU. */
qtm_status qtm_combine_moments(int32_t n_shards, int32_t n_values, int32_t n_obs, const int32_t *scale_exp,
                               const int64_t *words, const int64_t *counts, double *mean, double *stderr_out,
                               double *sum, double *sumsq);

/* Maximum scratch of qtm_ensemble_reduce_static, in doubles (4 MiB), and the
 * largest n_values it accepts. */
#define QTM_STATIC_SCRATCH_DOUBLES (1 << 19)
#define QTM_STATIC_MAX_VALUES (QTM_STATIC_SCRATCH_DOUBLES / 2)

/* Ensemble mean and standard error of per-trajectory values the caller already
 * holds on the device, computed without allocating any device memory.  The
 * paper has no counterpart: it exists for callers that may not let a library
 * allocate -- for example a host framework whose memory planner owns every
 * device buffer and only lends the library its inputs and outputs, or a
 * service that fixes its device footprint at start-up and must not grow it
 * while it runs.  qtm_run / qtm_expect allocate through their context; this
 * call does not (no cudaMalloc, no allocator hook, no library that allocates).
 *
 *   values_dev  DEVICE pointer, [ntraj][n_values] doubles (e.g. the layout of
 *               qtm_traj_expect: n_values = n_t * n_obs), read only.
 *   ntraj       >= 0 trajectories.
 *   n_values    1 .. QTM_STATIC_MAX_VALUES values per trajectory; larger sizes
 *               return QTM_ERR_ARG with a message in qtm_last_error(NULL).
 *   sum_dev, sumsq_dev, mean_dev, stderr_dev
 *               DEVICE pointers to n_values doubles each, written with the same
 *               quantities as qtm_sums and qtm_expect (sample variance, n - 1).
 *   cuda_stream the stream the work is ordered on (NULL = legacy default).
 *
 * Scratch: the per-segment partial sums live in one array of
 * QTM_STATIC_SCRATCH_DOUBLES doubles that is part of the library's device
 * image, so every GPU that loads the library holds those 4 MiB until the
 * process exits.  Every call on a device uses the same array: calls whose work
 * overlaps on the GPU (different streams without ordering between them) race
 * on it and give wrong results; order them on one stream.  Each call writes
 * every scratch element it reads before reading it, so nothing needs clearing
 * between calls.  The first call in each CUDA context -- on each device, and
 * again once a device's context has been destroyed and created anew (after
 * cudaDeviceReset, say) -- looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it for that
 * context, so make that first call before any stream capture on that device.
 * The call is asynchronous; results are ready when the stream reaches it. */
qtm_status qtm_ensemble_reduce_static(const double *values_dev, int64_t ntraj, int32_t n_values,
                                      double *sum_dev, double *sumsq_dev, double *mean_dev,
                                      double *stderr_dev, void *cuda_stream);

/* The per-trajectory values that Sec. 3 averages: Re<psi|A_k|psi>/<psi|psi> of
 * every trajectory of the last run at every output time, [traj][j][k]
 * (ntraj * n_t * n_obs doubles). */
qtm_status qtm_traj_expect(qtm_ctx *ctx, double *out);

/* The jumps of Algorithm 1 step (C) in the last run (needs QTM_FLAG_RECORD_JUMPS): n_jumps[ntraj] total
 * jumps per trajectory; jump_t / jump_ch [ntraj][max_jumps_recorded] hold the first
 * max_jumps_recorded jump times and channel indices (unused slots: NaN / -1). */
qtm_status qtm_jumps(qtm_ctx *ctx, int32_t *n_jumps, double *jump_t, int32_t *jump_ch);

/* ---------------------------------------------------------------------------
 * Learned jump-time proposal.  A small network (6 -> 64 -> 64 -> 1, SiLU, FP32)
 * predicts the time left until the trajectory's norm falls to its threshold r
 * (the crossing of Algorithm 1, step (B)) from cheap features of the state: the
 * decay rate Gamma = <sum_n C_n^dag C_n> (from the norm ratio over the last
 * step), its slope, <psi|psi>, log r, and the latest output values of the first
 * two observables.  Its output y corrects the constant-rate estimate:
 * time left = log(<psi|psi> / r) / Gamma * exp(y).  When enabled, a step that
 * would contain the predicted crossing is shortened to end a fraction `margin`
 * past it, so less of that step is discarded at the jump.  The exact root find
 * of the continuous extension still decides every jump; only the step sequence
 * changes (so results move by the integration tolerance, not more).  The paper
 * has no such component: it is the learned part of this library's design.
 *
 * Under the exponential method (qtm_set_method) the proposal acts inside the
 * crossing search instead: once an output interval is known to contain the
 * crossing, the features are taken over that interval (the decay rate from the
 * norms at its two ends, its change since the previous interval, the norm at
 * its start, log r, the latest two outputs), the network corrects the
 * constant-rate estimate of the crossing time, and the search first tries the
 * ladder bracket of width delta that holds the prediction -- formed with the
 * binary digits of its start, which are exactly the levels the plain descent
 * would keep -- and checks it with one product.  On a hit the crossing is found
 * from the same state, bit for bit, with fewer products; on a miss the plain
 * descent takes over (qtm_stats_t.proposal_misses counts them).  Pairs for this
 * use are collected by qtm_proposal_collect on a context that uses the
 * exponential method (one record per crossing).
 * Supported for QTM_PREC_C128 and QTM_PREC_DF64 at dimension <= 64 (the
 * single-warp lane layouts, where it is compiled into separate kernels so the
 * plain kernels carry none of it); other contexts get QTM_ERR_UNSUPPORTED from
 * qtm_proposal_collect and from qtm_proposal_enable(on != 0).
 * ------------------------------------------------------------------------- */

/* Floats of a network's parameter block: W1[64][6], b1[64], W2[64][64], b2[64],
 * w3[64], b3, feature means[6], feature scales[6]. */
#define QTM_PROPOSAL_FLOATS 4685

/* Runs trajectories 0 .. ntraj-1 of the plain method (proposal off) and records,
 * every `stride` accepted steps and at most max_per_traj times per trajectory,
 * the 6 raw features and the time left to the next jump; records of a
 * trajectory's last jump interval (no jump followed) are dropped.  Under the
 * exponential method a record is taken at every `stride`-th crossing, with the
 * features of the output interval that contains it and the time from the
 * interval's start to the crossing.  Keeps the
 * pairs for qtm_proposal_train; *npairs (may be NULL) = their number.
 * Synchronises; the run's observables are available as after qtm_run. */
qtm_status qtm_proposal_collect(qtm_ctx *ctx, int64_t ntraj, uint64_t seed, int32_t stride,
                                int32_t max_per_traj, int64_t *npairs);

/* Copies up to `capacity` collected pairs: features [capacity][6] (raw), dt [capacity]. */
qtm_status qtm_proposal_pairs(qtm_ctx *ctx, float *features, float *dt, int64_t capacity);

/* Trains the network on the collected pairs with the library's GPU kernels:
 * features standardised, targets y = log(dt / constant-rate estimate), mean
 * squared error, Adam (learning rate lr), `steps` minibatches of `batch` pairs of
 * a shuffled order (shuffle and Glorot initialisation from `seed`).  *loss (may
 * be NULL) = final mean squared error over all pairs; *loss_rate_estimate (may be
 * NULL) = the same error of the constant-rate estimate alone (y = 0). */
qtm_status qtm_proposal_train(qtm_ctx *ctx, int32_t steps, int32_t batch, float lr, uint64_t seed,
                              float *loss, float *loss_rate_estimate);

/* Loads / reads a parameter block of QTM_PROPOSAL_FLOATS floats (host memory). */
qtm_status qtm_proposal_set(qtm_ctx *ctx, const float *params);
qtm_status qtm_proposal_get(qtm_ctx *ctx, float *params);

/* Turns the proposal on (on != 0) or off for later runs; margin in (0, 1). */
qtm_status qtm_proposal_enable(qtm_ctx *ctx, int32_t on, float margin);

/* Mean squared error and its gradient with respect to the first 4673 parameters
 * for standardised inputs x[n][6] and targets t[n], computed by the training
 * kernels on the current device (host pointers; for checking the kernels). */
qtm_status qtm_mlp_loss_grad(const float *params, const float *x, const float *t, int64_t n, float *loss,
                             float *grad);

/* Counters of the last run (synchronises): accepted and rejected steps of
 * Algorithm 1 (B), products, jumps (C), root-find iterations. */
qtm_status qtm_stats(qtm_ctx *ctx, qtm_stats_t *out);

/* The error level of the paper's zvode_method_for_mc (Sec. 3) as text:
 * human-readable message of the last error of ctx (or of the last failed
 * qtm_create when ctx is NULL).  Never NULL; valid until the next call. */
const char *qtm_last_error(const qtm_ctx *ctx);

/* Name of a status code, e.g. "QTM_ERR_ARG" (plumbing; no counterpart in the paper). */
const char *qtm_status_string(qtm_status status);

/* Time-dependent Hamiltonian (Sec. 3: mpi_main accepts an extra function for a
 * time-dependent H, and the right-hand side sees the current time):
 *   H(t) = H + sum_k a_k cos(omega_k t + phi_k) H_k,   k < n_terms <= 8.
 * H: n_terms Hermitian operators of the context's dimension (HOST, copied);
 * coef: HOST, [n_terms][3] = a_k, omega_k, phi_k (finite).  Every right-hand-side
 * evaluation of a trajectory uses the time of its Dormand-Prince stage (and
 * t0 + h0 in the starting-step estimate); the collapse operators, observables and
 * the jump rule are unchanged.  n_terms = 0 removes the terms.  Applies to later
 * runs; QTM_ERR_UNSUPPORTED for QTM_PREC_BF16X6 (its operator is constant) or
 * when the operators no longer fit a kernel (reported by qtm_run). */
qtm_status qtm_set_drive(qtm_ctx *ctx, int32_t n_terms, const qtm_op *H, const double *coef);

/* No counterpart in the paper (failure detection of the tensor-core engine).
 * Bound (nanoseconds of wall clock) on any single device-side wait of the
 * tensor-core engine (QTM_PREC_BF16X6: its producer, tensor-core and TMA roles
 * hand tiles to one another through shared-memory barriers).  A wait that runs
 * past it ends the launch: every role winds down, the engine's device state is
 * released, and the next synchronising call returns QTM_ERR_TIMEOUT; the context
 * stays usable.  0 restores the default (2 s).  No effect on the other
 * arithmetics (their kernels have no cross-role waits). */
qtm_status qtm_set_wait_limit(qtm_ctx *ctx, uint64_t limit_ns);

/* The right-hand side of the trajectory equation (Sec. 2.2, Eq.
 * eqn:effective:hamiltonian) in batch: my[v] = M y[v] with M = -i H_eff, for n_vec vectors
 * y (HOST, [n_vec][dim] complex, interleaved (re, im) doubles; rounded to FP32)
 * through the tensor-core engine's product (QTM_PREC_BF16X6 contexts only;
 * QTM_ERR_UNSUPPORTED otherwise).  my: HOST, [n_vec][dim] complex.  Runs on the
 * context stream and synchronises it; leaves the results of qtm_run untouched. */
qtm_status qtm_rhs_batch(qtm_ctx *ctx, int64_t n_vec, const double *y, double *my);

/* ---------------------------------------------------------------------------
 * Exponential propagation for stiff problems.  Sec. 2.1 of the paper lets the
 * user switch ZVODE from Adams to BDF when the trajectory equations are stiff
 * (rates of H_eff spread over decades, so that an explicit integrator's step is
 * limited by stability, not accuracy).  With a constant Hamiltonian the no-jump
 * evolution dpsi/dt = M psi (M = -i H_eff) has the exact solution
 * psi(t) = exp(M (t - t_k)) psi_k, which this method applies instead of
 * integrating:
 *   - at qtm_set_method the library computes, in FP64 on the host, the ladder
 *     P_l = exp(M delta 2^l), l = 0..L, by scaling and squaring (Taylor degree
 *     12 at nu delta <= 1/16, nu = max(||M||_1, ||M||_inf)), with delta 2^L the
 *     output spacing (uniform grids) or the largest output interval;
 *   - a trajectory moves from output to output with one dense product P_L psi
 *     (uniform grids) or with the binary digits of the interval in units of
 *     delta plus a Taylor remainder (degree 9; degree 5 for the FP32 state of
 *     QTM_PREC_C64 and QTM_PREC_BF16X6, whose truncation is then below 8.3e-11);
 *   - the squared norm cannot increase (d||psi||^2/dt = -sum_n ||C_n psi||^2),
 *     so a jump happened before t_j exactly when ||psi(t_j)||^2 < r (Algorithm 1
 *     (B)); the crossing is then bracketed within delta by a binary descent over
 *     the ladder and solved by Newton's method on the Taylor polynomial of
 *     exp(s M) psi (to 1e-15 max(1, |t|));
 *   - steps (C) and (D) are those of the default method.
 * Results differ from the exact trajectory by rounding and the root tolerance
 * only (rtol and atol are not used), at a cost that does not depend on the
 * stiffness.  Counters (qtm_stats) under this method: accepted = propagations
 * ending at an output or a jump, rejected = ladder levels that overshot a
 * crossing, rhs_evals = matrix-vector products (ladder levels and M),
 * root_iters = Newton iterations.
 * ------------------------------------------------------------------------- */

/* Selects the method of later runs.  QTM_METHOD_EXPONENTIAL computes and uploads
 * the ladder (host FP64, O(L n^3 + 12 nnz(M) n) operations; (L + 1) n^2 complex
 * values of device memory, rounded to the context's arithmetic) and needs
 * dimension <= 256 and no time-dependent terms (QTM_ERR_UNSUPPORTED otherwise),
 * in any arithmetic:
 *   QTM_PREC_C128, QTM_PREC_DF64, QTM_PREC_C64 (FP32 propagators and state,
 *     double-float norms: a trajectory's jump times move by about the FP32
 *     rounding accumulated over the products) -- one trajectory per lane group;
 *   QTM_PREC_BF16X6 -- all trajectories of a run in lock step, which needs a
 *     uniform output grid (QTM_ERR_UNSUPPORTED otherwise): per output interval
 *     one tensor-core product forms (P_L - I) psi for every trajectory (the
 *     engine's BF16x6 split, FP32 accumulation; the library adds psi in FP32),
 *     and a per-interval kernel records the outputs; a trajectory whose norm
 *     crosses its threshold inside the interval waits for a catch-up launch
 *     (every sixteen intervals and after the last) that runs its crossing search,
 *     jump and propagation in complex64 and the intervals it missed, after which
 *     it rejoins.  Device memory per run: two FP32 state blocks of
 *     ntraj x 2 x (dim rounded up to 64) values, 100 bytes per trajectory.
 *     qtm_stats reports one product launch's device time (product_ms).
 * The learned proposal works with it on the contexts that support the proposal
 * (complex128 or double-float, dimension <= 64; see above).  QTM_METHOD_DOPRI5
 * restores the default (for QTM_PREC_BF16X6 the Dormand-Prince tensor-core
 * engine).  QTM_ERR_ARG for any other value. */
qtm_status qtm_set_method(qtm_ctx *ctx, int32_t method);

/* The exponential method's ladder (exp(M delta 2^l), the no-jump evolution of
 * Sec. 2.2 over powers of two of a base step): number of levels L + 1 and the base step
 * delta (either pointer may be NULL).  QTM_ERR_STATE when the context does not
 * use the exponential method. */
qtm_status qtm_expo_ladder(const qtm_ctx *ctx, int32_t *levels, double *delta);

/* The no-jump propagator of Sec. 2.2: exp(M dt) for the problem's
 * M = -i H - (1/2) sum_n C_n^dag C_n (only dim, H,
 * n_c and C are read; HOST pointers), dt >= 0, by the same scaling and squaring
 * as the exponential method's ladder.  out: HOST, n x n complex, row-major,
 * interleaved (re, im).  Needs no GPU; the message of an error is available
 * from qtm_last_error(NULL). */
qtm_status qtm_propagator(const qtm_problem *problem, double dt, double *out);

/* ---------------------------------------------------------------------------
 * Arithmetic peaks of the current GPU, for the roofline fractions of the
 * trajectory kernels (whose state never leaves the SM, so arithmetic bounds
 * them).  The paper has no counterpart: this measures the machine.
 * ------------------------------------------------------------------------- */
enum {
    QTM_PEAK_FP64 = 0,  /* FP64 fused multiply-adds (the complex128 path's pipe) */
    QTM_PEAK_FP32 = 1,  /* FP32 fused multiply-adds (the complex64 path's pipe) */
    QTM_PEAK_DF64 = 2   /* double-float multiply-adds as the double-float path forms them
                           (12 FP32 instructions each), counted as two FP64-class flops */
};

/* Launches (asynchronously, on cuda_stream) one probe kernel of `kind`: a grid
 * that fills every SM, each thread running 8 independent multiply-add chains of
 * `iters` steps (>= 1).  scratch_dev: a DEVICE buffer of at least 8 bytes (never
 * written in practice; it keeps the chains from being optimised away).  *flop =
 * the launch's flops (2 per multiply-add); the caller times the launch with
 * events on the same stream. */
qtm_status qtm_arith_peak_launch(int32_t kind, int64_t iters, void *scratch_dev, void *cuda_stream, double *flop);

/* Releases the context's device memory (after synchronising its stream); the end
 * of mpi_main's run (Sec. 3).  NULL is ignored. */
void qtm_destroy(qtm_ctx *ctx);

/* Library version string, e.g. "0.1.0 sm_103a" (no counterpart in the paper). */
const char *qtm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QTM_H */
