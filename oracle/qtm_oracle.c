/*
 * qtm_oracle.c -- plain, slow, FP64 CPU oracle for the Monte Carlo wave-function
 * (quantum trajectories) method of Sawerwain & Wisniewska, "QTM: computational
 * package using MPI protocol for quantum trajectories method" (arXiv 1810.03047).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is compared
 * against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may build, load or call it; the library never does.  It shares no code,
 * header, table or helper with the CUDA path: the Dormand-Prince coefficients, the
 * Philox generator and every step of the trajectory are written out here again,
 * from their publications, in the simplest form that is still fast enough to run
 * a few thousand trajectories in seconds.
 *
 * What it computes (one function per item, each citing what it follows):
 *   - the effective Hamiltonian H_eff = H - (i/2) sum_n C_n^dag C_n (Sec. 2.2,
 *     Eq. eqn:effective:hamiltonian), stored as M = -i H_eff so that the
 *     trajectory ODE reads dpsi/dt = M psi (hbar = 1, as in the Sec. 4.1 listing);
 *   - the random stream: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed
 *     (seed, 0) with counter (jump index k, trajectory id, 0, 0); it stands in for
 *     the LFSR113 generator of Sec. 2.3 so that every trajectory's draws are
 *     addressable by (seed, trajectory, jump);
 *   - the explicit Dormand-Prince 5(4) pair with its 4th-order continuous
 *     extension (Dormand & Prince 1980; Hairer, Norsett & Wanner, Solving ODEs I,
 *     Sec. II.4-II.6), which replaces the ZVODE solver of Sec. 2.1;
 *   - one trajectory, Algorithm 1 steps (A)-(D) of Sec. 2.2: a threshold r,
 *     integration under H_eff while <psi|psi> >= r, location of the crossing time,
 *     channel choice by the cumulative probabilities of Eq. eqn:probability:of:cn,
 *     the jump of Eq. eqn:state:for:new:time, a new r, continue from that time;
 *   - the observables Re<psi|A|psi>/<psi|psi> at the output times and their
 *     average over trajectories (Sec. 3, averaging of trajectories);
 *   - a companion Lindblad master-equation integrator (Sec. 2.2, Eq. for
 *     rho-dot) used to check the ensemble statistics on small systems;
 *   - optionally a time-dependent Hamiltonian H(t) = H + sum_k f_k(t) H_k with
 *     f_k(t) = a_k cos(omega_k t + phi_k) (Sec. 3: mpi_main takes an extra
 *     function for a time-dependent Hamiltonian, and the right-hand side sees the
 *     current time); every right-hand-side evaluation uses the time of its stage.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous on them):
 *   - step (C) draws a fresh uniform c_k for the channel instead of re-using r;
 *   - P_i = w_i / sum_j w_j with w_i = ||C_i psi||^2 at the (unnormalised) jump
 *     state, and the jump divides by ||C_n psi|| of that state;
 *   - the jump happens at the first time ||psi||^2 equals r on the step's dense
 *     output; output times at or before it use the pre-jump state;
 *   - r and c are in the open interval (0, 1).
 *
 * Parity with the CUDA path is exact up to rounding only because both follow the
 * same published algorithm with the same step-size controller, initial step and
 * output rules; none of those is shared code.
 */

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------------------
 * Public structures (mirrored by ctypes in oracle.py)
 * ------------------------------------------------------------------------- */

typedef struct {
    int32_t n;               /* rows (= columns) */
    const int32_t *row_ptr;  /* n + 1 */
    const int32_t *col;      /* nnz */
    const double *val;       /* 2 * nnz, (re, im) interleaved */
} orc_op;

typedef struct {
    int32_t dim;
    orc_op H;
    int32_t n_c;
    const orc_op *C;
    int32_t n_obs;
    const orc_op *A;
    const double *psi0;      /* 2 * dim */
    int32_t n_t;
    const double *t;         /* n_t, strictly increasing */
    double rtol, atol;
    int64_t max_steps;       /* attempted steps per trajectory */
    int32_t n_drive;         /* time-dependent terms (0: H is constant) */
    const orc_op *drive;     /* n_drive Hermitian H_k */
    const double *drive_coef;/* 3 * n_drive: a_k, omega_k, phi_k of f_k(t) = a_k cos(omega_k t + phi_k) */
} orc_problem;

typedef struct {
    double *obs_re;          /* ntraj * n_t * n_obs, required */
    double *obs_im;          /* same shape, may be NULL */
    int32_t max_jumps;       /* capacity per trajectory of the jump arrays below */
    int32_t *n_jumps;        /* ntraj, may be NULL */
    double *jump_t;          /* ntraj * max_jumps, may be NULL */
    int32_t *jump_ch;        /* ntraj * max_jumps, may be NULL */
    double *jump_norm;       /* ntraj * max_jumps: ||psi||^2 right after each jump, may be NULL */
    int32_t *status;         /* ntraj, may be NULL */
    int64_t *counts;         /* ntraj * 4: accepted, rejected, rhs evaluations, jumps; may be NULL */
} orc_result;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_MAXSTEPS = 4, ORC_ERR_STEPSIZE = 5,
       ORC_ERR_NONFINITE = 6, ORC_ERR_NO_CHANNEL = 7, ORC_ERR_NOMEM = 3 };

/* ---------------------------------------------------------------------------
 * Sparse complex matrices (CSR, the storage of Sec. 2.2 / Sec. 3)
 * ------------------------------------------------------------------------- */

typedef struct {
    int n;
    int *row_ptr;
    int *col;
    cplx *val;
} csr;

static void csr_free(csr *a)
{
    free(a->row_ptr);
    free(a->col);
    free(a->val);
    memset(a, 0, sizeof(*a));
}

static int csr_from_op(const orc_op *op, csr *out)
{
    int n = op->n, nnz = op->row_ptr[op->n];
    out->n = n;
    out->row_ptr = malloc(sizeof(int) * (size_t)(n + 1));
    out->col = malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    out->val = malloc(sizeof(cplx) * (size_t)(nnz > 0 ? nnz : 1));
    if (!out->row_ptr || !out->col || !out->val) return ORC_ERR_NOMEM;
    for (int i = 0; i <= n; i++) out->row_ptr[i] = op->row_ptr[i];
    for (int k = 0; k < nnz; k++) {
        out->col[k] = op->col[k];
        out->val[k] = op->val[2 * k] + I * op->val[2 * k + 1];
    }
    return ORC_OK;
}

/* dense n x n (row-major) -> CSR, dropping exact zeros */
static int csr_from_dense(int n, const cplx *d, csr *out)
{
    int nnz = 0;
    for (int i = 0; i < n * n; i++) nnz += (d[i] != 0.0);
    out->n = n;
    out->row_ptr = malloc(sizeof(int) * (size_t)(n + 1));
    out->col = malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    out->val = malloc(sizeof(cplx) * (size_t)(nnz > 0 ? nnz : 1));
    if (!out->row_ptr || !out->col || !out->val) return ORC_ERR_NOMEM;
    int k = 0;
    for (int i = 0; i < n; i++) {
        out->row_ptr[i] = k;
        for (int j = 0; j < n; j++) {
            cplx v = d[(size_t)i * n + j];
            if (v != 0.0) {
                out->col[k] = j;
                out->val[k] = v;
                k++;
            }
        }
    }
    out->row_ptr[n] = k;
    return ORC_OK;
}

/* y = A x */
static void csr_mv(const csr *a, const cplx *x, cplx *y)
{
    for (int i = 0; i < a->n; i++) {
        cplx s = 0.0;
        for (int k = a->row_ptr[i]; k < a->row_ptr[i + 1]; k++) s += a->val[k] * x[a->col[k]];
        y[i] = s;
    }
}

static double norm2(int n, const cplx *x)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    return s;
}

/* <x|y> */
static cplx inner(int n, const cplx *x, const cplx *y)
{
    cplx s = 0.0;
    for (int i = 0; i < n; i++) s += conj(x[i]) * y[i];
    return s;
}

/* ---------------------------------------------------------------------------
 * Effective Hamiltonian, Sec. 2.2 Eq. eqn:effective:hamiltonian:
 *   H_eff = H - (i/2) sum_n C_n^dag C_n   (hbar = 1)
 * The trajectory right-hand side is M psi with M = -i H_eff
 *   = -i H - (1/2) sum_n C_n^dag C_n,
 * which is the matrix the Sec. 4.1 listing stores in its array "H".
 * Formed densely: (C^dag C)_{ij} = sum_k conj(C_{ki}) C_{kj}.
 * ------------------------------------------------------------------------- */

static int effective_matrix_dense(const orc_problem *p, cplx *M)
{
    int n = p->dim;
    memset(M, 0, sizeof(cplx) * (size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int k = p->H.row_ptr[i]; k < p->H.row_ptr[i + 1]; k++) {
            cplx h = p->H.val[2 * k] + I * p->H.val[2 * k + 1];
            M[(size_t)i * n + p->H.col[k]] += -I * h;
        }
    for (int c = 0; c < p->n_c; c++) {
        const orc_op *C = &p->C[c];
        for (int k = 0; k < n; k++) /* row k of C contributes conj(C_ki) C_kj */
            for (int a = C->row_ptr[k]; a < C->row_ptr[k + 1]; a++) {
                cplx cki = C->val[2 * a] + I * C->val[2 * a + 1];
                int i = C->col[a];
                for (int b = C->row_ptr[k]; b < C->row_ptr[k + 1]; b++) {
                    cplx ckj = C->val[2 * b] + I * C->val[2 * b + 1];
                    M[(size_t)i * n + C->col[b]] += -0.5 * conj(cki) * ckj;
                }
            }
    }
    return ORC_OK;
}

int orc_effective_matrix(const orc_problem *p, double *M_out /* 2*n*n */)
{
    if (!p || p->dim <= 0 || !M_out) return ORC_ERR_ARG;
    cplx *M = malloc(sizeof(cplx) * (size_t)p->dim * p->dim);
    if (!M) return ORC_ERR_NOMEM;
    effective_matrix_dense(p, M);
    memcpy(M_out, M, sizeof(cplx) * (size_t)p->dim * p->dim);
    free(M);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Philox4x64-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  Round: two 64x64->128 products of the counter words 0 and 2 with the
 * published multipliers; the high halves are xored with counter words 1 and 3 and
 * the key; the key is bumped by the published Weyl constants between rounds.
 * ------------------------------------------------------------------------- */

#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* 53 random bits -> a double in the open interval (0, 1) */
static double u01_open(uint64_t w)
{
    return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

/* The draws of Algorithm 1 for jump index k of trajectory traj: r_k (the
 * threshold of steps (A)/(D)) and c_k (the channel draw of step (C)). */
void orc_uniforms(uint64_t seed, int64_t traj, int64_t k, double *r, double *c)
{
    uint64_t ctr[4] = {(uint64_t)k, (uint64_t)traj, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t w[4];
    orc_philox4x64_10(ctr, key, w);
    *r = u01_open(w[0]);
    *c = u01_open(w[1]);
}

/* ---------------------------------------------------------------------------
 * Dormand-Prince 5(4), 7 stages, first-same-as-last (Dormand & Prince 1980;
 * Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.5, Table 5.2).
 * ------------------------------------------------------------------------- */

static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0},
    {1.0 / 5.0},
    {3.0 / 40.0, 9.0 / 40.0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0},
};
/* 5th-order weights (= last row of A, the FSAL property) and the 4th-order ones */
static const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0,
                               -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double DP_BHAT[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                  -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

/* Continuous extension of order 4 (Hairer, Norsett & Wanner, Sec. II.6, the
 * dense output of DOPRI5): y(t + theta h) = y + h sum_j b_j(theta) k_j with
 *   b_j(theta) = theta^2 (3 - 2 theta) b_j + theta^2 (theta-1)^2 * d_j(theta)
 * plus theta (theta-1)^2 for j = 1 and theta^2 (theta-1) for j = 7. */
static void dp_dense_weights(double th, double w[7])
{
    double th2 = th * th;
    double p = th2 * (3.0 - 2.0 * th);
    double q = th2 * (th - 1.0) * (th - 1.0);
    w[0] = p * DP_B[0] + th * (th - 1.0) * (th - 1.0)
         - q * 5.0 * (2558722523.0 - 31403016.0 * th) / 11282082432.0;
    w[1] = 0.0;
    w[2] = p * DP_B[2] + q * 100.0 * (882725551.0 - 15701508.0 * th) / 32700410799.0;
    w[3] = p * DP_B[3] - q * 25.0 * (443332067.0 - 31403016.0 * th) / 1880347072.0;
    w[4] = p * DP_B[4] + q * 32805.0 * (23143187.0 - 3489224.0 * th) / 199316789632.0;
    w[5] = p * DP_B[5] - q * 55.0 * (29972135.0 - 7076736.0 * th) / 822651844.0;
    w[6] = th2 * (th - 1.0) + q * 10.0 * (7414447.0 - 829305.0 * th) / 29380423.0;
}

typedef void (*rhs_fn)(void *ctx, double t, const cplx *y, cplx *dy);

/* One attempted step of size h from (t, y) with K[0] = f(t, y) already known.
 * Fills K[1..6] (K[s] = f(t + c_s h, y_s), K[6] = f(t + h, ynew)), ynew, and
 * returns the scaled RMS error norm
 *   sqrt( (1/n) sum_i |e_i|^2 / sc_i^2 ),  e = h sum_j (b_j - bhat_j) k_j,
 *   sc_i = atol + rtol max(|y_i|, |ynew_i|)   (HNW Sec. II.4, Eq. (4.10)-(4.11)). */
static double dp_step(int n, rhs_fn f, void *ctx, double t, const cplx *y, cplx *K[7], double h,
                      cplx *ynew, cplx *ytmp, double rtol, double atol)
{
    for (int s = 1; s < 7; s++) {
        cplx *ys = (s == 6) ? ynew : ytmp;
        for (int i = 0; i < n; i++) {
            cplx acc = 0.0;
            for (int j = 0; j < s; j++) acc += DP_A[s][j] * K[j][i];
            ys[i] = y[i] + h * acc;
        }
        f(ctx, t + DP_C[s] * h, ys, K[s]);
    }
    double sum = 0.0;
    for (int i = 0; i < n; i++) {
        cplx e = 0.0;
        for (int j = 0; j < 7; j++) e += (DP_B[j] - DP_BHAT[j]) * K[j][i];
        e *= h;
        double ay = sqrt(creal(y[i]) * creal(y[i]) + cimag(y[i]) * cimag(y[i]));
        double an = sqrt(creal(ynew[i]) * creal(ynew[i]) + cimag(ynew[i]) * cimag(ynew[i]));
        double sc = atol + rtol * (ay > an ? ay : an);
        sum += (creal(e) * creal(e) + cimag(e) * cimag(e)) / (sc * sc);
    }
    return sqrt(sum / n);
}

/* y(t + theta h) from the continuous extension */
static void dp_dense(int n, const cplx *y, cplx *K[7], double h, double theta, cplx *out)
{
    double w[7];
    dp_dense_weights(theta, w);
    for (int i = 0; i < n; i++) {
        cplx acc = 0.0;
        for (int j = 0; j < 7; j++) acc += w[j] * K[j][i];
        out[i] = y[i] + h * acc;
    }
}

/* Starting step size (HNW Sec. II.4, "Starting step size", with p = 4):
 * h0 from ||y0|| / ||f0||, one explicit Euler step to estimate the second
 * derivative, h1 = (0.01 / max(d1, d2))^(1/5), h = min(100 h0, h1). */
static double dp_initial_step(int n, rhs_fn f, void *ctx, double t0, const cplx *y0, const cplx *f0,
                              double span, double rtol, double atol, cplx *y1, cplx *f1,
                              int64_t *rhs_count)
{
    double d0 = 0.0, d1 = 0.0;
    for (int i = 0; i < n; i++) {
        double ay = sqrt(creal(y0[i]) * creal(y0[i]) + cimag(y0[i]) * cimag(y0[i]));
        double sc = atol + rtol * ay;
        d0 += (creal(y0[i]) * creal(y0[i]) + cimag(y0[i]) * cimag(y0[i])) / (sc * sc);
        d1 += (creal(f0[i]) * creal(f0[i]) + cimag(f0[i]) * cimag(f0[i])) / (sc * sc);
    }
    d0 = sqrt(d0 / n);
    d1 = sqrt(d1 / n);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    if (h0 > span) h0 = span;
    for (int i = 0; i < n; i++) y1[i] = y0[i] + h0 * f0[i];
    f(ctx, t0 + h0, y1, f1);
    (*rhs_count)++;
    double d2 = 0.0;
    for (int i = 0; i < n; i++) {
        double ay = sqrt(creal(y0[i]) * creal(y0[i]) + cimag(y0[i]) * cimag(y0[i]));
        double sc = atol + rtol * ay;
        cplx df = f1[i] - f0[i];
        d2 += (creal(df) * creal(df) + cimag(df) * cimag(df)) / (sc * sc);
    }
    d2 = sqrt(d2 / n) / h0;
    double dm = d1 > d2 ? d1 : d2;
    double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
    double h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
    if (h > span) h = span;
    return h;
}

/* Step-size controller constants (HNW Sec. II.4, Eq. (4.13)): safety 0.9,
 * factor clamped to [0.2, 10], exponent 1/5; no growth right after a rejection. */
#define DP_SAFETY 0.9
#define DP_FACMIN 0.2
#define DP_FACMAX 10.0

/* ---------------------------------------------------------------------------
 * Test hooks for the integrator alone: dy/dt = M y with dense M.
 * ------------------------------------------------------------------------- */

typedef struct {
    int n;
    const cplx *M;
} dense_ctx;

static void dense_rhs(void *vctx, double t, const cplx *y, cplx *dy)
{
    const dense_ctx *c = vctx;
    for (int i = 0; i < c->n; i++) {
        cplx s = 0.0;
        for (int j = 0; j < c->n; j++) s += c->M[(size_t)i * c->n + j] * y[j];
        dy[i] = s;
    }
}

/* nsteps fixed steps of size h from y0; returns y(nsteps h) in y_out, the last
 * step's error estimate vector h sum (b - bhat) k in err_out (may be NULL), and,
 * if y_dense is given, the continuous extension at theta inside the last step. */
int orc_dopri5_fixed(int n, const double *M, const double *y0, double h, int nsteps,
                     double theta, double *y_out, double *err_out, double *y_dense)
{
    if (n <= 0 || nsteps <= 0) return ORC_ERR_ARG;
    dense_ctx ctx = {n, (const cplx *)M};
    cplx *buf = calloc((size_t)n * 10, sizeof(cplx));
    if (!buf) return ORC_ERR_NOMEM;
    cplx *y = buf, *ynew = buf + n, *ytmp = buf + 2 * n, *K[7];
    for (int j = 0; j < 7; j++) K[j] = buf + (size_t)(3 + j) * n;
    memcpy(y, y0, sizeof(cplx) * n);
    for (int s = 0; s < nsteps; s++) {
        dense_rhs(&ctx, 0.0, y, K[0]);
        dp_step(n, dense_rhs, &ctx, 0.0, y, K, h, ynew, ytmp, 1.0, 1.0);
        if (s == nsteps - 1) {
            if (err_out) {
                cplx *e = (cplx *)err_out;
                for (int i = 0; i < n; i++) {
                    cplx acc = 0.0;
                    for (int j = 0; j < 7; j++) acc += (DP_B[j] - DP_BHAT[j]) * K[j][i];
                    e[i] = h * acc;
                }
            }
            if (y_dense) dp_dense(n, y, K, h, theta, (cplx *)y_dense);
        }
        memcpy(y, ynew, sizeof(cplx) * n);
    }
    memcpy(y_out, y, sizeof(cplx) * n);
    free(buf);
    return ORC_OK;
}

void orc_dense_weights(double theta, double w[7]) { dp_dense_weights(theta, w); }

/* ---------------------------------------------------------------------------
 * One trajectory: Algorithm 1 of Sec. 2.2.
 * ------------------------------------------------------------------------- */

typedef struct {
    int n;
    csr M;       /* -i H_eff */
    int n_c;
    csr *C;
    int n_obs;
    csr *A;
    cplx *psi0;  /* normalised */
    int n_drive;
    csr *D;      /* -i H_k of the time-dependent terms */
    const orc_problem *p;
} model;

/* The right-hand side's context: the shared, read-only model and this
 * thread's scratch vector for the time-dependent terms. */
typedef struct {
    const model *m;
    cplx *dtmp;
} rhs_ctx;

/* f_k(t) = a_k cos(omega_k t + phi_k) */
static double drive_coef(const orc_problem *p, int k, double t)
{
    const double *c = p->drive_coef + 3 * k;
    return c[0] * cos(c[1] * t + c[2]);
}

/* dpsi/dt = M psi + sum_k f_k(t) (-i H_k) psi */
static void model_rhs(void *vctx, double t, const cplx *y, cplx *dy)
{
    const rhs_ctx *c = vctx;
    const model *m = c->m;
    csr_mv(&m->M, y, dy);
    for (int k = 0; k < m->n_drive; k++) {
        double f = drive_coef(m->p, k, t);
        csr_mv(&m->D[k], y, c->dtmp);
        for (int i = 0; i < m->n; i++) dy[i] += f * c->dtmp[i];
    }
}

typedef struct {
    cplx *psi, *ynew, *ytmp, *K[7], *yd, *cy, *ay, *dtmp;
} workspace;

/* Re and Im of <y|A_k|y>/<y|y> at output time index j */
static void record_outputs(const model *m, const cplx *y, cplx *ay, int j, double *obs_re,
                           double *obs_im)
{
    double nn = norm2(m->n, y);
    for (int k = 0; k < m->n_obs; k++) {
        csr_mv(&m->A[k], y, ay);
        cplx e = inner(m->n, y, ay) / nn;
        obs_re[(size_t)j * m->n_obs + k] = creal(e);
        if (obs_im) obs_im[(size_t)j * m->n_obs + k] = cimag(e);
    }
}

/* g(theta) = ||y(t + theta h)||^2 - r on the step's continuous extension */
static double crossing_fn(const model *m, workspace *w, double h, double theta, double r)
{
    dp_dense(m->n, w->psi, w->K, h, theta, w->yd);
    return norm2(m->n, w->yd) - r;
}

/* First theta in (0, 1] with ||y(theta)||^2 = r: the first of the eight
 * sub-intervals [(i-1)/8, i/8] whose right end lies below r brackets it; plain
 * bisection then shrinks the bracket to 1e-15 (in units of the step). */
static double locate_crossing(const model *m, workspace *w, double h, double r, int64_t *iters)
{
    double lo = 0.0, hi = 1.0;
    int found = 0;
    for (int i = 1; i <= 8; i++) {
        double th = i / 8.0;
        if (crossing_fn(m, w, h, th, r) < 0.0) {
            lo = (i - 1) / 8.0;
            hi = th;
            found = 1;
            break;
        }
    }
    if (!found) return 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15; it++) {
        double mid = 0.5 * (lo + hi);
        (*iters)++;
        if (crossing_fn(m, w, h, mid, r) < 0.0)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

typedef struct {
    double *obs_re, *obs_im;          /* n_t * n_obs for this trajectory */
    int32_t max_jumps;
    int32_t *n_jumps;
    double *jump_t, *jump_norm;
    int32_t *jump_ch;
    int64_t counts[4];                /* accepted, rejected, rhs, jumps */
    double *trace;                    /* test hook: (t, h, accepted) of every attempt, or NULL */
    int64_t max_trace, n_trace;
} traj_out;

static int run_trajectory(const model *m, uint64_t seed, int64_t traj, workspace *w, traj_out *o)
{
    const orc_problem *p = m->p;
    const int n = m->n, n_t = p->n_t;
    const double t_end = p->t[n_t - 1];
    const double rtol = p->rtol, atol = p->atol;
    int64_t attempts = 0, accepted = 0, rejected = 0, rhs = 0, jumps = 0, root_iters = 0;
    int status = ORC_OK;

    /* (A): the first threshold r_0 (and channel draw c_0) */
    int64_t k = 0;
    double r, c;
    orc_uniforms(seed, traj, k, &r, &c);

    double t = p->t[0];
    memcpy(w->psi, m->psi0, sizeof(cplx) * n);
    record_outputs(m, w->psi, w->ay, 0, o->obs_re, o->obs_im);
    int j = 1; /* next output index */

    rhs_ctx rc = {m, w->dtmp};
    model_rhs(&rc, t, w->psi, w->K[0]);
    rhs++;
    double h = dp_initial_step(n, model_rhs, &rc, t, w->psi, w->K[0], t_end - t, rtol, atol,
                               w->ytmp, w->ynew, &rhs);
    int rejected_before = 0;

    while (j < n_t) {
        /* a remaining span below rounding of t_end: the state is final */
        if (t_end - t <= 4.0 * 2.220446049250313e-16 * fabs(t_end)) {
            for (; j < n_t; j++) record_outputs(m, w->psi, w->ay, j, o->obs_re, o->obs_im);
            break;
        }
        if (attempts >= p->max_steps) { status = ORC_ERR_MAXSTEPS; break; }
        int last = 0;
        if (t + 1.01 * h >= t_end) {
            h = t_end - t;
            last = 1;
        }
        if (h < 1e-14 * fmax(1.0, fabs(t))) { status = ORC_ERR_STEPSIZE; break; }

        /* (B): integrate dpsi/dt = -i H_eff psi over [t, t + h] */
        double err = dp_step(n, model_rhs, &rc, t, w->psi, w->K, h, w->ynew, w->ytmp, rtol, atol);
        rhs += 6;
        attempts++;
        if (o->trace && o->n_trace < o->max_trace) {
            double *q = o->trace + 3 * o->n_trace++;
            q[0] = t;
            q[1] = h;
            q[2] = err <= 1.0 ? 1.0 : 0.0;
        }
        if (!(err <= 1.0)) {
            if (!isfinite(err)) { status = ORC_ERR_NONFINITE; break; }
            double fac = DP_SAFETY * pow(err, -0.2);
            if (fac < DP_FACMIN) fac = DP_FACMIN;
            h *= fac;
            rejected_before = 1;
            rejected++;
            continue;
        }
        accepted++;
        double t_new = last ? t_end : t + h;
        double n_new = norm2(n, w->ynew);

        if (n_new < r) {
            /* (B) ends: <psi|psi> fell to r inside this step; find that time */
            double th = locate_crossing(m, w, h, r, &root_iters);
            double tau = t + th * h;
            if (tau > t_new) tau = t_new;
            for (; j < n_t && p->t[j] <= tau; j++) {
                double thj = (p->t[j] - t) / h;
                if (thj > 1.0) thj = 1.0;
                dp_dense(n, w->psi, w->K, h, thj, w->yd);
                record_outputs(m, w->yd, w->ay, j, o->obs_re, o->obs_im);
            }
            dp_dense(n, w->psi, w->K, h, th, w->yd);

            /* (C): channel n* = min{n : sum_{i<=n} P_i >= c}, P_i = w_i / sum w */
            double wsum = 0.0;
            double wts[64];
            double *wt = m->n_c <= 64 ? wts : malloc(sizeof(double) * m->n_c);
            for (int q = 0; q < m->n_c; q++) {
                csr_mv(&m->C[q], w->yd, w->cy);
                wt[q] = norm2(n, w->cy);
                wsum += wt[q];
            }
            if (!(wsum > 0.0)) {
                if (wt != wts) free(wt);
                status = ORC_ERR_NO_CHANNEL;
                break;
            }
            double target = c * wsum, cum = 0.0;
            int ch = m->n_c - 1;
            for (int q = 0; q < m->n_c; q++) {
                cum += wt[q];
                if (cum >= target) { ch = q; break; }
            }
            /* the jump of Eq. eqn:state:for:new:time: psi <- C_n psi / ||C_n psi|| */
            csr_mv(&m->C[ch], w->yd, w->cy);
            double nc = sqrt(wt[ch]);
            for (int i = 0; i < n; i++) w->psi[i] = w->cy[i] / nc;
            if (wt != wts) free(wt);
            if (jumps < o->max_jumps) {
                if (o->jump_t) o->jump_t[jumps] = tau;
                if (o->jump_ch) o->jump_ch[jumps] = ch;
                if (o->jump_norm) o->jump_norm[jumps] = norm2(n, w->psi);
            }
            jumps++;

            /* (D): a new threshold; continue from tau with the step size just accepted */
            k++;
            orc_uniforms(seed, traj, k, &r, &c);
            t = tau;
            model_rhs(&rc, t, w->psi, w->K[0]);
            rhs++;
            rejected_before = 0;
            continue;
        }

        for (; j < n_t && p->t[j] <= t_new; j++) {
            double thj = (p->t[j] - t) / h;
            if (thj > 1.0) thj = 1.0;
            dp_dense(n, w->psi, w->K, h, thj, w->yd);
            record_outputs(m, w->yd, w->ay, j, o->obs_re, o->obs_im);
        }
        double fac = (err == 0.0) ? DP_FACMAX : DP_SAFETY * pow(err, -0.2);
        if (fac > DP_FACMAX) fac = DP_FACMAX;
        if (fac < DP_FACMIN) fac = DP_FACMIN;
        if (rejected_before && fac > 1.0) fac = 1.0;
        rejected_before = 0;
        t = t_new;
        memcpy(w->psi, w->ynew, sizeof(cplx) * n);
        memcpy(w->K[0], w->K[6], sizeof(cplx) * n); /* first same as last */
        h *= fac;
    }
    if (status != ORC_OK)
        for (; j < n_t; j++)
            for (int q = 0; q < m->n_obs; q++) {
                o->obs_re[(size_t)j * m->n_obs + q] = NAN;
                if (o->obs_im) o->obs_im[(size_t)j * m->n_obs + q] = NAN;
            }
    if (o->n_jumps) *o->n_jumps = (int32_t)jumps;
    o->counts[0] = accepted;
    o->counts[1] = rejected;
    o->counts[2] = rhs;
    o->counts[3] = jumps;
    (void)root_iters;
    return status;
}

/* ---------------------------------------------------------------------------
 * Ensemble over trajectories traj0 .. traj0 + ntraj - 1 (threads share nothing
 * but the read-only model; trajectory i is handled by thread i mod nthreads).
 * ------------------------------------------------------------------------- */

static void model_free(model *m)
{
    csr_free(&m->M);
    for (int i = 0; i < m->n_c; i++) csr_free(&m->C[i]);
    for (int i = 0; i < m->n_obs; i++) csr_free(&m->A[i]);
    for (int i = 0; i < m->n_drive; i++) csr_free(&m->D[i]);
    free(m->C);
    free(m->A);
    free(m->D);
    free(m->psi0);
}

/* D = -i H_k of each time-dependent term */
static int drive_init(const orc_problem *p, int n, int *n_drive, csr **D)
{
    *n_drive = 0;
    *D = NULL;
    if (p->n_drive <= 0) return ORC_OK;
    if (!p->drive || !p->drive_coef) return ORC_ERR_ARG;
    *D = calloc((size_t)p->n_drive, sizeof(csr));
    if (!*D) return ORC_ERR_NOMEM;
    for (int k = 0; k < p->n_drive; k++) {
        if (p->drive[k].n != n) return ORC_ERR_ARG;
        int st = csr_from_op(&p->drive[k], &(*D)[k]);
        if (st) return st;
        ++*n_drive;
        csr *d = &(*D)[k];
        for (int e = 0; e < d->row_ptr[d->n]; e++) d->val[e] *= -I;
    }
    return ORC_OK;
}

static int model_init(const orc_problem *p, model *m)
{
    memset(m, 0, sizeof(*m));
    int n = p->dim;
    if (n <= 0 || p->n_t < 1 || !p->t || !p->psi0 || p->H.n != n || p->n_c < 0 || p->n_obs < 0)
        return ORC_ERR_ARG;
    m->n = n;
    m->p = p;
    cplx *Md = malloc(sizeof(cplx) * (size_t)n * n);
    if (!Md) return ORC_ERR_NOMEM;
    effective_matrix_dense(p, Md);
    int st = csr_from_dense(n, Md, &m->M);
    free(Md);
    if (st) return st;
    m->n_c = p->n_c;
    m->n_obs = p->n_obs;
    m->C = calloc((size_t)(p->n_c > 0 ? p->n_c : 1), sizeof(csr));
    m->A = calloc((size_t)(p->n_obs > 0 ? p->n_obs : 1), sizeof(csr));
    m->psi0 = malloc(sizeof(cplx) * n);
    if (!m->C || !m->A || !m->psi0) return ORC_ERR_NOMEM;
    for (int i = 0; i < p->n_c; i++)
        if ((st = csr_from_op(&p->C[i], &m->C[i]))) return st;
    for (int i = 0; i < p->n_obs; i++)
        if ((st = csr_from_op(&p->A[i], &m->A[i]))) return st;
    if ((st = drive_init(p, n, &m->n_drive, &m->D))) return st;
    double nn = 0.0;
    for (int i = 0; i < n; i++) {
        m->psi0[i] = p->psi0[2 * i] + I * p->psi0[2 * i + 1];
        nn += p->psi0[2 * i] * p->psi0[2 * i] + p->psi0[2 * i + 1] * p->psi0[2 * i + 1];
    }
    if (!(nn > 0.0)) return ORC_ERR_ARG;
    nn = sqrt(nn);
    for (int i = 0; i < n; i++) m->psi0[i] /= nn;
    return ORC_OK;
}

typedef struct {
    const model *m;
    uint64_t seed;
    int64_t traj0, ntraj;
    int tid, nthreads;
    orc_result *res;
    int status;
} worker_arg;

/* the vectors of one trajectory's workspace, carved from 16 n complex values */
static void workspace_carve(workspace *w, cplx *buf, int n)
{
    w->psi = buf; w->ynew = buf + n; w->ytmp = buf + 2 * n; w->yd = buf + 3 * n;
    w->cy = buf + 4 * n; w->ay = buf + 5 * n; w->dtmp = buf + 15 * n;
    for (int j = 0; j < 7; j++) w->K[j] = buf + (size_t)(6 + j) * n;
}

static void *worker(void *varg)
{
    worker_arg *a = varg;
    const model *m = a->m;
    int n = m->n;
    const orc_problem *p = m->p;
    cplx *buf = calloc((size_t)n * 16, sizeof(cplx));
    if (!buf) { a->status = ORC_ERR_NOMEM; return NULL; }
    workspace w;
    workspace_carve(&w, buf, n);
    orc_result *res = a->res;
    size_t per = (size_t)p->n_t * p->n_obs;
    for (int64_t i = a->tid; i < a->ntraj; i += a->nthreads) {
        traj_out o;
        memset(&o, 0, sizeof(o));
        o.obs_re = res->obs_re + (size_t)i * per;
        o.obs_im = res->obs_im ? res->obs_im + (size_t)i * per : NULL;
        o.max_jumps = res->max_jumps;
        o.n_jumps = res->n_jumps ? res->n_jumps + i : NULL;
        o.jump_t = res->jump_t ? res->jump_t + (size_t)i * res->max_jumps : NULL;
        o.jump_ch = res->jump_ch ? res->jump_ch + (size_t)i * res->max_jumps : NULL;
        o.jump_norm = res->jump_norm ? res->jump_norm + (size_t)i * res->max_jumps : NULL;
        int st = run_trajectory(m, a->seed, a->traj0 + i, &w, &o);
        if (res->status) res->status[i] = st;
        if (res->counts) memcpy(res->counts + 4 * i, o.counts, sizeof(o.counts));
        if (st != ORC_OK && a->status == ORC_OK) a->status = st;
    }
    free(buf);
    return NULL;
}

/* Runs trajectories traj0 .. traj0+ntraj-1 of the ensemble keyed by seed.
 * Returns 0 or the first per-trajectory error code (all trajectories still run). */
int orc_mcwf(const orc_problem *p, uint64_t seed, int64_t traj0, int64_t ntraj, int nthreads,
             orc_result *res)
{
    if (!p || !res || !res->obs_re || ntraj < 0 || traj0 < 0) return ORC_ERR_ARG;
    if (res->max_jumps < 0) return ORC_ERR_ARG;
    for (int i = 1; i < p->n_t; i++)
        if (!(p->t[i] > p->t[i - 1])) return ORC_ERR_ARG;
    if (!(p->rtol > 0.0) || !(p->atol >= 0.0) || p->max_steps <= 0) return ORC_ERR_ARG;
    model m;
    int st = model_init(p, &m);
    if (st) { model_free(&m); return st; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    worker_arg args[256];
    for (int i = 0; i < nthreads; i++) {
        args[i] = (worker_arg){&m, seed, traj0, ntraj, i, nthreads, res, ORC_OK};
        if (nthreads == 1) worker(&args[i]);
        else pthread_create(&th[i], NULL, worker, &args[i]);
    }
    int first = ORC_OK;
    for (int i = 0; i < nthreads; i++) {
        if (nthreads > 1) pthread_join(th[i], NULL);
        if (first == ORC_OK && args[i].status != ORC_OK) first = args[i].status;
    }
    model_free(&m);
    return first;
}

/* Test hook: the step sequence of one trajectory.  Runs trajectory `traj` alone
 * and stores, for each attempted Dormand-Prince step, its start time, its size and
 * 1 (accepted) or 0 (rejected) in rec[3 i .. 3 i + 2], for at most max_rec
 * attempts; *n_rec = the number stored.  Observables are computed and dropped. */
int orc_step_trace(const orc_problem *p, uint64_t seed, int64_t traj, int64_t max_rec, double *rec,
                   int64_t *n_rec)
{
    if (!p || !rec || !n_rec || max_rec < 0 || traj < 0) return ORC_ERR_ARG;
    if (!(p->rtol > 0.0) || !(p->atol >= 0.0) || p->max_steps <= 0) return ORC_ERR_ARG;
    model m;
    int st = model_init(p, &m);
    if (st) { model_free(&m); return st; }
    const int n = m.n;
    cplx *buf = calloc((size_t)n * 16, sizeof(cplx));
    double *obs = calloc((size_t)p->n_t * (p->n_obs > 0 ? p->n_obs : 1), sizeof(double));
    if (!buf || !obs) {
        free(buf);
        free(obs);
        model_free(&m);
        return ORC_ERR_NOMEM;
    }
    workspace w;
    workspace_carve(&w, buf, n);
    traj_out o;
    memset(&o, 0, sizeof(o));
    o.obs_re = obs;
    o.trace = rec;
    o.max_trace = max_rec;
    st = run_trajectory(&m, seed, traj, &w, &o);
    *n_rec = o.n_trace;
    free(buf);
    free(obs);
    model_free(&m);
    return st;
}

/* ---------------------------------------------------------------------------
 * Lindblad master equation (Sec. 2.2):
 *   drho/dt = -i [H, rho] + sum_n (1/2) (2 C_n rho C_n^dag - rho C_n^dag C_n - C_n^dag C_n rho)
 * integrated as a vector of n^2 complex entries with the same Dormand-Prince pair
 * and controller; the output Tr(A_k rho) is read from the continuous extension.
 * ------------------------------------------------------------------------- */

typedef struct {
    int n;
    csr H;
    int n_c;
    csr *C;
    csr *CdC;   /* C_n^dag C_n */
    cplx *tmp, *tmp2;
    int n_drive;
    csr *Hd;    /* the time-dependent terms' H_k */
    const orc_problem *p;
} lind_model;

/* Y = A X for CSR A and dense row-major X */
static void csr_mm(const csr *a, const cplx *X, cplx *Y, int n)
{
    for (int i = 0; i < n; i++) {
        cplx *yi = Y + (size_t)i * n;
        for (int c = 0; c < n; c++) yi[c] = 0.0;
        for (int k = a->row_ptr[i]; k < a->row_ptr[i + 1]; k++) {
            const cplx *xr = X + (size_t)a->col[k] * n;
            cplx v = a->val[k];
            for (int c = 0; c < n; c++) yi[c] += v * xr[c];
        }
    }
}

/* Y = X A^dag: Y_ij = sum_k X_ik conj(A_jk) */
static void mm_csr_dag(const cplx *X, const csr *a, cplx *Y, int n)
{
    memset(Y, 0, sizeof(cplx) * (size_t)n * n);
    for (int jr = 0; jr < n; jr++)
        for (int k = a->row_ptr[jr]; k < a->row_ptr[jr + 1]; k++) {
            int kc = a->col[k];
            cplx v = conj(a->val[k]);
            for (int i = 0; i < n; i++) Y[(size_t)i * n + jr] += X[(size_t)i * n + kc] * v;
        }
}

static void lindblad_rhs(void *vctx, double t, const cplx *rho, cplx *drho)
{
    lind_model *L = vctx;
    int n = L->n;
    size_t nn = (size_t)n * n;
    /* -i (H rho - rho H);  rho H = rho H^dag for Hermitian H */
    csr_mm(&L->H, rho, L->tmp, n);
    mm_csr_dag(rho, &L->H, L->tmp2, n);
    for (size_t i = 0; i < nn; i++) drho[i] = -I * (L->tmp[i] - L->tmp2[i]);
    /* -i f_k(t) [H_k, rho] */
    for (int k = 0; k < L->n_drive; k++) {
        double f = drive_coef(L->p, k, t);
        csr_mm(&L->Hd[k], rho, L->tmp, n);
        mm_csr_dag(rho, &L->Hd[k], L->tmp2, n);
        for (size_t i = 0; i < nn; i++) drho[i] += -I * f * (L->tmp[i] - L->tmp2[i]);
    }
    for (int c = 0; c < L->n_c; c++) {
        csr_mm(&L->C[c], rho, L->tmp, n);          /* C rho */
        mm_csr_dag(L->tmp, &L->C[c], L->tmp2, n);  /* C rho C^dag */
        for (size_t i = 0; i < nn; i++) drho[i] += L->tmp2[i];
        csr_mm(&L->CdC[c], rho, L->tmp, n);        /* C^dag C rho */
        mm_csr_dag(rho, &L->CdC[c], L->tmp2, n);   /* rho (C^dag C)^dag = rho C^dag C */
        for (size_t i = 0; i < nn; i++) drho[i] -= 0.5 * (L->tmp[i] + L->tmp2[i]);
    }
}

/* Tr(A rho) = sum_{i,k} A_ik rho_ki */
static cplx trace_A_rho(const csr *a, const cplx *rho, int n)
{
    cplx s = 0.0;
    for (int i = 0; i < n; i++)
        for (int k = a->row_ptr[i]; k < a->row_ptr[i + 1]; k++)
            s += a->val[k] * rho[(size_t)a->col[k] * n + i];
    return s;
}

/* Integrates rho from rho0 = |psi0><psi0| (normalised) over the output grid and
 * writes Re Tr(A_k rho(t_j)) to out (n_t * n_obs) and Im to out_im (may be NULL). */
int orc_lindblad(const orc_problem *p, double rtol, double atol, double *out, double *out_im)
{
    if (!p || !out || p->dim <= 0 || p->n_t < 1) return ORC_ERR_ARG;
    int n = p->dim;
    size_t nn = (size_t)n * n;
    lind_model L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.n_c = p->n_c;
    int st = csr_from_op(&p->H, &L.H);
    if (st) return st;
    L.C = calloc((size_t)(p->n_c > 0 ? p->n_c : 1), sizeof(csr));
    L.CdC = calloc((size_t)(p->n_c > 0 ? p->n_c : 1), sizeof(csr));
    csr *A = calloc((size_t)(p->n_obs > 0 ? p->n_obs : 1), sizeof(csr));
    cplx *dense = calloc(nn, sizeof(cplx));
    cplx *buf = calloc(nn * 13, sizeof(cplx));
    if (!L.C || !L.CdC || !A || !dense || !buf) return ORC_ERR_NOMEM;
    for (int c = 0; c < p->n_c; c++) {
        csr_from_op(&p->C[c], &L.C[c]);
        memset(dense, 0, sizeof(cplx) * nn);
        for (int k = 0; k < n; k++)
            for (int a = L.C[c].row_ptr[k]; a < L.C[c].row_ptr[k + 1]; a++)
                for (int b = L.C[c].row_ptr[k]; b < L.C[c].row_ptr[k + 1]; b++)
                    dense[(size_t)L.C[c].col[a] * n + L.C[c].col[b]] +=
                        conj(L.C[c].val[a]) * L.C[c].val[b];
        csr_from_dense(n, dense, &L.CdC[c]);
    }
    for (int k = 0; k < p->n_obs; k++) csr_from_op(&p->A[k], &A[k]);
    L.p = p;
    if (p->n_drive > 0) {
        if (!p->drive || !p->drive_coef) return ORC_ERR_ARG;
        L.Hd = calloc((size_t)p->n_drive, sizeof(csr));
        if (!L.Hd) return ORC_ERR_NOMEM;
        for (int k = 0; k < p->n_drive; k++) {
            if (p->drive[k].n != n) return ORC_ERR_ARG;
            if ((st = csr_from_op(&p->drive[k], &L.Hd[k]))) return st;
            L.n_drive++;
        }
    }
    L.tmp = buf;
    L.tmp2 = buf + nn;
    cplx *rho = buf + 2 * nn, *rnew = buf + 3 * nn, *rtmp = buf + 4 * nn, *rd = buf + 5 * nn;
    cplx *K[7];
    for (int j = 0; j < 7; j++) K[j] = buf + (size_t)(6 + j) * nn;

    double pn = 0.0;
    for (int i = 0; i < n; i++)
        pn += p->psi0[2 * i] * p->psi0[2 * i] + p->psi0[2 * i + 1] * p->psi0[2 * i + 1];
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++) {
            cplx a = (p->psi0[2 * i] + I * p->psi0[2 * i + 1]);
            cplx b = (p->psi0[2 * k] + I * p->psi0[2 * k + 1]);
            rho[(size_t)i * n + k] = a * conj(b) / pn;
        }
    const int no = p->n_obs;
    for (int k = 0; k < no; k++) {
        cplx e = trace_A_rho(&A[k], rho, n);
        out[k] = creal(e);
        if (out_im) out_im[k] = cimag(e);
    }
    double t = p->t[0], t_end = p->t[p->n_t - 1];
    int j = 1;
    int64_t rhs = 0;
    lindblad_rhs(&L, t, rho, K[0]);
    double h = dp_initial_step((int)nn, lindblad_rhs, &L, t, rho, K[0], t_end - t, rtol, atol, rtmp,
                               rnew, &rhs);
    int rejected_before = 0;
    int status = ORC_OK;
    int64_t attempts = 0;
    while (j < p->n_t) {
        if (attempts++ > 50000000) { status = ORC_ERR_MAXSTEPS; break; }
        int last = 0;
        if (t + 1.01 * h >= t_end) {
            h = t_end - t;
            last = 1;
        }
        double err = dp_step((int)nn, lindblad_rhs, &L, t, rho, K, h, rnew, rtmp, rtol, atol);
        if (!(err <= 1.0)) {
            if (!isfinite(err)) { status = ORC_ERR_NONFINITE; break; }
            double fac = DP_SAFETY * pow(err, -0.2);
            h *= fac < DP_FACMIN ? DP_FACMIN : fac;
            rejected_before = 1;
            continue;
        }
        double t_new = last ? t_end : t + h;
        for (; j < p->n_t && p->t[j] <= t_new; j++) {
            double thj = (p->t[j] - t) / h;
            if (thj > 1.0) thj = 1.0;
            dp_dense((int)nn, rho, K, h, thj, rd);
            for (int k = 0; k < no; k++) {
                cplx e = trace_A_rho(&A[k], rd, n);
                out[(size_t)j * no + k] = creal(e);
                if (out_im) out_im[(size_t)j * no + k] = cimag(e);
            }
        }
        double fac = (err == 0.0) ? DP_FACMAX : DP_SAFETY * pow(err, -0.2);
        if (fac > DP_FACMAX) fac = DP_FACMAX;
        if (fac < DP_FACMIN) fac = DP_FACMIN;
        if (rejected_before && fac > 1.0) fac = 1.0;
        rejected_before = 0;
        t = t_new;
        memcpy(rho, rnew, sizeof(cplx) * nn);
        memcpy(K[0], K[6], sizeof(cplx) * nn);
        h *= fac;
    }
    csr_free(&L.H);
    for (int c = 0; c < p->n_c; c++) {
        csr_free(&L.C[c]);
        csr_free(&L.CdC[c]);
    }
    for (int k = 0; k < p->n_obs; k++) csr_free(&A[k]);
    for (int k = 0; k < L.n_drive; k++) csr_free(&L.Hd[k]);
    free(L.Hd);
    free(L.C);
    free(L.CdC);
    free(A);
    free(dense);
    free(buf);
    return status;
}
