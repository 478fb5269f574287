// qtm_api.cpp -- host side of the C ABI declared in include/qtm.h.
//
// qtm_create validates the problem statement (the inputs of the paper's
// mpi_main, Sec. 3), forms M = -i H_eff = -i H - (1/2) sum_n C_n^dag C_n
// (Sec. 2.2, Eq. eqn:effective:hamiltonian; hbar = 1, the stored form of the
// Sec. 4.1 listing), normalises psi0, packs every operator into one CSR blob and
// uploads it.  qtm_run launches the trajectory kernel and the ensemble
// reduction on the context's stream; the synchronising calls copy results back.
// No numerical step of a trajectory runs on the host.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qtm.h"
#include "dense_tc.h"
#include "moments.h"
#include "proposal.cuh"
#include "qtm_launch.h"

using cd = std::complex<double>;
using qtm::KernelArgs;
using qtm::LaunchInfo;
using qtm::OpOffsets;

namespace {

struct Allocator {
    qtm_alloc_fn alloc = nullptr;
    qtm_free_fn free = nullptr;
    void *user = nullptr;
};

Allocator g_allocator;
thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Csr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<cd> val;
};

}  // namespace

struct qtm_ctx {
    cudaStream_t stream = nullptr;
    Allocator alloc;
    int device = 0;
    int n = 0, n_c = 0, n_obs = 0, n_t = 0;
    int precision = 0, flags = 0, max_jumps = 0;
    double rtol = 0, atol = 0;
    long long max_steps = 0;
    std::vector<int> ints;
    std::vector<double> reals;
    std::vector<OpOffsets> ops;
    std::vector<double> t;
    std::vector<cd> psi0;
    Csr M;                       // host copies of the operators, for repacking
    std::vector<Csr> Cops, Aops;
    std::vector<Csr> Dops;       // -i H_k of the time-dependent terms
    std::vector<double> drive;   // 3 per term: a_k, omega_k, phi_k
    DevBuf d_ints, d_vals, d_t, d_psi0, d_queue, d_counters, d_first_error;
    DevBuf d_out, d_partial, d_moments, d_scale, d_njumps, d_jump_t, d_jump_ch;
    std::vector<int> scale_exp;  // per observable: values are bounded by 2^(E - 1) (moments.h)
    int krylov_shift = 0;        // 2^krylov_shift > ||M|| (Krylov form of the Dormand-Prince step)
    // learned jump-time proposal
    DevBuf d_rec, d_mlp, d_X, d_T, d_gpart, d_lpart, d_grad, d_loss, d_m, d_v;
    int rec_stride = 0, rec_max = 0;
    bool mlp_on = false, mlp_set = false;
    float prop_margin = 0.05f;
    std::vector<float> pair_f, pair_dt;  // collected (raw features, time left to the jump)
    qtm::Layout layout{0, 0};
    // tensor-core engine (QTM_PREC_BF16X6): bf16 operator splits, their tensor
    // map, the column state and per-column records
    int np = 0, sms = 0;
    unsigned long long wait_limit_ns = 0;  // 0: the engine's default bound
    DevBuf d_op, d_state, d_col, d_rhs, d_dense;
    std::vector<int> dense_off;  // per operator: float2 offset of its dense copy, -1 = SELL
    CUtensorMap op_map{};
    // exponential propagation (qtm_set_method): the ladder exp(M delta 2^l),
    // l < expo_levels, as [level][n][n] row-major complex (host copy)
    int method = QTM_METHOD_DOPRI5;
    std::vector<cd> ladder;
    int expo_levels = 0, expo_uniform = 0;
    double expo_delta = 0.0;
    DevBuf d_expo;
    // the exponential method on the tensor cores (QTM_PREC_BF16X6, uniform grid):
    // bf16 splits of the real form of P_L - I and their tensor map; the lock-step
    // columns' states, products, records and deferred list
    DevBuf d_op_expo, d_lpsi, d_ly, d_lcol, d_llist;
    CUtensorMap expo_map{};
    long long last_ntraj = -1;
    // kernel start, kernel end, reduction end; one tensor-core product's start and end
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool product_timed = false;
    bool timed = false;
    LaunchInfo info{};
    std::string err;
};

namespace {

qtm_status fail(qtm_ctx *ctx, qtm_status st, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return st;
}

qtm_status cuda_fail(qtm_ctx *ctx, cudaError_t e, const char *what)
{
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(ctx, QTM_ERR_CUDA, msg);
}

cudaError_t dev_alloc(qtm_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (ctx->alloc.alloc) {
        p = ctx->alloc.alloc(bytes, (void *)ctx->stream, ctx->alloc.user);
        if (!p) return cudaErrorMemoryAllocation;
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    b.p = p;
    b.bytes = bytes;
    return cudaSuccess;
}

void dev_free(qtm_ctx *ctx, DevBuf &b)
{
    if (!b.p) return;
    if (ctx->alloc.free)
        ctx->alloc.free(b.p, b.bytes, (void *)ctx->stream, ctx->alloc.user);
    else
        cudaFreeAsync(b.p, ctx->stream);
    b.p = nullptr;
    b.bytes = 0;
}

// grows b to at least `bytes` (contents are not preserved)
cudaError_t dev_reserve(qtm_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return cudaSuccess;
    dev_free(ctx, b);
    return dev_alloc(ctx, b, bytes);
}

bool is_finite(double x) { return std::isfinite(x); }

// Copies a user operator into CSR form, checking its structure.
qtm_status read_op(const qtm_op &op, int n, const char *name, Csr &out)
{
    char buf[256];
    if (op.n != n) {
        std::snprintf(buf, sizeof buf, "%s: n = %d differs from dim = %d", name, op.n, n);
        return fail(nullptr, QTM_ERR_ARG, buf);
    }
    out.n = n;
    out.rp.assign(n + 1, 0);
    out.ci.clear();
    out.val.clear();
    if (op.format == QTM_FORMAT_DENSE) {
        if (!op.values) return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": dense values are NULL");
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                const double re = op.values[2 * ((size_t)i * n + j)];
                const double im = op.values[2 * ((size_t)i * n + j) + 1];
                if (!is_finite(re) || !is_finite(im))
                    return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": non-finite entry");
                if (re != 0.0 || im != 0.0) {
                    out.ci.push_back(j);
                    out.val.emplace_back(re, im);
                }
            }
            out.rp[i + 1] = (int)out.ci.size();
        }
        return QTM_OK;
    }
    if (op.format != QTM_FORMAT_CSR)
        return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": unknown format");
    if (!op.row_ptr) return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": row_ptr is NULL");
    if (op.row_ptr[0] != 0) return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": row_ptr[0] != 0");
    for (int i = 0; i < n; ++i)
        if (op.row_ptr[i + 1] < op.row_ptr[i])
            return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": row_ptr decreases");
    const int64_t nnz = op.row_ptr[n];
    if (nnz != op.nnz) {
        std::snprintf(buf, sizeof buf, "%s: nnz = %lld but row_ptr[n] = %lld", name, (long long)op.nnz,
                      (long long)nnz);
        return fail(nullptr, QTM_ERR_ARG, buf);
    }
    if (nnz > 0 && (!op.col_ind || !op.values))
        return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": col_ind/values are NULL");
    for (int i = 0; i < n; ++i) {
        for (int k = op.row_ptr[i]; k < op.row_ptr[i + 1]; ++k) {
            const int c = op.col_ind[k];
            if (c < 0 || c >= n) {
                std::snprintf(buf, sizeof buf, "%s: column index %d out of range in row %d", name, c, i);
                return fail(nullptr, QTM_ERR_ARG, buf);
            }
            const double re = op.values[2 * (size_t)k], im = op.values[2 * (size_t)k + 1];
            if (!is_finite(re) || !is_finite(im))
                return fail(nullptr, QTM_ERR_ARG, std::string(name) + ": non-finite entry");
            out.ci.push_back(c);
            out.val.emplace_back(re, im);
        }
        out.rp[i + 1] = (int)out.ci.size();
    }
    return QTM_OK;
}

// Hermiticity within 1e-12 of the largest entry (duplicate entries are summed).
bool is_hermitian(const Csr &a)
{
    std::vector<std::map<int, cd>> rows(a.n);
    double amax = 0.0;
    for (int i = 0; i < a.n; ++i)
        for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
            rows[i][a.ci[k]] += a.val[k];
            amax = std::max(amax, std::abs(a.val[k]));
        }
    const double tol = 1e-12 * std::max(1.0, amax);
    for (int i = 0; i < a.n; ++i)
        for (const auto &kv : rows[i]) {
            auto it = rows[kv.first].find(i);
            const cd other = it == rows[kv.first].end() ? cd(0.0) : it->second;
            if (std::abs(kv.second - std::conj(other)) > tol) return false;
        }
    return true;
}

// M = -i H - (1/2) sum_n C_n^dag C_n; (C^dag C)_{ij} = sum_k conj(C_ki) C_kj.
// Entries are accumulated in the order H, then channel by channel, row by row.
Csr effective_matrix(const Csr &H, const std::vector<Csr> &C)
{
    const int n = H.n;
    std::vector<std::map<int, cd>> rows(n);
    for (int i = 0; i < n; ++i)
        for (int k = H.rp[i]; k < H.rp[i + 1]; ++k) rows[i][H.ci[k]] += cd(0.0, -1.0) * H.val[k];
    for (const Csr &c : C)
        for (int k = 0; k < n; ++k)
            for (int a = c.rp[k]; a < c.rp[k + 1]; ++a)
                for (int b = c.rp[k]; b < c.rp[k + 1]; ++b)
                    rows[c.ci[a]][c.ci[b]] += -0.5 * std::conj(c.val[a]) * c.val[b];
    Csr M;
    M.n = n;
    M.rp.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        for (const auto &kv : rows[i])
            if (kv.second != cd(0.0)) {
                M.ci.push_back(kv.first);
                M.val.push_back(kv.second);
            }
        M.rp[i + 1] = (int)M.ci.size();
    }
    return M;
}

// Appends one real part of an operator (selected entries of a) in SELL-G form.
qtm::SellPart pack_part(qtm_ctx *ctx, const Csr &a, bool imag, qtm::Layout lay)
{
    const int G = lay.G, R = lay.R, n = a.n;
    std::vector<std::vector<std::pair<int, double>>> rows(n);
    for (int i = 0; i < n; ++i)
        for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
            const double v = imag ? a.val[k].imag() : a.val[k].real();
            if (v != 0.0) rows[i].emplace_back(a.ci[k], v);
        }
    qtm::SellPart o;
    o.table = (int)ctx->ints.size();
    ctx->ints.resize(ctx->ints.size() + 2 * R, 0);
    o.cols = (int)ctx->ints.size();
    o.vals = (int)ctx->reals.size();
    int off = 0;
    for (int r = 0; r < R; ++r) {
        int width = 0;
        for (int gl = 0; gl < G; ++gl) {
            const int row = gl + G * r;
            if (row < n) width = std::max(width, (int)rows[row].size());
        }
        ctx->ints[o.table + 2 * r] = off;
        ctx->ints[o.table + 2 * r + 1] = width;
        for (int t = 0; t < width; ++t)
            for (int gl = 0; gl < G; ++gl) {
                const int row = gl + G * r;
                const bool has = row < n && t < (int)rows[row].size();
                ctx->ints.push_back(has ? rows[row][t].first : 0);
                ctx->reals.push_back(has ? rows[row][t].second : 0.0);
            }
        off += width * G;
    }
    return o;
}

// Appends operator a (both parts) for the layout (G, R).
void pack(qtm_ctx *ctx, const Csr &a, qtm::Layout lay)
{
    OpOffsets o;
    o.re = pack_part(ctx, a, false, lay);
    o.im = pack_part(ctx, a, true, lay);
    ctx->ops.push_back(o);
}

// Packs every operator (M, the C_n, the A_k) for layout lay (host side only).
void repack(qtm_ctx *ctx, qtm::Layout lay)
{
    ctx->layout = lay;
    ctx->ints.clear();
    ctx->reals.clear();
    ctx->ops.clear();
    pack(ctx, ctx->M, lay);
    for (const Csr &c : ctx->Cops) pack(ctx, c, lay);
    for (const Csr &a : ctx->Aops) pack(ctx, a, lay);
    for (const Csr &d : ctx->Dops) pack(ctx, d, lay);
}

// Real values in the layout of the kernel's arithmetic: doubles for complex128,
// (hi, lo) float pairs with hi = fl32(x), lo = fl32(x - hi) for double-float,
// floats for complex64.
std::vector<unsigned char> encode_reals(const std::vector<double> &v, int precision)
{
    std::vector<unsigned char> out;
    if (precision == QTM_PREC_C128) {
        out.resize(v.size() * sizeof(double));
        std::memcpy(out.data(), v.data(), out.size());
    } else if (precision == QTM_PREC_DF64) {
        std::vector<float> f(v.size() * 2);
        for (size_t i = 0; i < v.size(); ++i) {
            const float h = (float)v[i];
            f[2 * i] = h;
            f[2 * i + 1] = (float)(v[i] - (double)h);
        }
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    } else {
        std::vector<float> f(v.begin(), v.end());
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    }
    if (out.empty()) out.resize(16);
    return out;
}

// Complex values in the layout of the kernel's arithmetic: (re, im) doubles for
// complex128; (re_hi, re_lo, im_hi, im_lo) floats for double-float, with
// hi = fl32(x) and lo = fl32(x - hi); (re, im) floats for complex64.
std::vector<unsigned char> encode_values(const std::vector<cd> &v, int precision)
{
    std::vector<unsigned char> out;
    if (precision == QTM_PREC_C128) {
        out.resize(v.size() * sizeof(cd));
        std::memcpy(out.data(), v.data(), out.size());
    } else if (precision == QTM_PREC_DF64) {
        std::vector<float> f(v.size() * 4);
        for (size_t i = 0; i < v.size(); ++i) {
            const double re = v[i].real(), im = v[i].imag();
            const float rh = (float)re, ih = (float)im;
            f[4 * i + 0] = rh;
            f[4 * i + 1] = (float)(re - (double)rh);
            f[4 * i + 2] = ih;
            f[4 * i + 3] = (float)(im - (double)ih);
        }
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    } else {
        std::vector<float> f(v.size() * 2);
        for (size_t i = 0; i < v.size(); ++i) {
            f[2 * i] = (float)v[i].real();
            f[2 * i + 1] = (float)v[i].imag();
        }
        out.resize(f.size() * sizeof(float));
        std::memcpy(out.data(), f.data(), out.size());
    }
    if (out.empty()) out.resize(16);
    return out;
}

// ---- exponential propagation: the ladder exp(M delta 2^l) -------------------
//
// Scaling and squaring (Moler & Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix", 2003, the Taylor variant): with nu = max(||M||_1,
// ||M||_inf) >= ||M||_2, delta = span / 2^L is the largest such step with
// nu delta <= 1/16; exp(M delta) is the Taylor polynomial of degree 12 (its
// truncation error is below (1/16)^13 / 13! ~ 4e-26 relative) and each further
// level is the square of the one below.  FP64, on the host (setup).

constexpr double kExpoTheta = 1.0 / 16.0;
constexpr int kExpoDegree = 12;

double op_norm_bound(const Csr &M)
{
    std::vector<double> col(M.n, 0.0);
    double rmax = 0.0;
    for (int i = 0; i < M.n; ++i) {
        double r = 0.0;
        for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) {
            r += std::abs(M.val[k]);
            col[M.ci[k]] += std::abs(M.val[k]);
        }
        rmax = std::max(rmax, r);
    }
    double cmax = 0.0;
    for (double c : col) cmax = std::max(cmax, c);
    return std::max(rmax, cmax);
}

// Scale exponent of an observable's recorded values (moments.h): for Hermitian A,
// |<psi|A|psi>| / <psi|psi> <= ||A||_2 <= max_i sum_j |A_ij| <= max_i sum_j
// (|Re A_ij| + |Im A_ij|); the last form is summed with plain additions in CSR
// order, so every host computes the same exponent.
int observable_scale(const Csr &A)
{
    double bound = 0.0;
    for (int i = 0; i < A.n; ++i) {
        double r = 0.0;
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) r += std::fabs(A.val[k].real()) + std::fabs(A.val[k].imag());
        bound = std::max(bound, r);
    }
    return qtm::scale_exponent(bound);
}

// X = sum_{m <= degree} (h M)^m / m! by Horner's rule, X <- I + (h/m) M X (dense row-major)
void taylor_exp(const Csr &M, double h, int degree, cd *X)
{
    const int n = M.n;
    std::vector<cd> Y((size_t)n * n);
    for (size_t i = 0; i < (size_t)n * n; ++i) X[i] = 0.0;
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    for (int m = degree; m >= 1; --m) {
        std::fill(Y.begin(), Y.end(), cd(0.0));
        for (int i = 0; i < n; ++i)
            for (int k = M.rp[i]; k < M.rp[i + 1]; ++k) {
                const cd v = M.val[k];
                const cd *xr = X + (size_t)M.ci[k] * n;
                cd *yr = Y.data() + (size_t)i * n;
                for (int j = 0; j < n; ++j) yr[j] += v * xr[j];
            }
        const double c = h / m;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) X[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) + c * Y[(size_t)i * n + j];
    }
}

// Z = X X (dense row-major)
void square_into(const cd *X, cd *Z, int n)
{
    for (size_t i = 0; i < (size_t)n * n; ++i) Z[i] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const cd x = X[(size_t)i * n + k];
            if (x == cd(0.0)) continue;
            const cd *xr = X + (size_t)k * n;
            cd *zr = Z + (size_t)i * n;
            for (int j = 0; j < n; ++j) zr[j] += x * xr[j];
        }
}

// ladder[l] = exp(M delta 2^l), l = 0..L, with delta 2^L = span; returns L + 1
// (0 when span is not positive and finite or needs more than 60 halvings)
int expm_ladder(const Csr &M, double span, std::vector<cd> &ladder, double &delta)
{
    if (!(span > 0.0) || !std::isfinite(span)) return 0;
    const int n = M.n;
    const double nu = op_norm_bound(M);
    int L = 0;
    if (nu * span > kExpoTheta) L = (int)std::ceil(std::log2(nu * span / kExpoTheta));
    while (L > 0 && std::ldexp(span, -(L - 1)) * nu <= kExpoTheta) --L;  // log2 rounding
    while (std::ldexp(span, -L) * nu > kExpoTheta) ++L;
    if (L > 60) return 0;
    delta = std::ldexp(span, -L);
    const size_t nn = (size_t)n * n;
    ladder.assign((size_t)(L + 1) * nn, cd(0.0));
    taylor_exp(M, delta, kExpoDegree, ladder.data());
    for (int l = 1; l <= L; ++l) square_into(ladder.data() + (l - 1) * nn, ladder.data() + l * nn, n);
    return L + 1;
}

void destroy_ctx(qtm_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    DevBuf *bufs[] = {&ctx->d_ints, &ctx->d_vals, &ctx->d_t, &ctx->d_psi0, &ctx->d_queue,
                      &ctx->d_counters, &ctx->d_first_error, &ctx->d_out, &ctx->d_partial,
                      &ctx->d_moments, &ctx->d_scale, &ctx->d_njumps, &ctx->d_jump_t, &ctx->d_jump_ch,
                      &ctx->d_rec, &ctx->d_mlp, &ctx->d_X, &ctx->d_T, &ctx->d_gpart, &ctx->d_lpart,
                      &ctx->d_grad, &ctx->d_loss, &ctx->d_m, &ctx->d_v, &ctx->d_op, &ctx->d_state,
                      &ctx->d_col, &ctx->d_rhs, &ctx->d_dense, &ctx->d_expo, &ctx->d_op_expo, &ctx->d_lpsi,
                      &ctx->d_ly, &ctx->d_lcol, &ctx->d_llist};
    for (DevBuf *b : bufs) dev_free(ctx, *b);
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

}  // namespace

namespace qtm {
void set_last_error(const char *msg) { g_create_error = msg; }
}  // namespace qtm

extern "C" {

namespace {

// bf16 with round-to-nearest-even (finite inputs)
uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// The tensor-core engine's operator: the real form Mr = [[Re M, -Im M], [Im M, Re M]]
// of M (2 np x 2 np, zero-padded), row i = output, column k = input, split into
// three bf16 terms x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1):
// out = [x0 rows][x1 rows][x2 rows].
// The engine's operator: the real form of 2^-shift M (the Krylov form's scaled
// operator; scaling by a power of two is exact), split into three bf16 terms.
std::vector<uint16_t> tc_split(const std::vector<double> &mr);

std::vector<uint16_t> tc_operator(const Csr &M, int np, int shift)
{
    const int kd = 2 * np;
    const double sc = std::ldexp(1.0, -shift);
    std::vector<double> mr((size_t)kd * kd, 0.0);
    for (int i = 0; i < M.n; ++i)
        for (int e = M.rp[i]; e < M.rp[i + 1]; ++e) {
            const int k = M.ci[e];
            const double re = sc * M.val[e].real(), im = sc * M.val[e].imag();
            mr[(size_t)i * kd + k] = re;
            mr[(size_t)i * kd + np + k] = -im;
            mr[(size_t)(np + i) * kd + k] = im;
            mr[(size_t)(np + i) * kd + np + k] = re;
        }
    return tc_split(mr);
}

// The same real form and split for a dense n x n complex matrix (row-major): the
// exponential method's top-level propagator minus the identity.
std::vector<uint16_t> tc_operator_dense(const cd *P, int n, int np)
{
    const int kd = 2 * np;
    std::vector<double> mr((size_t)kd * kd, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double re = P[(size_t)i * n + k].real(), im = P[(size_t)i * n + k].imag();
            mr[(size_t)i * kd + k] = re;
            mr[(size_t)i * kd + np + k] = -im;
            mr[(size_t)(np + i) * kd + k] = im;
            mr[(size_t)(np + i) * kd + np + k] = re;
        }
    return tc_split(mr);
}

// [x0 rows][x1 rows][x2 rows] of the three-term bf16 split of mr
std::vector<uint16_t> tc_split(const std::vector<double> &mr)
{
    std::vector<uint16_t> out(3 * mr.size());
    for (size_t i = 0; i < mr.size(); ++i) {
        double r = mr[i];
        for (int q = 0; q < 3; ++q) {
            const uint16_t b = bf16_rne((float)r);
            out[q * mr.size() + i] = b;
            r -= (double)bf16_value(b);
        }
    }
    return out;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map over the operator splits [3 kd rows][kd] bf16: boxes of 64 (one
// 128-byte row) x 128 rows with the 128-byte swizzle the MMA descriptors expect.
qtm_status tc_make_map(qtm_ctx *ctx, void *base, CUtensorMap *map)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qtm_create: driver entry point");
    if (q != cudaDriverEntryPointSuccess || !fn)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_create: the driver has no cuTensorMapEncodeTiled");
    const int kd = 2 * ctx->np;
    const cuuint64_t dims[2] = {(cuuint64_t)kd, (cuuint64_t)(3 * kd)};
    const cuuint64_t strides[1] = {(cuuint64_t)kd * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = ((EncodeTiledFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, QTM_ERR_CUDA, "qtm_create: cuTensorMapEncodeTiled failed");
    return QTM_OK;
}

// Uploads the operator splits and builds the tensor map (QTM_PREC_BF16X6); also
// the copies the engine's control warps use for their products (channel weights,
// jumps, K_0 after a jump, observables): the np diagonal values of a diagonal
// operator, a dense column-major FP32 copy [n][np] of an operator with at least
// n^2/4 non-zeros; the others stay SELL.
qtm_status tc_setup(qtm_ctx *ctx)
{
    ctx->np = qtm::tc_padded_dim(ctx->n);
    std::vector<uint16_t> op = tc_operator(ctx->M, ctx->np, ctx->krylov_shift);
    std::vector<const Csr *> all{&ctx->M};
    for (const Csr &c : ctx->Cops) all.push_back(&c);
    for (const Csr &a : ctx->Aops) all.push_back(&a);
    std::vector<float> dense;
    ctx->dense_off.assign(all.size(), -1);
    const size_t n = (size_t)ctx->n, np = (size_t)ctx->np;
    for (size_t i = 0; i < all.size(); ++i) {
        const Csr &m = *all[i];
        bool diagonal = true;
        for (int r = 0; r < m.n && diagonal; ++r)
            for (int e = m.rp[r]; e < m.rp[r + 1]; ++e)
                if (m.ci[e] != r) diagonal = false;
        if (diagonal) {  // np complex values, encoded as -2 - offset
            const size_t off = dense.size() / 2;
            dense.resize(dense.size() + 2 * np, 0.f);
            for (int r = 0; r < m.n; ++r)
                for (int e = m.rp[r]; e < m.rp[r + 1]; ++e) {
                    dense[2 * (off + r)] = (float)m.val[e].real();
                    dense[2 * (off + r) + 1] = (float)m.val[e].imag();
                }
            ctx->dense_off[i] = -2 - (int)off;
            continue;
        }
        if (4 * m.ci.size() < n * n) continue;
        ctx->dense_off[i] = (int)(dense.size() / 2);
        dense.resize(dense.size() + 2 * n * np, 0.f);
        float *d = dense.data() + 2 * (size_t)ctx->dense_off[i];
        for (int r = 0; r < m.n; ++r)
            for (int e = m.rp[r]; e < m.rp[r + 1]; ++e) {
                d[2 * ((size_t)m.ci[e] * np + r)] = (float)m.val[e].real();
                d[2 * ((size_t)m.ci[e] * np + r) + 1] = (float)m.val[e].imag();
            }
    }
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device)) ||
        (e = dev_alloc(ctx, ctx->d_op, op.size() * sizeof(uint16_t))) ||
        (e = dev_alloc(ctx, ctx->d_dense, dense.size() * sizeof(float))) ||
        (e = cudaMemcpyAsync(ctx->d_op.p, op.data(), op.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                             ctx->stream)) ||
        (!dense.empty() && (e = cudaMemcpyAsync(ctx->d_dense.p, dense.data(), dense.size() * sizeof(float),
                                                cudaMemcpyHostToDevice, ctx->stream))) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_create: tensor-core operator upload");
    return tc_make_map(ctx, ctx->d_op.p, &ctx->op_map);
}

}  // namespace

const char *qtm_version(void) { return "0.1.0 sm_103a"; }

const char *qtm_status_string(qtm_status s)
{
    switch (s) {
    case QTM_OK: return "QTM_OK";
    case QTM_ERR_ARG: return "QTM_ERR_ARG";
    case QTM_ERR_CUDA: return "QTM_ERR_CUDA";
    case QTM_ERR_NOMEM: return "QTM_ERR_NOMEM";
    case QTM_ERR_MAXSTEPS: return "QTM_ERR_MAXSTEPS";
    case QTM_ERR_STEPSIZE: return "QTM_ERR_STEPSIZE";
    case QTM_ERR_NONFINITE: return "QTM_ERR_NONFINITE";
    case QTM_ERR_NO_CHANNEL: return "QTM_ERR_NO_CHANNEL";
    case QTM_ERR_TIMEOUT: return "QTM_ERR_TIMEOUT";
    case QTM_ERR_STATE: return "QTM_ERR_STATE";
    case QTM_ERR_UNSUPPORTED: return "QTM_ERR_UNSUPPORTED";
    }
    return "QTM_ERR_UNKNOWN";
}

const char *qtm_last_error(const qtm_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

qtm_status qtm_set_allocator(qtm_alloc_fn alloc, qtm_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(nullptr, QTM_ERR_ARG, "qtm_set_allocator: alloc and free must both be set or both NULL");
    g_allocator.alloc = alloc;
    g_allocator.free = free_fn;
    g_allocator.user = user;
    return QTM_OK;
}

qtm_status qtm_create(const qtm_problem *p, void *cuda_stream, qtm_ctx **out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, QTM_ERR_ARG, "qtm_create: out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, QTM_ERR_ARG, "qtm_create: problem is NULL");
    const int n = p->dim;
    char buf[256];
    if (n < 1) return fail(nullptr, QTM_ERR_ARG, "qtm_create: dim must be >= 1");
    if (p->n_c < 0 || p->n_obs < 0) return fail(nullptr, QTM_ERR_ARG, "qtm_create: negative operator count");
    if (p->n_c > 0 && !p->C) return fail(nullptr, QTM_ERR_ARG, "qtm_create: C is NULL");
    if (p->n_obs > 0 && !p->A) return fail(nullptr, QTM_ERR_ARG, "qtm_create: A is NULL");
    if (p->n_t < 1 || !p->t) return fail(nullptr, QTM_ERR_ARG, "qtm_create: need n_t >= 1 output times");
    for (int i = 0; i < p->n_t; ++i)
        if (!is_finite(p->t[i])) return fail(nullptr, QTM_ERR_ARG, "qtm_create: non-finite output time");
    for (int i = 1; i < p->n_t; ++i)
        if (!(p->t[i] > p->t[i - 1]))
            return fail(nullptr, QTM_ERR_ARG, "qtm_create: output times must be strictly increasing");
    if (!(p->rtol > 0.0) || !(p->atol >= 0.0) || !is_finite(p->rtol) || !is_finite(p->atol))
        return fail(nullptr, QTM_ERR_ARG, "qtm_create: need rtol > 0 and atol >= 0");
    if (p->max_steps <= 0) return fail(nullptr, QTM_ERR_ARG, "qtm_create: max_steps must be > 0");
    if (p->precision != QTM_PREC_C128 && p->precision != QTM_PREC_C64 && p->precision != QTM_PREC_DF64 &&
        p->precision != QTM_PREC_BF16X6)
        return fail(nullptr, QTM_ERR_ARG, "qtm_create: unknown precision");
    if ((p->flags & ~QTM_FLAG_RECORD_JUMPS) != 0) return fail(nullptr, QTM_ERR_ARG, "qtm_create: unknown flags");
    if ((p->flags & QTM_FLAG_RECORD_JUMPS) && p->max_jumps_recorded < 1)
        return fail(nullptr, QTM_ERR_ARG, "qtm_create: RECORD_JUMPS needs max_jumps_recorded >= 1");
    if (!p->psi0) return fail(nullptr, QTM_ERR_ARG, "qtm_create: psi0 is NULL");

    Csr H;
    qtm_status st = read_op(p->H, n, "H", H);
    if (st) return st;
    if (!is_hermitian(H)) return fail(nullptr, QTM_ERR_ARG, "qtm_create: H is not Hermitian (tolerance 1e-12)");
    std::vector<Csr> C(p->n_c), A(p->n_obs);
    for (int i = 0; i < p->n_c; ++i) {
        std::snprintf(buf, sizeof buf, "C[%d]", i);
        if ((st = read_op(p->C[i], n, buf, C[i]))) return st;
    }
    for (int i = 0; i < p->n_obs; ++i) {
        std::snprintf(buf, sizeof buf, "A[%d]", i);
        if ((st = read_op(p->A[i], n, buf, A[i]))) return st;
        if (!is_hermitian(A[i])) {
            std::snprintf(buf, sizeof buf, "qtm_create: A[%d] is not Hermitian (tolerance 1e-12)", i);
            return fail(nullptr, QTM_ERR_ARG, buf);
        }
    }
    double nn = 0.0;
    for (int i = 0; i < n; ++i) {
        const double re = p->psi0[2 * i], im = p->psi0[2 * i + 1];
        if (!is_finite(re) || !is_finite(im)) return fail(nullptr, QTM_ERR_ARG, "qtm_create: non-finite psi0");
        nn += re * re + im * im;
    }
    if (!(nn > 0.0)) return fail(nullptr, QTM_ERR_ARG, "qtm_create: psi0 is zero");
    if (1 + p->n_c + p->n_obs > qtm::kMaxOps) {
        std::snprintf(buf, sizeof buf, "qtm_create: at most %d operators in total", qtm::kMaxOps);
        return fail(nullptr, QTM_ERR_UNSUPPORTED, buf);
    }
    if (p->n_c > qtm::kMaxChannels) {
        std::snprintf(buf, sizeof buf, "qtm_create: at most %d collapse operators", qtm::kMaxChannels);
        return fail(nullptr, QTM_ERR_UNSUPPORTED, buf);
    }
    if (p->precision == QTM_PREC_BF16X6 && n > qtm::kTcMaxDim) {
        std::snprintf(buf, sizeof buf, "qtm_create: the tensor-core path takes dim <= %d", qtm::kTcMaxDim);
        return fail(nullptr, QTM_ERR_UNSUPPORTED, buf);
    }
    if (qtm::layout_for_dim(n).G == 0) {
        std::snprintf(buf, sizeof buf, "qtm_create: dim %d exceeds the largest supported dimension %d", n,
                      qtm::kMaxDimSparse);
        return fail(nullptr, QTM_ERR_UNSUPPORTED, buf);
    }

    qtm_ctx *ctx = new (std::nothrow) qtm_ctx;
    if (!ctx) return fail(nullptr, QTM_ERR_NOMEM, "qtm_create: out of host memory");
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->alloc = g_allocator;
    ctx->n = n;
    ctx->n_c = p->n_c;
    ctx->n_obs = p->n_obs;
    ctx->n_t = p->n_t;
    ctx->precision = p->precision;
    ctx->flags = p->flags;
    ctx->max_jumps = (p->flags & QTM_FLAG_RECORD_JUMPS) ? p->max_jumps_recorded : 0;
    ctx->rtol = p->rtol;
    ctx->atol = p->atol;
    ctx->max_steps = p->max_steps;
    ctx->t.assign(p->t, p->t + p->n_t);
    const double nrm = std::sqrt(nn);
    ctx->psi0.resize(n);
    for (int i = 0; i < n; ++i) ctx->psi0[i] = cd(p->psi0[2 * i] / nrm, p->psi0[2 * i + 1] / nrm);
    ctx->M = effective_matrix(H, C);
    ctx->Cops = C;
    ctx->Aops = A;
    for (int i = 0; i < p->n_obs; ++i) ctx->scale_exp.push_back(observable_scale(A[i]));
    {
        const double nu = op_norm_bound(ctx->M);  // >= ||M||_2
        const int e = nu > 0.0 ? std::ilogb(nu) + 1 : 0;
        ctx->krylov_shift = std::max(-100, std::min(100, e));
    }
    // the tensor-core engine's control warps use one lane per row group of 32
    repack(ctx, p->precision == QTM_PREC_BF16X6 ? qtm::Layout{32, qtm::tc_padded_dim(n) / 32}
                                                : qtm::layout_for_dim(n));
    if (p->precision != QTM_PREC_BF16X6 && ctx->layout.G <= 32) {
        // single-warp layouts keep the operators in shared memory beside four
        // trajectories' ten vector slots; operators that cannot fit there (dense
        // ones) go to the 64-lane layout, whose kernels read them from L2
        const size_t real_b = p->precision == QTM_PREC_C64 ? 4 : 8;
        const size_t cplx_b = p->precision == QTM_PREC_C64 ? 8 : 16;
        // threads per CTA of the plain kernel (trajectory_block): 320 for the
        // double-float and complex64 kernels with R x complex size <= 32 bytes
        const bool big = (p->precision == QTM_PREC_DF64 || p->precision == QTM_PREC_C64) &&
                         ctx->layout.R * cplx_b <= 32;
        const size_t groups = (big ? 320 : 128) / ctx->layout.G;
        const size_t need = ctx->ints.size() * 4 + ctx->reals.size() * real_b +
                            groups * 10 * (size_t)ctx->layout.G * ctx->layout.R * cplx_b + 4096;
        if (need > 220 * 1024) repack(ctx, qtm::Layout{64, 2});
    }

    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        qtm_status s = cuda_fail(nullptr, e, "qtm_create: cudaGetDevice");
        delete ctx;
        return s;
    }
    // device representation of the complex values for the chosen arithmetic
    std::vector<unsigned char> vals_dev = encode_reals(ctx->reals, ctx->precision);
    std::vector<unsigned char> psi0_dev = encode_values(ctx->psi0, ctx->precision);
    const size_t ib = ctx->ints.size() * sizeof(int), vb = vals_dev.size();
    struct {
        DevBuf *b;
        size_t bytes;
    } allocs[] = {{&ctx->d_ints, ib}, {&ctx->d_vals, vb}, {&ctx->d_t, ctx->t.size() * sizeof(double)},
                  {&ctx->d_psi0, psi0_dev.size()}, {&ctx->d_queue, 16},
                  {&ctx->d_counters, qtm::kNumCounters * sizeof(unsigned long long)},
                  {&ctx->d_first_error, 16}, {&ctx->d_scale, ctx->scale_exp.size() * sizeof(int)}};
    for (cudaEvent_t &ev : ctx->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
            qtm_status s = cuda_fail(nullptr, e, "qtm_create: cudaEventCreate");
            destroy_ctx(ctx);
            return s;
        }
    for (auto &al : allocs) {
        if ((e = dev_alloc(ctx, *al.b, al.bytes)) != cudaSuccess) {
            qtm_status s = cuda_fail(nullptr, e, "qtm_create: device allocation");
            destroy_ctx(ctx);
            return s == QTM_ERR_CUDA && e == cudaErrorMemoryAllocation ? QTM_ERR_NOMEM : s;
        }
    }
    if ((e = cudaMemcpyAsync(ctx->d_ints.p, ctx->ints.data(), ib, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_vals.p, vals_dev.data(), vb, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_t.p, ctx->t.data(), ctx->t.size() * sizeof(double),
                             cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_psi0.p, psi0_dev.data(), psi0_dev.size(), cudaMemcpyHostToDevice,
                             ctx->stream)) ||
        (!ctx->scale_exp.empty() &&
         (e = cudaMemcpyAsync(ctx->d_scale.p, ctx->scale_exp.data(), ctx->scale_exp.size() * sizeof(int),
                              cudaMemcpyHostToDevice, ctx->stream))) ||
        (e = cudaStreamSynchronize(ctx->stream))) {
        qtm_status s = cuda_fail(nullptr, e, "qtm_create: upload");
        destroy_ctx(ctx);
        return s;
    }
    if (ctx->precision == QTM_PREC_BF16X6) {
        qtm_status s = tc_setup(ctx);
        if (s) {
            g_create_error = ctx->err;
            destroy_ctx(ctx);
            return s;
        }
    }
    *out = ctx;
    return QTM_OK;
}

// Device buffers of a run of ntraj trajectories (grown, never shrunk).
static qtm_status reserve_run(qtm_ctx *ctx, int64_t ntraj)
{
    const size_t P = (size_t)ctx->n_t * ctx->n_obs;
    const int S = qtm::reduce_segments(ntraj);
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_out, (size_t)ntraj * P * sizeof(double))) ||
        (e = dev_reserve(ctx, ctx->d_partial, qtm::kMomentWords * (size_t)S * P * sizeof(long long))) ||
        (e = dev_reserve(ctx, ctx->d_moments, qtm::kMomentWords * P * sizeof(long long))))
        return cuda_fail(ctx, e, "qtm_run: device allocation");
    if (ctx->precision == QTM_PREC_BF16X6 && ctx->method == QTM_METHOD_EXPONENTIAL && ntraj > 0) {
        const size_t vb = (size_t)ntraj * 2 * ctx->np * sizeof(float);
        if ((e = dev_reserve(ctx, ctx->d_lpsi, vb)) || (e = dev_reserve(ctx, ctx->d_ly, vb)) ||
            (e = dev_reserve(ctx, ctx->d_lcol, (size_t)ntraj * qtm::kLockColBytes)) ||
            (e = dev_reserve(ctx, ctx->d_llist, (size_t)ntraj * sizeof(int))))
            return cuda_fail(ctx, e, "qtm_run: device allocation");
    } else if (ctx->precision == QTM_PREC_BF16X6 && ntraj > 0) {
        const size_t cols = (size_t)qtm::dense_tc_ctas(ntraj, ctx->sms) * qtm::kTcCols;
        if ((e = dev_reserve(ctx, ctx->d_state, qtm::kNumDenseVecs * cols * 2 * ctx->np * sizeof(float))) ||
            (e = dev_reserve(ctx, ctx->d_col, cols * sizeof(qtm::DenseCol))))
            return cuda_fail(ctx, e, "qtm_run: device allocation");
    }
    if (ctx->max_jumps > 0) {
        if ((e = dev_reserve(ctx, ctx->d_njumps, (size_t)ntraj * sizeof(int))) ||
            (e = dev_reserve(ctx, ctx->d_jump_t, (size_t)ntraj * ctx->max_jumps * sizeof(double))) ||
            (e = dev_reserve(ctx, ctx->d_jump_ch, (size_t)ntraj * ctx->max_jumps * sizeof(int))))
            return cuda_fail(ctx, e, "qtm_run: device allocation");
    }
    return QTM_OK;
}

// Enqueues one run on stream s (buffers reserved): counter resets, the
// trajectory kernel and the ensemble reduction; with_events brackets them with
// the context's timing events.  Performs no allocation, so it can be captured.
static qtm_status enqueue_run(qtm_ctx *ctx, int64_t first, int64_t ntraj, uint64_t seed, cudaStream_t s,
                              bool with_events)
{
    const size_t P = (size_t)ctx->n_t * ctx->n_obs;
    cudaError_t e;
    if (ctx->max_jumps > 0) {
        if ((e = cudaMemsetAsync(ctx->d_njumps.p, 0, (size_t)ntraj * sizeof(int), s)) ||
            (e = cudaMemsetAsync(ctx->d_jump_t.p, 0xff, (size_t)ntraj * ctx->max_jumps * sizeof(double), s)) ||
            (e = cudaMemsetAsync(ctx->d_jump_ch.p, 0xff, (size_t)ntraj * ctx->max_jumps * sizeof(int), s)))
            return cuda_fail(ctx, e, "qtm_run: cudaMemsetAsync");
    }
    if ((e = cudaMemsetAsync(ctx->d_queue.p, 0, 16, s)) ||
        (e = cudaMemsetAsync(ctx->d_counters.p, 0, qtm::kNumCounters * sizeof(unsigned long long), s)) ||
        (e = cudaMemsetAsync(ctx->d_first_error.p, 0, 16, s)))
        return cuda_fail(ctx, e, "qtm_run: cudaMemsetAsync");
    if (with_events && (e = cudaEventRecord(ctx->ev[0], s)) != cudaSuccess)
        return cuda_fail(ctx, e, "qtm_run: cudaEventRecord");
    if (ntraj > 0) {
        KernelArgs a{};
        a.n = ctx->n;
        a.n_c = ctx->n_c;
        a.n_obs = ctx->n_obs;
        a.n_t = ctx->n_t;
        a.G = ctx->layout.G;
        a.R = ctx->layout.R;
        a.ints = (const int *)ctx->d_ints.p;
        a.vals = ctx->d_vals.p;
        a.n_ints = (int)ctx->ints.size();
        a.n_vals = (int)ctx->reals.size();
        for (size_t i = 0; i < ctx->ops.size(); ++i) a.op[i] = ctx->ops[i];
        a.t = (const double *)ctx->d_t.p;
        a.psi0 = ctx->d_psi0.p;
        a.rtol = ctx->rtol;
        a.atol = ctx->atol;
        a.max_steps = ctx->max_steps;
        a.seed = seed;
        a.traj0 = first;
        a.ntraj = ntraj;
        a.queue = (unsigned long long *)ctx->d_queue.p;
        a.out = (double *)ctx->d_out.p;
        a.counters = (unsigned long long *)ctx->d_counters.p;
        a.first_error = (int *)ctx->d_first_error.p;
        a.max_jumps = ctx->max_jumps;
        a.n_jumps = (int *)ctx->d_njumps.p;
        a.jump_t = (double *)ctx->d_jump_t.p;
        a.jump_ch = (int *)ctx->d_jump_ch.p;
        a.n_drive = (int)ctx->Dops.size();
        a.drive_op0 = 1 + ctx->n_c + ctx->n_obs;
        for (int k = 0; k < a.n_drive; ++k)
            for (int q = 0; q < 3; ++q) a.drive[k][q] = ctx->drive[3 * k + q];
        a.rec_stride = ctx->rec_stride;
        a.rec_max = ctx->rec_max;
        a.rec = (float *)ctx->d_rec.p;
        a.mlp = ctx->mlp_on ? (const float *)ctx->d_mlp.p : nullptr;
        a.prop_margin = ctx->prop_margin;
        a.krylov_shift = ctx->krylov_shift;
        const bool prop = a.rec_stride > 0 || a.mlp != nullptr;
        if (ctx->precision == QTM_PREC_BF16X6 && ctx->method == QTM_METHOD_EXPONENTIAL) {
            if (prop) return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: no learned proposal on the tensor-core path");
            // lock-step exponential method: interval 0 starts every column; then
            // per output interval the tensor cores form (P_L - I) psi for all
            // columns and the per-interval kernel finishes each column's interval
            a.expo = ctx->d_expo.p;
            a.expo_levels = ctx->expo_levels;
            a.expo_uniform = 1;
            a.expo_delta = ctx->expo_delta;
            a.lock_psi = (float *)ctx->d_lpsi.p;
            a.lock_y = (const float *)ctx->d_ly.p;
            a.lock_col = ctx->d_lcol.p;
            a.lock_ld = 2 * ctx->np;
            a.lock_list = (int *)ctx->d_llist.p;
            a.dense = (const float2 *)ctx->d_dense.p;
            a.dense_ld = ctx->np;
            for (int i = 0; i < qtm::kMaxOps; ++i)
                a.dense_off[i] = i < (int)ctx->dense_off.size() && ctx->dense_off[i] >= 0 ? ctx->dense_off[i] : -1;
            qtm::DenseArgs d{};
            d.k = a;
            d.np = ctx->np;
            d.mode = qtm::kDenseRhs;
            d.wait_limit_ns = ctx->wait_limit_ns;
            d.rhs_in = (const float *)ctx->d_lpsi.p;
            d.rhs_out = (float *)ctx->d_ly.p;
            d.rhs_n = ntraj;
            qtm::LaunchInfo tc_info{};
            // a column whose norm crosses its threshold inside an interval leaves
            // the lock step until the next catch-up launch (every kCatchUpEvery
            // intervals and after the last), which resolves the deferred columns
            // with every group of the GPU working through the list, instead of
            // each interval waiting for its slowest crossing.  Measured on the
            // dense N = 256 workload: every 4 intervals 416k trajectories/s, 8
            // 475k, 12 493k, 16 507k, 24 and 32 the same as 16 (fewer, fuller
            // catch-ups outweigh the extra intervals a deferred column then makes
            // up on the ladder, up to 16)
            constexpr int kCatchUpEvery = 16;
            ctx->product_timed = with_events && ctx->n_t > 1;
            auto lockstep = [&](int mode, int j) -> qtm_status {
                a.lock_mode = mode;
                a.lock_j = j;
                const cudaError_t le = qtm::launch_expo_lockstep(a, s, &ctx->info);
                if (le == cudaErrorInvalidValue)
                    return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: no lock-step kernel fits this problem");
                if (le != cudaSuccess) return cuda_fail(ctx, le, "qtm_run: lock-step kernel launch");
                return QTM_OK;
            };
            qtm_status ls;
            for (int j = 0; j < ctx->n_t; ++j) {
                if (j == 1 && with_events && (e = cudaEventRecord(ctx->ev[3], s)) != cudaSuccess)
                    return cuda_fail(ctx, e, "qtm_run: cudaEventRecord");
                if (j > 0 && (e = qtm::launch_dense_tc(d, ctx->expo_map, s, &tc_info)) != cudaSuccess)
                    return cuda_fail(ctx, e, "qtm_run: tensor-core product launch");
                if (j == 1 && with_events && (e = cudaEventRecord(ctx->ev[4], s)) != cudaSuccess)
                    return cuda_fail(ctx, e, "qtm_run: cudaEventRecord");
                if ((ls = lockstep(qtm::kLockInterval, j))) return ls;
                if (j > 0 && (j % kCatchUpEvery == 0 || j == ctx->n_t - 1)) {
                    if ((ls = lockstep(qtm::kLockCatchUp, j))) return ls;
                    if ((e = cudaMemsetAsync(ctx->d_queue.p, 0, 16, s)) != cudaSuccess)
                        return cuda_fail(ctx, e, "qtm_run: cudaMemsetAsync");
                }
            }
            if ((ls = lockstep(qtm::kLockFinish, 0))) return ls;
        } else if (ctx->precision == QTM_PREC_BF16X6) {
            if (prop) return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: no learned proposal on the tensor-core path");
            qtm::DenseArgs d{};
            d.k = a;
            d.np = ctx->np;
            d.cols = qtm::dense_tc_ctas(ntraj, ctx->sms) * qtm::kTcCols;
            d.state = (float *)ctx->d_state.p;
            d.col = (qtm::DenseCol *)ctx->d_col.p;
            d.mode = qtm::kDenseRun;
            d.wait_limit_ns = ctx->wait_limit_ns;
            d.dense = (const float2 *)ctx->d_dense.p;
            for (int i = 0; i < qtm::kMaxOps; ++i)
                d.dense_off[i] = i < (int)ctx->dense_off.size() ? ctx->dense_off[i] : -1;
            e = qtm::launch_dense_tc(d, ctx->op_map, s, &ctx->info);
            if (e == cudaErrorInvalidValue)
                return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: no tensor-core kernel fits this problem");
            if (e != cudaSuccess) return cuda_fail(ctx, e, "qtm_run: tensor-core kernel launch");
        } else {
        if (prop && (ctx->precision == QTM_PREC_C64 || ctx->layout.G > 32))
            return fail(ctx, QTM_ERR_UNSUPPORTED,
                        "qtm_run: the learned proposal needs complex128 or double-float and dimension <= 64");
        if (prop && a.n_drive > 0)
            return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: the learned proposal takes a constant Hamiltonian");
        if (ctx->method == QTM_METHOD_EXPONENTIAL && a.n_drive > 0)
            return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: the exponential method takes a constant Hamiltonian");
        if (ctx->method == QTM_METHOD_EXPONENTIAL) {
            a.expo = ctx->d_expo.p;
            a.expo_levels = ctx->expo_levels;
            a.expo_uniform = ctx->expo_uniform;
            a.expo_delta = ctx->expo_delta;
            if (prop)
                e = ctx->precision == QTM_PREC_DF64 ? qtm::launch_mcwf_df64_expo_prop(a, s, &ctx->info)
                                                    : qtm::launch_mcwf_c128_expo_prop(a, s, &ctx->info);
            else
                e = ctx->precision == QTM_PREC_DF64  ? qtm::launch_mcwf_df64_expo(a, s, &ctx->info)
                  : ctx->precision == QTM_PREC_C64   ? qtm::launch_mcwf_c64_expo(a, s, &ctx->info)
                                                     : qtm::launch_mcwf_c128_expo(a, s, &ctx->info);
        } else if (a.n_drive > 0)
            e = ctx->precision == QTM_PREC_DF64  ? qtm::launch_mcwf_df64_drive(a, s, &ctx->info)
              : ctx->precision == QTM_PREC_C64   ? qtm::launch_mcwf_c64_drive(a, s, &ctx->info)
                                                 : qtm::launch_mcwf_c128_drive(a, s, &ctx->info);
        else if (ctx->precision == QTM_PREC_DF64)
            e = prop ? qtm::launch_mcwf_df64_prop(a, s, &ctx->info) : qtm::launch_mcwf_df64(a, s, &ctx->info);
        else if (ctx->precision == QTM_PREC_C64)
            e = qtm::launch_mcwf_c64(a, s, &ctx->info);
        else
            e = prop ? qtm::launch_mcwf_c128_prop(a, s, &ctx->info) : qtm::launch_mcwf_c128(a, s, &ctx->info);
        if (e == cudaErrorInvalidValue)
            return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_run: no trajectory kernel fits this problem");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "qtm_run: trajectory kernel launch");
        }
    }
    if (with_events && (e = cudaEventRecord(ctx->ev[1], s)) != cudaSuccess)
        return cuda_fail(ctx, e, "qtm_run: cudaEventRecord");
    e = qtm::launch_ensemble_moments((const double *)ctx->d_out.p, ntraj, (int)P, ctx->n_obs,
                                     (const int *)ctx->d_scale.p, (long long *)ctx->d_partial.p,
                                     (long long *)ctx->d_moments.p, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qtm_run: ensemble reduction launch");
    if (with_events && (e = cudaEventRecord(ctx->ev[2], s)) != cudaSuccess)
        return cuda_fail(ctx, e, "qtm_run: cudaEventRecord");
    return QTM_OK;
}

qtm_status qtm_run_range(qtm_ctx *ctx, int64_t first, int64_t ntraj, uint64_t seed)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_run: ctx is NULL");
    ctx->err.clear();
    if (first < 0 || ntraj < 0) return fail(ctx, QTM_ERR_ARG, "qtm_run: first and ntraj must be >= 0");
    if (ntraj > ((int64_t)1 << 40)) return fail(ctx, QTM_ERR_ARG, "qtm_run: ntraj too large");
    qtm_status st = reserve_run(ctx, ntraj);
    if (st) return st;
    if ((st = enqueue_run(ctx, first, ntraj, seed, ctx->stream, true))) return st;
    ctx->timed = true;
    ctx->last_ntraj = ntraj;
    return QTM_OK;
}

qtm_status qtm_run_batch(qtm_ctx *const *ctxs, const int64_t *first, const int64_t *ntraj, int32_t n,
                         uint64_t seed)
{
    if (!ctxs || !ntraj || n < 1) return fail(nullptr, QTM_ERR_ARG, "qtm_run_batch: need n >= 1 contexts");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(nullptr, QTM_ERR_ARG, "qtm_run_batch: NULL context");
        if (ntraj[i] < 0 || ntraj[i] > ((int64_t)1 << 40))
            return fail(ctxs[i], QTM_ERR_ARG, "qtm_run_batch: ntraj out of range");
        if (first && first[i] < 0) return fail(ctxs[i], QTM_ERR_ARG, "qtm_run_batch: first must be >= 0");
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(ctxs[i], QTM_ERR_ARG, "qtm_run_batch: contexts on different devices");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(ctxs[i], QTM_ERR_ARG, "qtm_run_batch: context listed twice");
    }
    for (int i = 0; i < n; ++i) {
        ctxs[i]->err.clear();
        qtm_status st = reserve_run(ctxs[i], ntraj[i]);
        if (st) return st;
    }
    qtm_ctx *lead = ctxs[0];
    cudaStream_t main = lead->stream;  // the graph runs here (may be the legacy stream)
    cudaStream_t cap = nullptr;        // capture happens on a private stream
    std::vector<cudaStream_t> branch(n, nullptr);
    std::vector<cudaEvent_t> joins(n, nullptr), before(n, nullptr);
    cudaEvent_t fork = nullptr, done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    qtm_status st = QTM_OK;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        if (graph) cudaGraphDestroy(graph);
        if (exec) cudaGraphExecDestroy(exec);  // released once the launched work completes
        for (auto &b : branch)
            if (b) cudaStreamDestroy(b);
        if (cap) cudaStreamDestroy(cap);
        for (auto &j : joins)
            if (j) cudaEventDestroy(j);
        for (auto &j : before)
            if (j) cudaEventDestroy(j);
        if (fork) cudaEventDestroy(fork);
        if (done) cudaEventDestroy(done);
    };
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    for (int i = 0; i < n && !e; ++i) {
        e = cudaStreamCreateWithFlags(&branch[i], cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
        if (!e) e = cudaEventCreateWithFlags(&before[i], cudaEventDisableTiming);
    }
    if (e) {
        cleanup();
        return cuda_fail(lead, e, "qtm_run_batch: stream/event creation");
    }
    // one graph: every system's run on its own branch, all branches joined; the
    // systems' persistent kernels overlap on the GPU
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed)) || (e = cudaEventRecord(fork, cap))) {
        cleanup();
        return cuda_fail(lead, e, "qtm_run_batch: capture");
    }
    for (int i = 0; i < n && st == QTM_OK; ++i) {
        if ((e = cudaStreamWaitEvent(branch[i], fork, 0))) break;
        st = enqueue_run(ctxs[i], first ? first[i] : 0, ntraj[i], seed, branch[i], false);
        if (st) break;
        if ((e = cudaEventRecord(joins[i], branch[i])) || (e = cudaStreamWaitEvent(cap, joins[i], 0))) break;
    }
    cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    if (st == QTM_OK && e == cudaSuccess) e = ec;
    if (st == QTM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    // the launch follows earlier work queued on every context's own stream
    for (int i = 1; i < n && st == QTM_OK && e == cudaSuccess; ++i)
        if (ctxs[i]->stream != main) {
            e = cudaEventRecord(before[i], ctxs[i]->stream);
            if (!e) e = cudaStreamWaitEvent(main, before[i], 0);
        }
    if (st == QTM_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, main);
    if (st == QTM_OK && e == cudaSuccess) e = cudaEventRecord(done, main);
    for (int i = 1; i < n && st == QTM_OK && e == cudaSuccess; ++i)
        if (ctxs[i]->stream != main) e = cudaStreamWaitEvent(ctxs[i]->stream, done, 0);
    cleanup();
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(lead, e, "qtm_run_batch: graph capture or launch");
    for (int i = 0; i < n; ++i) {
        ctxs[i]->timed = false;
        ctxs[i]->last_ntraj = ntraj[i];
    }
    return QTM_OK;
}

qtm_status qtm_run(qtm_ctx *ctx, int64_t ntraj, uint64_t seed) { return qtm_run_range(ctx, 0, ntraj, seed); }

// Uploads the exponential method's ladder in the device layout of the current
// lane layout: level l, column c at (l n + c) G R, rows >= n zero.
static qtm_status upload_ladder(qtm_ctx *ctx)
{
    const int n = ctx->n, NP = ctx->layout.G * ctx->layout.R;
    std::vector<cd> dev((size_t)ctx->expo_levels * n * NP, cd(0.0));
    for (int l = 0; l < ctx->expo_levels; ++l)
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < n; ++r)
                dev[((size_t)l * n + c) * NP + r] = ctx->ladder[((size_t)l * n + r) * n + c];
    std::vector<unsigned char> bytes = encode_values(dev, ctx->precision);
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_expo, bytes.size())) ||
        (e = cudaMemcpyAsync(ctx->d_expo.p, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_set_method: upload");
    return QTM_OK;
}

// Re-uploads the packed operators (after repack), and the ladder of the
// exponential method, whose device layout follows the lane layout.
static qtm_status upload_ops(qtm_ctx *ctx)
{
    if (ctx->method == QTM_METHOD_EXPONENTIAL) {
        qtm_status st = upload_ladder(ctx);
        if (st) return st;
    }
    std::vector<unsigned char> vals_dev = encode_reals(ctx->reals, ctx->precision);
    const size_t ib = ctx->ints.size() * sizeof(int), vb = vals_dev.size();
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_ints, ib)) || (e = dev_reserve(ctx, ctx->d_vals, vb)))
        return cuda_fail(ctx, e, "qtm_autotune: device allocation");
    if ((e = cudaMemcpyAsync(ctx->d_ints.p, ctx->ints.data(), ib, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_vals.p, vals_dev.data(), vb, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_autotune: upload");
    return QTM_OK;
}

qtm_status qtm_set_layout(qtm_ctx *ctx, int32_t group, int32_t rows)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_set_layout: ctx is NULL");
    ctx->err.clear();
    if (ctx->precision == QTM_PREC_BF16X6)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_layout: the tensor-core path has one fixed layout");
    qtm::Layout cand[2];
    const int nc = qtm::layout_candidates(ctx->n, cand);
    for (int i = 0; i < nc; ++i)
        if (cand[i].G == group && cand[i].R == rows) {
            repack(ctx, cand[i]);
            qtm_status st = upload_ops(ctx);
            if (st) return st;
            ctx->last_ntraj = -1;
            return QTM_OK;
        }
    return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_layout: not a layout for this dimension");
}

qtm_status qtm_autotune(qtm_ctx *ctx, int64_t sample, uint64_t seed, int32_t *group, int32_t *rows)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_autotune: ctx is NULL");
    ctx->err.clear();
    if (sample < 1 || sample > ((int64_t)1 << 40)) return fail(ctx, QTM_ERR_ARG, "qtm_autotune: sample must be >= 1");
    if (ctx->precision == QTM_PREC_BF16X6)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_autotune: the tensor-core path has one fixed layout");
    qtm::Layout cand[2];
    const int nc = qtm::layout_candidates(ctx->n, cand);
    if (nc < 1) return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_autotune: no layout for this dimension");
    qtm_status st = reserve_run(ctx, sample);
    if (st) return st;
    float best = 0.f;
    int best_i = -1;
    for (int i = 0; i < nc; ++i) {
        repack(ctx, cand[i]);
        if ((st = upload_ops(ctx))) return st;
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {  // first pass warms up
            st = enqueue_run(ctx, 0, sample, seed, ctx->stream, true);
            if (st == QTM_ERR_UNSUPPORTED) {
                ok = false;  // shared memory of this layout does not fit
                ctx->err.clear();
                break;
            }
            if (st) return st;
            cudaError_t e = cudaEventSynchronize(ctx->ev[2]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "qtm_autotune: timing");
            if ((e = cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[2])) != cudaSuccess)
                return cuda_fail(ctx, e, "qtm_autotune: timing");
        }
        if (ok && (best_i < 0 || ms < best)) {
            best = ms;
            best_i = i;
        }
    }
    if (best_i < 0) return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_autotune: no layout fits");
    repack(ctx, cand[best_i]);
    if ((st = upload_ops(ctx))) return st;
    ctx->last_ntraj = -1;  // the sample runs are not results
    if (group) *group = cand[best_i].G;
    if (rows) *rows = cand[best_i].R;
    return QTM_OK;
}

static qtm_status sync_and_status(qtm_ctx *ctx)
{
    if (ctx->last_ntraj < 0) return fail(ctx, QTM_ERR_STATE, "no qtm_run on this context yet");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int first = 0;
    e = cudaMemcpy(&first, ctx->d_first_error.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    if (first != 0) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "a trajectory stopped with %s", qtm_status_string((qtm_status)first));
        return fail(ctx, (qtm_status)first, buf);
    }
    return QTM_OK;
}

// The run's moment words (host copy) and, from them, any of mean / standard
// error / sum / sum of squares per output value (moments.h).
static qtm_status copy_moments(qtm_ctx *ctx, std::vector<long long> &w)
{
    const size_t P = (size_t)ctx->n_t * ctx->n_obs;
    w.assign(P * qtm::kMomentWords, 0);
    if (P == 0) return QTM_OK;
    cudaError_t e = cudaMemcpy(w.data(), ctx->d_moments.p, w.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? QTM_OK : cuda_fail(ctx, e, "cudaMemcpy");
}

static qtm_status finish_stats(qtm_ctx *ctx, double *mean, double *se, double *sum, double *sumsq)
{
    std::vector<long long> w;
    qtm_status s = copy_moments(ctx, w);
    if (s) return s;
    const size_t P = (size_t)ctx->n_t * ctx->n_obs;
    for (size_t p = 0; p < P; ++p)
        qtm::moments_finish(w.data() + p * qtm::kMomentWords, ctx->last_ntraj, ctx->scale_exp[p % ctx->n_obs],
                            mean ? mean + p : nullptr, se ? se + p : nullptr, sum ? sum + p : nullptr,
                            sumsq ? sumsq + p : nullptr);
    return QTM_OK;
}

qtm_status qtm_expect(qtm_ctx *ctx, double *mean, double *stderr_out)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_expect: ctx is NULL");
    if (!mean) return fail(ctx, QTM_ERR_ARG, "qtm_expect: mean is NULL");
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    qtm_status s = finish_stats(ctx, mean, stderr_out, nullptr, nullptr);
    return s ? s : run_status;
}

qtm_status qtm_sums(qtm_ctx *ctx, double *sum, double *sumsq, int64_t *count)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_sums: ctx is NULL");
    if (!sum || !sumsq || !count) return fail(ctx, QTM_ERR_ARG, "qtm_sums: NULL output");
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    qtm_status s = finish_stats(ctx, nullptr, nullptr, sum, sumsq);
    if (s) return s;
    *count = ctx->last_ntraj;
    return run_status;
}

qtm_status qtm_moments(qtm_ctx *ctx, int64_t *words, int64_t *count, int32_t *scale_exp)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_moments: ctx is NULL");
    if (!words || !count) return fail(ctx, QTM_ERR_ARG, "qtm_moments: NULL output");
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    std::vector<long long> w;
    qtm_status s = copy_moments(ctx, w);
    if (s) return s;
    std::memcpy(words, w.data(), w.size() * sizeof(long long));
    *count = ctx->last_ntraj;
    if (scale_exp)
        for (int k = 0; k < ctx->n_obs; ++k) scale_exp[k] = ctx->scale_exp[k];
    return run_status;
}

qtm_status qtm_moments_device(qtm_ctx *ctx, int64_t *words_dev)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_moments_device: ctx is NULL");
    if (!words_dev) return fail(ctx, QTM_ERR_ARG, "qtm_moments_device: NULL output");
    if (ctx->last_ntraj < 0) return fail(ctx, QTM_ERR_STATE, "no qtm_run on this context yet");
    const size_t P = (size_t)ctx->n_t * ctx->n_obs;
    if (P == 0) return QTM_OK;
    cudaError_t e = cudaMemcpyAsync(words_dev, ctx->d_moments.p, P * qtm::kMomentWords * sizeof(long long),
                                    cudaMemcpyDeviceToDevice, ctx->stream);
    return e == cudaSuccess ? QTM_OK : cuda_fail(ctx, e, "qtm_moments_device: cudaMemcpyAsync");
}

qtm_status qtm_scale_exponents(const qtm_problem *p, int32_t *scale_exp)
{
    if (!p || !scale_exp) return fail(nullptr, QTM_ERR_ARG, "qtm_scale_exponents: NULL argument");
    if (p->dim < 1 || p->n_obs < 0 || (p->n_obs > 0 && !p->A))
        return fail(nullptr, QTM_ERR_ARG, "qtm_scale_exponents: need dim >= 1 and the n_obs observables");
    char buf[32];
    for (int i = 0; i < p->n_obs; ++i) {
        std::snprintf(buf, sizeof buf, "A[%d]", i);
        Csr A;
        qtm_status st = read_op(p->A[i], p->dim, buf, A);
        if (st) return st;
        scale_exp[i] = observable_scale(A);
    }
    return QTM_OK;
}

qtm_status qtm_traj_expect(qtm_ctx *ctx, double *out)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_traj_expect: ctx is NULL");
    if (!out) return fail(ctx, QTM_ERR_ARG, "qtm_traj_expect: out is NULL");
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    const size_t bytes = (size_t)ctx->last_ntraj * ctx->n_t * ctx->n_obs * sizeof(double);
    if (bytes) {
        cudaError_t e = cudaMemcpy(out, ctx->d_out.p, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    }
    return run_status;
}

qtm_status qtm_jumps(qtm_ctx *ctx, int32_t *n_jumps, double *jump_t, int32_t *jump_ch)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_jumps: ctx is NULL");
    if (ctx->max_jumps == 0) return fail(ctx, QTM_ERR_STATE, "qtm_jumps: context was created without QTM_FLAG_RECORD_JUMPS");
    if (!n_jumps || !jump_t || !jump_ch) return fail(ctx, QTM_ERR_ARG, "qtm_jumps: NULL output");
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    const size_t nt = (size_t)ctx->last_ntraj;
    if (nt) {
        cudaError_t e;
        if ((e = cudaMemcpy(n_jumps, ctx->d_njumps.p, nt * sizeof(int), cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(jump_t, ctx->d_jump_t.p, nt * ctx->max_jumps * sizeof(double), cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(jump_ch, ctx->d_jump_ch.p, nt * ctx->max_jumps * sizeof(int), cudaMemcpyDeviceToHost)))
            return cuda_fail(ctx, e, "cudaMemcpy");
    }
    return run_status;
}

qtm_status qtm_stats(qtm_ctx *ctx, qtm_stats_t *out)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_stats: ctx is NULL");
    if (!out) return fail(ctx, QTM_ERR_ARG, "qtm_stats: out is NULL");
    std::memset(out, 0, sizeof(*out));
    qtm_status run_status = sync_and_status(ctx);
    if (run_status == QTM_ERR_STATE || run_status == QTM_ERR_CUDA) return run_status;
    unsigned long long c[qtm::kNumCounters];
    cudaError_t e = cudaMemcpy(c, ctx->d_counters.p, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    out->trajectories = ctx->last_ntraj;
    out->accepted = (int64_t)c[qtm::kAccepted];
    out->rejected = (int64_t)c[qtm::kRejected];
    out->rhs_evals = (int64_t)c[qtm::kRhs];
    out->jumps = (int64_t)c[qtm::kJumps];
    out->root_iters = (int64_t)c[qtm::kRootIters];
    out->failed = (int64_t)c[qtm::kFailed];
    out->proposal_misses = (int64_t)c[qtm::kPropMiss];
    out->first_error = (int32_t)run_status;
    out->kernel_group = ctx->info.group;
    out->kernel_rows = ctx->info.rows;
    out->grid = ctx->info.grid;
    out->block = ctx->info.block;
    if (ctx->timed) {
        float ms = 0.f;
        if (ctx->last_ntraj > 0 && cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess)
            out->kernel_ms = ms;
        if (cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]) == cudaSuccess) out->reduce_ms = ms;
        if (ctx->product_timed && ctx->method == QTM_METHOD_EXPONENTIAL && ctx->precision == QTM_PREC_BF16X6 &&
            cudaEventElapsedTime(&ms, ctx->ev[3], ctx->ev[4]) == cudaSuccess)
            out->product_ms = ms;
    }
    return QTM_OK;
}

// ---------------------------------------------------------------------------
// learned jump-time proposal
// ---------------------------------------------------------------------------

namespace {
// splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): deterministic initialisation and shuffling
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double uniform01(uint64_t &x) { return (double)(splitmix64(x) >> 11) * 0x1.0p-53; }

// constant-rate estimate of the time left: log(<psi|psi> / r) / Gamma
double rate_estimate(const float *f) { return (std::log((double)f[2]) - (double)f[3]) / (double)f[0]; }

// The proposal is compiled into the complex128 and double-float kernels of the
// single-warp lane layouts only.
bool proposal_supported(const qtm_ctx *ctx)
{
    return (ctx->precision == QTM_PREC_C128 || ctx->precision == QTM_PREC_DF64) && ctx->layout.G <= 32;
}
}  // namespace

qtm_status qtm_proposal_collect(qtm_ctx *ctx, int64_t ntraj, uint64_t seed, int32_t stride, int32_t max_per_traj,
                                int64_t *npairs)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_collect: ctx is NULL");
    ctx->err.clear();
    if (ntraj < 1 || stride < 1 || max_per_traj < 1 || ntraj > ((int64_t)1 << 32))
        return fail(ctx, QTM_ERR_ARG, "qtm_proposal_collect: need ntraj, stride, max_per_traj >= 1");
    if (!proposal_supported(ctx))
        return fail(ctx, QTM_ERR_UNSUPPORTED,
                    "qtm_proposal_collect: the proposal needs complex128 or double-float and dimension <= 64");
    qtm_status st = reserve_run(ctx, ntraj);
    if (st) return st;
    const size_t rec_floats = (size_t)ntraj * max_per_traj * qtm::kRecFloats;
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_rec, rec_floats * sizeof(float))) ||
        (e = cudaMemsetAsync(ctx->d_rec.p, 0xff, rec_floats * sizeof(float), ctx->stream)))
        return cuda_fail(ctx, e, "qtm_proposal_collect: record buffer");
    const bool was_on = ctx->mlp_on;
    ctx->mlp_on = false;  // pairs come from the plain method
    ctx->rec_stride = stride;
    ctx->rec_max = max_per_traj;
    st = enqueue_run(ctx, 0, ntraj, seed, ctx->stream, true);
    ctx->rec_stride = 0;
    ctx->mlp_on = was_on;
    if (st) return st;
    ctx->timed = true;
    ctx->last_ntraj = ntraj;
    std::vector<float> rec(rec_floats);
    if ((e = cudaMemcpyAsync(rec.data(), ctx->d_rec.p, rec_floats * sizeof(float), cudaMemcpyDeviceToHost,
                             ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_proposal_collect: copy");
    ctx->pair_f.clear();
    ctx->pair_dt.clear();
    for (size_t q = 0; q < rec.size() / qtm::kRecFloats; ++q) {
        const float *r = &rec[q * qtm::kRecFloats];
        // a complete record: positive rate, a jump that followed, a finite estimate
        if (!(r[0] > 0.f) || !(r[7] > 0.f) || !std::isfinite(r[7])) continue;
        const double est = rate_estimate(r);
        if (!(est > 0.0) || !std::isfinite(est)) continue;
        ctx->pair_f.insert(ctx->pair_f.end(), r, r + qtm::kMlpIn);
        ctx->pair_dt.push_back(r[7]);
    }
    if (npairs) *npairs = (int64_t)ctx->pair_dt.size();
    return QTM_OK;
}

qtm_status qtm_proposal_pairs(qtm_ctx *ctx, float *features, float *dt, int64_t capacity)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_pairs: ctx is NULL");
    if (!features || !dt) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_pairs: NULL output");
    const int64_t n = std::min<int64_t>(capacity, (int64_t)ctx->pair_dt.size());
    std::memcpy(features, ctx->pair_f.data(), (size_t)n * qtm::kMlpIn * sizeof(float));
    std::memcpy(dt, ctx->pair_dt.data(), (size_t)n * sizeof(float));
    return QTM_OK;
}

qtm_status qtm_proposal_train(qtm_ctx *ctx, int32_t steps, int32_t batch, float lr, uint64_t seed, float *loss,
                              float *loss_rate_estimate)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_train: ctx is NULL");
    ctx->err.clear();
    const int64_t np = (int64_t)ctx->pair_dt.size();
    if (np < 64) return fail(ctx, QTM_ERR_STATE, "qtm_proposal_train: collect at least 64 pairs first");
    if (steps < 1 || batch < 1 || !(lr > 0.f)) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_train: bad settings");
    if (batch > np) batch = (int32_t)np;
    // feature normalisation and targets: y = log(true time left / constant-rate estimate)
    double mu[qtm::kMlpIn] = {0}, sd[qtm::kMlpIn] = {0};
    for (int64_t i = 0; i < np; ++i)
        for (int k = 0; k < qtm::kMlpIn; ++k) mu[k] += ctx->pair_f[i * qtm::kMlpIn + k];
    for (double &m : mu) m /= (double)np;
    for (int64_t i = 0; i < np; ++i)
        for (int k = 0; k < qtm::kMlpIn; ++k) {
            const double d = ctx->pair_f[i * qtm::kMlpIn + k] - mu[k];
            sd[k] += d * d;
        }
    for (double &s : sd) s = std::sqrt(s / (double)np) + 1e-12;
    std::vector<int64_t> order(np);
    for (int64_t i = 0; i < np; ++i) order[i] = i;
    uint64_t rng = seed ^ 0x5DEECE66DULL;
    for (int64_t i = np - 1; i > 0; --i) std::swap(order[i], order[(int64_t)(uniform01(rng) * (double)(i + 1))]);
    std::vector<float> X((size_t)np * qtm::kMlpIn), T((size_t)np);
    double base = 0.0;
    for (int64_t i = 0; i < np; ++i) {
        const float *f = &ctx->pair_f[order[i] * qtm::kMlpIn];
        for (int k = 0; k < qtm::kMlpIn; ++k) X[i * qtm::kMlpIn + k] = (float)((f[k] - mu[k]) / sd[k]);
        T[i] = (float)std::log((double)ctx->pair_dt[order[i]] / rate_estimate(f));
        base += (double)T[i] * T[i];
    }
    // Glorot-uniform weights, zero biases
    std::vector<float> P(qtm::kMlpBlock, 0.f);
    auto glorot = [&](int off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) P[off + i] = (float)((2.0 * uniform01(rng) - 1.0) * a);
    };
    glorot(qtm::kOffW1, qtm::kMlpHidden, qtm::kMlpIn);
    glorot(qtm::kOffW2, qtm::kMlpHidden, qtm::kMlpHidden);
    glorot(qtm::kOffW3, 1, qtm::kMlpHidden);
    for (int k = 0; k < qtm::kMlpIn; ++k) {
        P[qtm::kOffMu + k] = (float)mu[k];
        P[qtm::kOffSd + k] = (float)sd[k];
    }
    const int tiles = qtm::mlp_tile_count(batch);
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_mlp, qtm::kMlpBlock * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_X, X.size() * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_T, T.size() * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_gpart, (size_t)tiles * qtm::kMlpParams * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_lpart, (size_t)tiles * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_grad, qtm::kMlpParams * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_loss, 16)) ||
        (e = dev_reserve(ctx, ctx->d_m, qtm::kMlpParams * sizeof(float))) ||
        (e = dev_reserve(ctx, ctx->d_v, qtm::kMlpParams * sizeof(float))))
        return cuda_fail(ctx, e, "qtm_proposal_train: device allocation");
    if ((e = cudaMemcpyAsync(ctx->d_mlp.p, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_X.p, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(ctx->d_T.p, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemsetAsync(ctx->d_m.p, 0, qtm::kMlpParams * sizeof(float), ctx->stream)) ||
        (e = cudaMemsetAsync(ctx->d_v.p, 0, qtm::kMlpParams * sizeof(float), ctx->stream)))
        return cuda_fail(ctx, e, "qtm_proposal_train: upload");
    float *dP = (float *)ctx->d_mlp.p, *dX = (float *)ctx->d_X.p, *dT = (float *)ctx->d_T.p;
    for (int s = 0; s < steps; ++s) {
        int64_t off = ((int64_t)s * batch) % np;
        if (off + batch > np) off = 0;
        if ((e = qtm::mlp_loss_grad(dP, dX + off * qtm::kMlpIn, dT + off, batch, (float *)ctx->d_gpart.p,
                                    (float *)ctx->d_lpart.p, (float *)ctx->d_grad.p, (float *)ctx->d_loss.p,
                                    ctx->stream)) ||
            (e = qtm::mlp_adam_step(dP, (float *)ctx->d_m.p, (float *)ctx->d_v.p, (const float *)ctx->d_grad.p, lr,
                                    s + 1, ctx->stream)))
            return cuda_fail(ctx, e, "qtm_proposal_train: training kernels");
    }
    // final loss over every pair (network forward pass on the GPU)
    DevBuf dY;
    if ((e = dev_alloc(ctx, dY, (size_t)np * sizeof(float))) ||
        (e = qtm::mlp_forward(dP, dX, np, (float *)dY.p, ctx->stream)))
        return cuda_fail(ctx, e, "qtm_proposal_train: evaluation");
    std::vector<float> Y((size_t)np);
    e = cudaMemcpyAsync(Y.data(), dY.p, Y.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, dY);
    if (e) return cuda_fail(ctx, e, "qtm_proposal_train: evaluation");
    double l = 0.0;
    for (int64_t i = 0; i < np; ++i) l += ((double)Y[i] - T[i]) * ((double)Y[i] - T[i]);
    if (loss) *loss = (float)(l / (double)np);
    if (loss_rate_estimate) *loss_rate_estimate = (float)(base / (double)np);
    ctx->mlp_set = true;
    return QTM_OK;
}

qtm_status qtm_proposal_set(qtm_ctx *ctx, const float *params)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_set: ctx is NULL");
    if (!params) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_set: params is NULL");
    for (int k = 0; k < qtm::kMlpIn; ++k)
        if (!(params[qtm::kOffSd + k] > 0.f)) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_set: feature scales must be > 0");
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_mlp, qtm::kMlpBlock * sizeof(float))) ||
        (e = cudaMemcpyAsync(ctx->d_mlp.p, params, qtm::kMlpBlock * sizeof(float), cudaMemcpyHostToDevice,
                             ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_proposal_set: upload");
    ctx->mlp_set = true;
    return QTM_OK;
}

qtm_status qtm_proposal_get(qtm_ctx *ctx, float *params)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_get: ctx is NULL");
    if (!params) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_get: params is NULL");
    if (!ctx->mlp_set) return fail(ctx, QTM_ERR_STATE, "qtm_proposal_get: no network trained or set");
    cudaError_t e = cudaMemcpyAsync(params, ctx->d_mlp.p, qtm::kMlpBlock * sizeof(float), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    return e ? cuda_fail(ctx, e, "qtm_proposal_get: copy") : QTM_OK;
}

qtm_status qtm_proposal_enable(qtm_ctx *ctx, int32_t on, float margin)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_proposal_enable: ctx is NULL");
    if (on && !ctx->mlp_set) return fail(ctx, QTM_ERR_STATE, "qtm_proposal_enable: no network trained or set");
    if (!(margin > 0.f) || !(margin < 1.f)) return fail(ctx, QTM_ERR_ARG, "qtm_proposal_enable: margin in (0, 1)");
    if (on && !proposal_supported(ctx))
        return fail(ctx, QTM_ERR_UNSUPPORTED,
                    "qtm_proposal_enable: the proposal needs complex128 or double-float and dimension <= 64");
    ctx->mlp_on = on != 0;
    ctx->prop_margin = margin;
    return QTM_OK;
}

qtm_status qtm_mlp_loss_grad(const float *params, const float *x, const float *t, int64_t n, float *loss,
                             float *grad)
{
    if (!params || !x || !t || !loss || !grad || n < 1)
        return fail(nullptr, QTM_ERR_ARG, "qtm_mlp_loss_grad: NULL buffer or n < 1");
    const int tiles = qtm::mlp_tile_count(n);
    float *d = nullptr;
    const size_t nf = qtm::kMlpParams + (size_t)n * (qtm::kMlpIn + 1) + (size_t)tiles * (qtm::kMlpParams + 1) +
                      qtm::kMlpParams + 1;
    cudaError_t e = cudaMalloc(&d, nf * sizeof(float));
    if (e) return cuda_fail(nullptr, e, "qtm_mlp_loss_grad: cudaMalloc");
    float *dP = d, *dX = dP + qtm::kMlpParams, *dT = dX + n * qtm::kMlpIn, *dG = dT + n;
    float *dL = dG + (size_t)tiles * qtm::kMlpParams, *dgrad = dL + tiles, *dloss = dgrad + qtm::kMlpParams;
    if (!(e = cudaMemcpy(dP, params, qtm::kMlpParams * sizeof(float), cudaMemcpyHostToDevice)) &&
        !(e = cudaMemcpy(dX, x, (size_t)n * qtm::kMlpIn * sizeof(float), cudaMemcpyHostToDevice)) &&
        !(e = cudaMemcpy(dT, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice)) &&
        !(e = qtm::mlp_loss_grad(dP, dX, dT, n, dG, dL, dgrad, dloss, nullptr)) &&
        !(e = cudaMemcpy(grad, dgrad, qtm::kMlpParams * sizeof(float), cudaMemcpyDeviceToHost)))
        e = cudaMemcpy(loss, dloss, sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e ? cuda_fail(nullptr, e, "qtm_mlp_loss_grad") : QTM_OK;
}

qtm_status qtm_set_drive(qtm_ctx *ctx, int32_t n_terms, const qtm_op *H, const double *coef)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_set_drive: ctx is NULL");
    ctx->err.clear();
    if (n_terms < 0 || n_terms > qtm::kMaxDrive) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "qtm_set_drive: n_terms must be in [0, %d]", qtm::kMaxDrive);
        return fail(ctx, QTM_ERR_ARG, buf);
    }
    if (n_terms > 0 && (!H || !coef)) return fail(ctx, QTM_ERR_ARG, "qtm_set_drive: H or coef is NULL");
    if (n_terms > 0 && ctx->precision == QTM_PREC_BF16X6)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_drive: the tensor-core path has a constant operator");
    if (n_terms > 0 && ctx->method == QTM_METHOD_EXPONENTIAL)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_drive: the exponential method has a constant operator");
    if (1 + ctx->n_c + ctx->n_obs + n_terms > qtm::kMaxOps)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_drive: too many operators in total");
    std::vector<Csr> D(n_terms);
    for (int k = 0; k < n_terms; ++k) {
        char name[32];
        std::snprintf(name, sizeof name, "drive H[%d]", k);
        qtm_status st = read_op(H[k], ctx->n, name, D[k]);
        if (st) {
            ctx->err = g_create_error;
            return st;
        }
        if (!is_hermitian(D[k])) {
            std::snprintf(name, sizeof name, "qtm_set_drive: H[%d] is not Hermitian", k);
            return fail(ctx, QTM_ERR_ARG, name);
        }
        for (int q = 0; q < 3; ++q)
            if (!is_finite(coef[3 * k + q])) return fail(ctx, QTM_ERR_ARG, "qtm_set_drive: non-finite coefficient");
        for (cd &v : D[k].val) v *= cd(0.0, -1.0);  // -i H_k
    }
    ctx->Dops = std::move(D);
    ctx->drive.assign(coef, coef + 3 * (size_t)n_terms);
    repack(ctx, ctx->layout);
    qtm_status st = upload_ops(ctx);
    if (st) return st;
    ctx->last_ntraj = -1;
    return QTM_OK;
}

qtm_status qtm_set_wait_limit(qtm_ctx *ctx, uint64_t limit_ns)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_set_wait_limit: ctx is NULL");
    ctx->err.clear();
    ctx->wait_limit_ns = limit_ns;
    return QTM_OK;
}

qtm_status qtm_rhs_batch(qtm_ctx *ctx, int64_t n_vec, const double *y, double *my)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_rhs_batch: ctx is NULL");
    ctx->err.clear();
    if (n_vec < 0 || (n_vec > 0 && (!y || !my))) return fail(ctx, QTM_ERR_ARG, "qtm_rhs_batch: bad arguments");
    if (ctx->precision != QTM_PREC_BF16X6)
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_rhs_batch: only the tensor-core precision has a batched product");
    if (n_vec == 0) return QTM_OK;
    const int n = ctx->n, np = ctx->np, kd = 2 * np;
    std::vector<float> in((size_t)n_vec * kd, 0.f), res((size_t)n_vec * kd);
    for (int64_t v = 0; v < n_vec; ++v)
        for (int i = 0; i < n; ++i) {
            in[(size_t)v * kd + i] = (float)y[2 * ((size_t)v * n + i)];
            in[(size_t)v * kd + np + i] = (float)y[2 * ((size_t)v * n + i) + 1];
        }
    const size_t bytes = in.size() * sizeof(float);
    cudaError_t e;
    if ((e = dev_reserve(ctx, ctx->d_rhs, 16 + 2 * bytes)))
        return cuda_fail(ctx, e, "qtm_rhs_batch: device allocation");
    int *d_status = (int *)ctx->d_rhs.p;  // this call's own status word
    float *d_in = (float *)((char *)ctx->d_rhs.p + 16), *d_out = d_in + in.size();
    if ((e = cudaMemcpyAsync(d_in, in.data(), bytes, cudaMemcpyHostToDevice, ctx->stream)))
        return cuda_fail(ctx, e, "qtm_rhs_batch: upload");
    qtm::DenseArgs d{};
    d.k.first_error = d_status;
    d.np = np;
    d.mode = qtm::kDenseRhs;
    d.wait_limit_ns = ctx->wait_limit_ns;
    d.rhs_in = d_in;
    d.rhs_out = d_out;
    d.rhs_n = n_vec;
    if ((e = cudaMemsetAsync(d_status, 0, 16, ctx->stream)) ||
        (e = qtm::launch_dense_tc(d, ctx->op_map, ctx->stream, nullptr)) ||
        (e = cudaMemcpyAsync(res.data(), d_out, bytes, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return cuda_fail(ctx, e, "qtm_rhs_batch: product");
    int first = 0;
    if ((e = cudaMemcpy(&first, d_status, sizeof(int), cudaMemcpyDeviceToHost)))
        return cuda_fail(ctx, e, "qtm_rhs_batch: status");
    if (first) return fail(ctx, (qtm_status)first, "qtm_rhs_batch: a device wait gave up");
    // the engine's operator is 2^-shift M: scale back (exact)
    const double up = std::ldexp(1.0, ctx->krylov_shift);
    for (int64_t v = 0; v < n_vec; ++v)
        for (int i = 0; i < n; ++i) {
            my[2 * ((size_t)v * n + i)] = up * res[(size_t)v * kd + i];
            my[2 * ((size_t)v * n + i) + 1] = up * res[(size_t)v * kd + np + i];
        }
    return QTM_OK;
}

qtm_status qtm_set_method(qtm_ctx *ctx, int32_t method)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_set_method: ctx is NULL");
    ctx->err.clear();
    if (method == QTM_METHOD_DOPRI5) {
        if (ctx->precision == QTM_PREC_BF16X6 && ctx->method == QTM_METHOD_EXPONENTIAL) {
            // back to the Dormand-Prince engine's packing: one lane per row group of 32
            ctx->method = QTM_METHOD_DOPRI5;
            repack(ctx, qtm::Layout{32, ctx->np / 32});
            qtm_status st = upload_ops(ctx);
            if (st) return st;
        }
        ctx->method = QTM_METHOD_DOPRI5;
        ctx->last_ntraj = -1;
        return QTM_OK;
    }
    if (method != QTM_METHOD_EXPONENTIAL) return fail(ctx, QTM_ERR_ARG, "qtm_set_method: unknown method");
    if (!ctx->Dops.empty())
        return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_method: the exponential method takes a constant Hamiltonian");
    if (ctx->n > qtm::kMaxDimExpo) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "qtm_set_method: the exponential method takes dim <= %d", qtm::kMaxDimExpo);
        return fail(ctx, QTM_ERR_UNSUPPORTED, buf);
    }
    // the output spacing: the top level propagates one interval of a uniform grid
    double span = 1.0;
    int uniform = 0;
    if (ctx->n_t > 1) {
        const double mean = (ctx->t.back() - ctx->t.front()) / (ctx->n_t - 1);
        double gmax = 0.0;
        uniform = 1;
        for (int j = 1; j < ctx->n_t; ++j) {
            const double gap = ctx->t[j] - ctx->t[j - 1];
            gmax = std::max(gmax, gap);
            if (std::abs(gap - mean) > 1e-12 * mean) uniform = 0;
        }
        span = uniform ? mean : gmax;
    }
    if (ctx->precision == QTM_PREC_BF16X6 && ctx->n_t > 1 && !uniform)
        return fail(ctx, QTM_ERR_UNSUPPORTED,
                    "qtm_set_method: the exponential method on the tensor cores needs a uniform output grid");
    std::vector<cd> ladder;
    double delta = 0.0;
    const int levels = expm_ladder(ctx->M, span, ladder, delta);
    if (levels < 1) return fail(ctx, QTM_ERR_UNSUPPORTED, "qtm_set_method: ||M|| times the output spacing is too large");
    ctx->ladder = std::move(ladder);
    ctx->expo_levels = levels;
    ctx->expo_uniform = uniform;
    ctx->expo_delta = delta;
    const int was = ctx->method;
    ctx->method = QTM_METHOD_EXPONENTIAL;
    qtm_status st;
    if (ctx->precision == QTM_PREC_BF16X6) {
        // the per-interval kernel's lane layout (its groups read the operators and
        // the ladder from device memory), and for the tensor cores the bf16 splits
        // of D = P_L - I: the per-interval kernel forms y = psi + D psi in FP32 with
        // rounding to nearest, so the tensor cores' accumulation error (several
        // times that of an FP32 product, met once per interval by the state)
        // scales with ||D|| ~ ||M dt|| instead of ||P_L|| ~ 1
        const int n = ctx->n;
        repack(ctx, n <= 64 ? qtm::Layout{32, 2} : n <= 128 ? qtm::Layout{64, 2} : qtm::Layout{128, 2});
        st = upload_ops(ctx);  // operators and ladder
        if (!st) {
            std::vector<cd> D(ctx->ladder.begin() + (size_t)(levels - 1) * n * n,
                              ctx->ladder.begin() + (size_t)levels * n * n);
            for (int i = 0; i < n; ++i) D[(size_t)i * n + i] -= 1.0;
            std::vector<uint16_t> op = tc_operator_dense(D.data(), n, ctx->np);
            cudaError_t e;
            if ((e = dev_reserve(ctx, ctx->d_op_expo, op.size() * sizeof(uint16_t))) ||
                (e = cudaMemcpyAsync(ctx->d_op_expo.p, op.data(), op.size() * sizeof(uint16_t),
                                     cudaMemcpyHostToDevice, ctx->stream)) ||
                (e = cudaStreamSynchronize(ctx->stream)))
                st = cuda_fail(ctx, e, "qtm_set_method: upload");
            else
                st = tc_make_map(ctx, ctx->d_op_expo.p, &ctx->expo_map);
        }
        if (st) {
            qtm_set_method(ctx, QTM_METHOD_DOPRI5);  // repacks for the engine
            return st;
        }
    } else {
        st = upload_ladder(ctx);
        if (st) {
            ctx->method = was == QTM_METHOD_EXPONENTIAL ? QTM_METHOD_DOPRI5 : was;
            return st;
        }
    }
    ctx->last_ntraj = -1;
    return QTM_OK;
}

qtm_status qtm_expo_ladder(const qtm_ctx *ctx, int32_t *levels, double *delta)
{
    if (!ctx) return fail(nullptr, QTM_ERR_ARG, "qtm_expo_ladder: ctx is NULL");
    if (ctx->method != QTM_METHOD_EXPONENTIAL) return QTM_ERR_STATE;
    if (levels) *levels = ctx->expo_levels;
    if (delta) *delta = ctx->expo_delta;
    return QTM_OK;
}

qtm_status qtm_propagator(const qtm_problem *p, double dt, double *out)
{
    g_create_error.clear();
    if (!p || !out) return fail(nullptr, QTM_ERR_ARG, "qtm_propagator: problem or out is NULL");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(nullptr, QTM_ERR_ARG, "qtm_propagator: need finite dt >= 0");
    const int n = p->dim;
    if (n < 1) return fail(nullptr, QTM_ERR_ARG, "qtm_propagator: dim must be >= 1");
    if (p->n_c < 0 || (p->n_c > 0 && !p->C)) return fail(nullptr, QTM_ERR_ARG, "qtm_propagator: bad collapse operators");
    Csr H;
    qtm_status st = read_op(p->H, n, "H", H);
    if (st) return st;
    if (!is_hermitian(H)) return fail(nullptr, QTM_ERR_ARG, "qtm_propagator: H is not Hermitian (tolerance 1e-12)");
    std::vector<Csr> C(p->n_c);
    for (int i = 0; i < p->n_c; ++i) {
        char buf[32];
        std::snprintf(buf, sizeof buf, "C[%d]", i);
        if ((st = read_op(p->C[i], n, buf, C[i]))) return st;
    }
    const Csr M = effective_matrix(H, C);
    const size_t nn = (size_t)n * n;
    if (dt == 0.0) {
        for (size_t i = 0; i < 2 * nn; ++i) out[i] = 0.0;
        for (int i = 0; i < n; ++i) out[2 * ((size_t)i * n + i)] = 1.0;
        return QTM_OK;
    }
    std::vector<cd> ladder;
    double delta = 0.0;
    const int levels = expm_ladder(M, dt, ladder, delta);
    if (levels < 1) return fail(nullptr, QTM_ERR_UNSUPPORTED, "qtm_propagator: ||M|| dt is too large");
    const cd *top = ladder.data() + (size_t)(levels - 1) * nn;
    for (size_t i = 0; i < nn; ++i) {
        out[2 * i] = top[i].real();
        out[2 * i + 1] = top[i].imag();
    }
    return QTM_OK;
}

void qtm_destroy(qtm_ctx *ctx) { destroy_ctx(ctx); }

}  // extern "C"
