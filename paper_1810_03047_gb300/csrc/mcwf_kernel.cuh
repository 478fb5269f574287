// mcwf_kernel.cuh -- the trajectory kernel: Algorithm 1 (Sec. 2.2) of the QTM
// paper for a whole ensemble in one persistent launch.
//
// Mapping onto the GPU.  G consecutive lanes of a warp own one trajectory; lane
// gl owns rows gl, gl+G, ... (R of them) of every Dormand-Prince vector.  The
// vectors of a trajectory -- the state psi, the candidate ynew, the seven stage
// derivatives K_0..K_6 and a two-half exchange buffer -- live in the group's
// slots of shared memory for the trajectory's whole life; nothing of the state
// touches HBM.  A lane reads and writes only its own rows of psi, ynew and K;
// the only data that crosses lanes is the vector entering each product M y,
// which goes through the exchange buffer (one warp-level barrier per product).
// All operators (M = -i H_eff, the C_n and the A_k) and the method's coefficient
// tables are staged once per CTA into shared memory.  Keeping the vectors in
// shared memory (not registers) lets the stage loops stay rolled, so the hot
// loop fits the instruction cache, and leaves registers for more resident warps.
// Groups pull trajectory ids from a global counter and start the next
// trajectory as soon as theirs ends, so uneven lifetimes do not idle lanes.
// Every decision (accept/reject, crossing, output times, channel) is taken from
// values reduced with a butterfly, which leaves the bitwise-identical value in
// every lane of the group, so control flow is uniform per group.
//
// The vector arithmetic is a policy (qtm_arith.cuh): complex128, double-float
// (FP64-class precision on the FP32 pipe) or complex64.  Time, step size, the
// crossing test and the jump-time root find are FP64 scalars in every policy.
//
// Per trajectory (paper step names):
//   (A) r_0, c_0 from Philox(seed, traj, k = 0); output 0 = psi0;
//   (B) Dormand-Prince 5(4) steps of dpsi/dt = M psi with error control; after an
//       accepted step the squared norm of ynew is compared with r;
//   (C) on a crossing, the time tau with ||psi(tau)||^2 = r is found on the
//       step's continuous extension (degree-10 polynomial in theta from a Gram
//       matrix, first sign change on an 8-point grid, then Newton with bisection
//       safeguard); outputs up to tau use the pre-jump interpolant; the channel
//       is n* = min{n : sum_{i<=n} w_i >= c_k sum_i w_i}, w_i = ||C_i psi(tau)||^2
//       (Eq. eqn:probability:of:cn), and psi <- C_n* psi(tau) / ||C_n* psi(tau)||
//       (Eq. eqn:state:for:new:time);
//   (D) k <- k + 1, new r_k, c_k; integration restarts at tau with the step size
//       of the accepted step.
#pragma once

#include "proposal.cuh"
#include "qtm_arith.cuh"
#include "qtm_device.cuh"
#include "qtm_launch.h"

namespace qtm {

// Vector slots of one trajectory group (each slot holds G * R complex rows).  The
// candidate ynew shares K_1's slot: K_1 has zero weight in the 5th-order
// solution, the error estimate and the continuous extension, so it is dead once
// the last stage vector has been formed.
enum Slot { kPsi = 0, kK0 = 1 /* K_q in kK0 + q, q = 0..6 */, kYn = 2 /* = K_1 */, kX0 = 8, kNumSlots = 10 };

// Method coefficients in the policy's arithmetic, staged per CTA.
template <class Ar>
struct Coefs {
    typename Ar::coef a[7][6];  // stage coupling a_sq (row 6 = 5th-order weights)
    typename Ar::coef e[7];     // error weights b_q - bhat_q
    typename Ar::coef W[7][5];  // continuous extension: coefficient of theta^(m+1) in w_j
};

// One operator in shared memory: its real and imaginary parts, each SELL-G (see OpOffsets).
template <class Ar>
struct CsrView {
    const int *tab_re, *col_re, *tab_im, *col_im;
    const typename Ar::real *val_re, *val_im;
};

template <class Ar>
__device__ __forceinline__ CsrView<Ar> csr_view(const OpOffsets &o, const int *si, const typename Ar::real *sv)
{
    return CsrView<Ar>{si + o.re.table, si + o.re.cols, si + o.im.table, si + o.im.cols,
                       sv + o.re.vals, sv + o.im.vals};
}

// The group's shared-memory view: slots plus the current exchange half.
template <class Ar, int G, int R>
struct Lanes {
    using cplx = typename Ar::cplx;
    static constexpr int NP = G * R;
    cplx *v;
    int gl, n, x;
    __device__ __forceinline__ cplx *slot(int s) const { return v + s * NP; }
    __device__ __forceinline__ cplx *kq(int q) const { return v + (kK0 + q) * NP; }
    // next half of the exchange buffer; every write to it is followed by a group
    // barrier before any lane reads, so a half is never rewritten while a lane
    // may still read it (that lane has passed the barrier of the write in between)
    __device__ __forceinline__ cplx *xnext()
    {
        x ^= 1;
        return v + (kX0 + x) * NP;
    }
};

// (A x)[row] for row = gl + G r (slice r of the SELL-G parts; the trip counts are
// uniform across the group, padded entries contribute 0 * x[0])
template <class Ar, int G>
__device__ __forceinline__ typename Ar::cplx spmv_row(const CsrView<Ar> &A, const typename Ar::cplx *x, int gl,
                                                      int r)
{
    typename Ar::acc acc;
    int off = A.tab_re[2 * r] + gl, w = A.tab_re[2 * r + 1];
    int t0 = 0;
    if (w > 0) {  // the first product starts the accumulator (the same bits as adding it to zero)
        acc = Ar::first_re(A.val_re[off], x[A.col_re[off]]);
        t0 = 1;
    } else {
        acc = Ar::zero();
    }
#pragma unroll 1
    for (int t = t0; t < w; ++t) Ar::mac_re(acc, A.val_re[off + t * G], x[A.col_re[off + t * G]]);
    off = A.tab_im[2 * r] + gl;
    w = A.tab_im[2 * r + 1];
#pragma unroll 1
    for (int t = 0; t < w; ++t) Ar::mac_im(acc, A.val_im[off + t * G], x[A.col_im[off + t * G]]);
    return Ar::get(acc);
}

// out[row] = (A x)[row] on the lane's rows
template <class Ar, int G, int R>
__device__ __forceinline__ void spmv_rows(const CsrView<Ar> &A, const typename Ar::cplx *x,
                                          typename Ar::cplx *out, int gl, int n)
{
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const typename Ar::cplx v = spmv_row<Ar, G>(A, x, gl, r);
        const int row = gl + G * r;
        if (row < n) out[row] = v;
    }
}

// v[r] = (D x)[gl + G r] for a dense complex64 operator D, column-major with
// column stride ld: one column per iteration, the group's rows of a column in
// consecutive lanes (coalesced loads), x_c broadcast from shared memory; sixteen
// columns in flight (the operator streams from L2 and the lock-step catch-ups
// are bound by the loads in flight: eight instead of four took the run from
// 290k to 395k trajectories/s, sixteen to 450k)
template <int G, int R>
__device__ __forceinline__ void dense_rows_f32(const float2 *D, int ld, const cpx<float> *x, int gl, int n,
                                               cpx<float> (&v)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cpx<float>{0.f, 0.f};
    const float2 *col = D + gl;
#pragma unroll 16
    for (int c = 0; c < n; ++c) {
        const cpx<float> xc = x[c];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (gl + G * r < n) {
                const float2 m = col[G * r];
                v[r].re = fmaf(m.x, xc.re, fmaf(-m.y, xc.im, v[r].re));
                v[r].im = fmaf(m.x, xc.im, fmaf(m.y, xc.re, v[r].im));
            }
        }
        col += ld;
    }
}

// out = A_i x on the lane's rows (x synchronised): from the dense FP32 copy when
// DENSE and the operator has one, else from the packed form
template <class Ar, int G, int R, bool DENSE>
__device__ __forceinline__ void op_rows(const KernelArgs &a, int i, const int *si, const typename Ar::real *sv,
                                        const typename Ar::cplx *x, typename Ar::cplx *out, int gl)
{
    if constexpr (DENSE) {
        static_assert(Ar::kId == 2, "dense operator copies are complex64");
        if (a.dense_off[i] >= 0) {
            cpx<float> v[R];
            dense_rows_f32<G, R>(a.dense + a.dense_off[i], a.dense_ld, x, gl, a.n, v);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (gl + G * r < a.n) out[gl + G * r] = v[r];
            return;
        }
    }
    spmv_rows<Ar, G, R>(csr_view<Ar>(a.op[i], si, sv), x, out, gl, a.n);
}

// dst = psi + h sum_j w_j K_j on the lane's rows (the continuous extension at theta)
template <class Ar, int G, int R>
__device__ __noinline__ void dense_rows(const Coefs<Ar> &C, const Lanes<Ar, G, R> &L, double h, double th,
                                           typename Ar::cplx *dst)
{
    typename Ar::coef w[7];
    Ar::weights(th, &C.W[0][0], w);
    const typename Ar::coef hc = Ar::coef_of(h);
    const typename Ar::cplx *psi = L.slot(kPsi);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = L.gl + G * r;
        if (row < L.n) {
            typename Ar::acc acc = Ar::zero();
#pragma unroll 1
            for (int j = 0; j < 7; ++j)
                if (j != 1) Ar::axpy(acc, w[j], L.kq(j)[row]);
            dst[row] = Ar::add_scaled(psi[row], hc, acc);
        }
    }
}

// The time-dependent part of the right-hand side: out[row] += f_k(time) (-i H_k x)[row]
// on the lane's rows, f_k = a_k cos(omega_k time + phi_k) in FP64 (x is the
// synchronised exchange vector the product M x was taken of).
template <class Ar, int G, int R>
__device__ __noinline__ void drive_rows(const KernelArgs &a, const int *si, const typename Ar::real *sv,
                                        const typename Ar::cplx *x, typename Ar::cplx *out, int gl,
                                        double time)
{
    for (int k = 0; k < a.n_drive; ++k) {
        const typename Ar::coef f = Ar::coef_of(a.drive[k][0] * cos(a.drive[k][1] * time + a.drive[k][2]));
        const CsrView<Ar> D = csr_view<Ar>(a.op[a.drive_op0 + k], si, sv);
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            const typename Ar::cplx v = spmv_row<Ar, G>(D, x, gl, r);
            const int row = gl + G * r;
            if (row < a.n) {
                typename Ar::acc acc = Ar::zero();
                Ar::axpy(acc, f, v);
                out[row] = Ar::add_scaled(out[row], Ar::coef_of(1.0), acc);
            }
        }
    }
}

// Output j: Re<y|A_k|y>/<y|y> for every observable, written by lane 0.  y is in
// the exchange half `y` and the group has synchronised after writing it.
// When obs is not NULL, lane 0 also stores the first two values there as floats.
template <class Ar, int G, int R>
__device__ __noinline__ void record_outputs(const KernelArgs &a, Group<G> g, const int *si,
                                            const typename Ar::real *sv, const typename Ar::cplx *y, int j,
                                            double *out, float *obs)
{
    using cplx = typename Ar::cplx;
    typename Ar::red nn = Ar::rzero();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = g.gl + G * r;
        if (row < a.n) nn = Ar::radd(nn, Ar::abs2(y[row]));
    }
    nn = Ar::rsum(g, nn);
    for (int k = 0; k < a.n_obs; ++k) {
        const CsrView<Ar> A = csr_view<Ar>(a.op[1 + a.n_c + k], si, sv);
        typename Ar::red ev = Ar::rzero();
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            const cplx ay = spmv_row<Ar, G>(A, y, g.gl, r);
            const int row = g.gl + G * r;
            if (row < a.n) ev = Ar::radd(ev, Ar::dot_re(y[row], ay));
        }
        ev = Ar::rsum(g, ev);
        const double value = Ar::ratio(ev, nn);
        if (g.gl == 0) {
            out[(size_t)j * a.n_obs + k] = value;
            if (obs && k < 2) obs[k] = (float)value;
        }
    }
}

// The learned proposal's network on features f (raw), evaluated by the group:
// thread gl computes hidden units gl, gl + G, ... of each layer; the first
// layer's activations pass through the group's 64-float scratch.
template <int G>
__device__ __noinline__ float mlp_eval(Group<G> g, const float *__restrict__ P, const float *f, float *h)
{
    g.sync();  // f was written by lane 0
    float x[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) x[i] = (f[i] - P[kOffMu + i]) / P[kOffSd + i];
    for (int j = g.gl; j < kMlpHidden; j += G) {
        float z = P[kOffB1 + j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) z = fmaf(P[kOffW1 + j * kMlpIn + i], x[i], z);
        h[j] = silu(z);
    }
    g.sync();
    float acc = 0.f;
    for (int k = g.gl; k < kMlpHidden; k += G) {
        float z = P[kOffB2 + k];
        for (int j = 0; j < kMlpHidden; ++j) z = fmaf(P[kOffW2 + k * kMlpHidden + j], h[j], z);
        acc = fmaf(P[kOffW3 + k], silu(z), acc);
    }
    acc = g.sum(acc);
    g.sync();
    return acc + P[kOffB3];
}

// Per-trajectory state of the learned proposal, kept in shared memory beside the
// network's scratch so that it takes no registers in the step loop.  Lane 0 alone
// writes it; the other lanes read it only after a group barrier.
struct PropState {
    float f[kMlpIn];   // features for the next step: Gamma, dGamma/dt, <psi|psi>, log r, two outputs
    float tmid;        // midpoint of the last accepted step, relative to the last jump
    float est;         // constant-rate estimate of the time left
    int rec_n, rec_open;
    double t_jump;     // time of the last jump (or the start)
    double h_ctrl;     // the controller's step when a proposed step replaced it
};
constexpr int kPropStride = kMlpHidden * 4 + (int)((sizeof(PropState) + 15) & ~size_t(15));

static __device__ __forceinline__ float *prop_records(const KernelArgs &a, long long il)
{
    return a.rec_stride > 0 ? a.rec + (size_t)il * a.rec_max * kRecFloats : nullptr;
}

// (lane 0) a fresh jump interval starting at t with threshold r
static __device__ __forceinline__ void prop_interval(PropState *P, double t, double r)
{
    P->f[0] = -1.f;
    P->f[1] = 0.f;
    P->f[2] = 1.f;
    P->f[3] = __logf((float)r);
    P->tmid = 0.f;
    P->t_jump = t;
}

// Before a step of size h at time t: stores a training record when one is due
// and, with a network loaded and the crossing near (constant-rate estimate within
// three steps), returns the proposed step ending a fraction prop_margin past the
// predicted crossing (0 when there is none).  Every lane gets the same value.
template <int G>
__device__ __noinline__ double prop_propose(const KernelArgs &a, Group<G> g, PropState *P, float *hscratch,
                                            long long il, unsigned long long n_acc, double t, double h)
{
    int want = 0;
    if (g.gl == 0 && P->f[0] > 0.f) {
        float *rec = prop_records(a, il);
        if (rec && P->rec_n < a.rec_max && n_acc % a.rec_stride == 0) {
            float *q = rec + (size_t)P->rec_n * kRecFloats;
            for (int i = 0; i < kMlpIn; ++i) q[i] = P->f[i];
            q[6] = (float)(t - P->t_jump);
            ++P->rec_n;
        }
        P->est = (__logf(P->f[2]) - P->f[3]) / P->f[0];
        want = a.mlp != nullptr && P->est < 3.f * (float)h;
    }
    if (!a.mlp) return 0.0;
    if (!g.bcast0(want)) return 0.0;
    const float y = mlp_eval<G>(g, a.mlp, P->f, hscratch);
    const double hp = (double)(P->est * __expf(y) * (1.f + a.prop_margin));
    return (hp < h && hp > 1e-3 * h) ? hp : 0.0;
}

// (lane 0) after an accepted step from t of size h ending with norm nn: the decay
// rate over the step from the norm ratio, and its slope against the last step's
static __device__ __noinline__ void prop_accepted(PropState *P, double nn, double t, double h)
{
    const float nnf = (float)nn, hf = (float)h;
    const float gam = -__logf(nnf / P->f[2]) / hf;
    const float tmid = (float)(t - P->t_jump) + 0.5f * hf;
    P->f[1] = P->f[0] > 0.f ? (gam - P->f[0]) / (tmid - P->tmid) : 0.f;
    P->f[0] = gam;
    P->f[2] = nnf;
    P->tmid = tmid;
}

// (lane 0) at a jump at tau: the interval's records get their time left, and the
// next interval starts with threshold r
static __device__ __noinline__ void prop_jumped(const KernelArgs &a, PropState *P, long long il, double tau, double r)
{
    float *rec = prop_records(a, il);
    if (rec) {
        const float left = (float)(tau - P->t_jump);
        for (int q = P->rec_open; q < P->rec_n; ++q) rec[(size_t)q * kRecFloats + 7] = left - rec[(size_t)q * kRecFloats + 6];
        P->rec_open = P->rec_n;
    }
    prop_interval(P, tau, r);
}

// The first theta in (0, 1] with f(theta) = sum_s P_s theta^s = 0, f(0) > 0: the
// first of eight sub-intervals whose right end has f < 0 brackets the root, then
// Newton's method with a bisection safeguard (FP64).  1 when f stays >= 0.
static __device__ __noinline__ double first_root(const double (&P)[11], int &iters)
{
    auto poly = [&](double x) {
        double f = P[10];
#pragma unroll
        for (int s = 9; s >= 0; --s) f = fma(f, x, P[s]);
        return f;
    };
    double lo = 0.0, hi = 1.0;
    bool found = false;
    for (int i = 1; i <= 8; ++i) {
        const double x = i / 8.0;
        if (poly(x) < 0.0) {
            lo = (i - 1) / 8.0;
            hi = x;
            found = true;
            break;
        }
    }
    if (!found) return 1.0;
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 100; ++it) {
        ++iters;
        double f = P[10], df = 0.0;
#pragma unroll
        for (int s = 9; s >= 0; --s) {
            df = fma(df, x, f);
            f = fma(f, x, P[s]);
        }
        if (f == 0.0) break;
        if (f < 0.0)
            hi = x;
        else
            lo = x;
        double xn = x - f / df;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 || hi - lo <= 1e-15) {
            x = xn;
            break;
        }
        x = xn;
    }
    return x;
}

// First theta in (0, 1] where ||y(theta)||^2 = r.  ||y(theta)||^2 = sum_s P_s theta^s
// with y(theta) = sum_m theta^m u_m, u_0 = psi, u_m = h sum_j W(j, m) K_j, and
// P_s = sum_{m + m' = s} Re<u_m, u_m'>.
template <class Ar, int G, int R>
__device__ __noinline__ double locate_crossing(const Coefs<Ar> &C, Lanes<Ar, G, R> L, Group<G> g, double h,
                                               double r, int &iters)
{
    using cplx = typename Ar::cplx;
    typename Ar::red gram[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) gram[q] = Ar::rzero();
    const typename Ar::coef hc = Ar::coef_of(h);
#pragma unroll 1
    for (int rr = 0; rr < R; ++rr) {
        const int row = L.gl + G * rr;
        if (row >= L.n) continue;
        cplx u[6];
        u[0] = L.slot(kPsi)[row];
#pragma unroll
        for (int m = 1; m <= 5; ++m) {
            typename Ar::acc acc = Ar::zero();
#pragma unroll
            for (int j = 0; j < 7; ++j)
                if (j != 1) Ar::axpy(acc, C.W[j][m - 1], L.kq(j)[row]);
            u[m] = Ar::add_scaled(Ar::czero(), hc, acc);
        }
        int q = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int m2 = m; m2 < 6; ++m2, ++q) gram[q] = Ar::radd(gram[q], Ar::dot_re(u[m], u[m2]));
    }
    double P[11];
#pragma unroll
    for (int s = 0; s < 11; ++s) P[s] = 0.0;
    {
        int q = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int m2 = m; m2 < 6; ++m2, ++q) {
                const double v = Ar::rval(Ar::rsum(g, gram[q]));
                P[m + m2] += (m == m2) ? v : 2.0 * v;
            }
    }
    P[0] -= r;
    return first_root(P, iters);
}

// Step (C) after the crossing time is known: y = psi(tau) is in a shared-memory
// vector (group synchronised).  Chooses the channel, writes C_n* y / ||C_n* y||
// to psi (lane rows; tmp is lane-row scratch), and returns the channel (or -1
// when every weight is zero).
// Channels whose products apply_jump keeps (DENSE: the scratch vectors after tmp)
constexpr int kJumpKeep = 9;

template <class Ar, int G, int R, bool DENSE = false>
__device__ __noinline__ int apply_jump(const KernelArgs &a, Group<G> g, const int *si,
                                       const typename Ar::real *sv, typename Ar::cplx *psi,
                                       typename Ar::cplx *tmp, const typename Ar::cplx *y, double ck)
{
    const int gl = g.gl, n = a.n;
    constexpr int NP = G * R;
    // DENSE (the exponential method's lock-step kernel): tmp heads kJumpKeep
    // scratch vectors, so each channel's C_q y is kept and the chosen one is not
    // formed a second time
    const bool keep = DENSE && a.n_c <= kJumpKeep;
    double wq[kMaxChannels];
    double wsum = 0.0;
    for (int q = 0; q < a.n_c; ++q) {
        typename Ar::cplx *dst = keep ? tmp + q * NP : tmp;
        op_rows<Ar, G, R, DENSE>(a, 1 + q, si, sv, y, dst, gl);
        typename Ar::red part = Ar::rzero();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) part = Ar::radd(part, Ar::abs2(dst[row]));
        }
        wq[q] = Ar::rval(Ar::rsum(g, part));
        wsum += wq[q];
    }
    if (!(wsum > 0.0)) return -1;
    const double target = ck * wsum;
    double cum = 0.0;
    int ch = a.n_c - 1;
    for (int q = 0; q < a.n_c; ++q) {
        cum += wq[q];
        if (cum >= target) {
            ch = q;
            break;
        }
    }
    if (!keep) op_rows<Ar, G, R, DENSE>(a, 1 + ch, si, sv, y, psi, gl);
    const typename Ar::cplx *cy = keep ? tmp + ch * NP : psi;
    const double nc = sqrt(wq[ch]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) psi[row] = Ar::div(cy[row], nc);
    }
    return ch;
}

// Compile-time features of an instantiation: the plain kernels carry neither.
enum Feature { kFeatProposal = 1, kFeatDrive = 2 };

template <class Ar, int G, int R, int FEAT>
__device__ void run_trajectory(const KernelArgs &a, const Group<G> &g, const int *si,
                               const typename Ar::real *sv, const Coefs<Ar> &C, Lanes<Ar, G, R> &L,
                               float *hscratch, PropState *P, long long il)
{
    constexpr bool PROP = (FEAT & kFeatProposal) != 0;
    constexpr bool DRIVE = (FEAT & kFeatDrive) != 0;
    using cplx = typename Ar::cplx;
    const int n = a.n;
    const int gl = g.gl;
    const long long traj = a.traj0 + il;
    const double t_end = a.t[a.n_t - 1];
    double *out = a.out + (size_t)il * a.n_t * a.n_obs;
    const CsrView<Ar> M = csr_view<Ar>(a.op[0], si, sv);
    const double rtol = a.rtol, atol = a.atol;
    cplx *psi = L.slot(kPsi);
    cplx *yn = L.slot(kYn);

    int status = 0;
    long long attempts = 0;
    unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0, n_jump = 0;
    int root_iters = 0;

    // (A)
    const cplx *psi0 = static_cast<const cplx *>(a.psi0);
    cplx *b = L.xnext();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) psi[row] = b[row] = psi0[row];
    }
    g.sync();
    long long k = 0;
    double rk, ck;
    jump_draws(a.seed, traj, k, rk, ck);
    double t = a.t[0];
    // learned proposal: its features live in P (FP32: the FP64 pipe is the scarce one)
    float *obs = nullptr;
    if constexpr (PROP) {
        if (gl == 0) {
            P->rec_n = P->rec_open = 0;
            prop_interval(P, t, rk);
        }
        obs = P->f + 4;
    }
    record_outputs<Ar, G, R>(a, g, si, sv, b, 0, out, obs);
    int j = 1;
    bool proposed = false;
    spmv_rows<Ar, G, R>(M, b, L.kq(0), gl, n);
    if constexpr (DRIVE) drive_rows<Ar, G, R>(a, si, sv, b, L.kq(0), gl, t);
    ++n_rhs;

    // starting step (Hairer, Norsett & Wanner, Sec. II.4), in FP64 scalars
    double h;
    {
        const double span = t_end - t;
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                const double yr = Ar::re(psi[row]), yi = Ar::im(psi[row]);
                const double fr = Ar::re(L.kq(0)[row]), fi = Ar::im(L.kq(0)[row]);
                const double sc = atol + rtol * sqrt(yr * yr + yi * yi);
                d0 += (yr * yr + yi * yi) / (sc * sc);
                d1 += (fr * fr + fi * fi) / (sc * sc);
            }
        }
        d0 = sqrt(g.sum(d0) / n);
        d1 = sqrt(g.sum(d1) / n);
        double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        if (h0 > span) h0 = span;
        const typename Ar::coef h0c = Ar::coef_of(h0);
        b = L.xnext();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                typename Ar::acc acc = Ar::zero();
                Ar::axpy(acc, Ar::coef_of(1.0), L.kq(0)[row]);
                b[row] = Ar::add_scaled(psi[row], h0c, acc);
            }
        }
        g.sync();
        cplx *f1 = L.kq(1);  // scratch: K_1 is recomputed by the first step
        spmv_rows<Ar, G, R>(M, b, f1, gl, n);
        if constexpr (DRIVE) drive_rows<Ar, G, R>(a, si, sv, b, f1, gl, t + h0);
        ++n_rhs;
        double d2 = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                const double yr = Ar::re(psi[row]), yi = Ar::im(psi[row]);
                const double sc = atol + rtol * sqrt(yr * yr + yi * yi);
                const double dre = Ar::re(f1[row]) - Ar::re(L.kq(0)[row]);
                const double dim = Ar::im(f1[row]) - Ar::im(L.kq(0)[row]);
                d2 += (dre * dre + dim * dim) / (sc * sc);
            }
        }
        d2 = sqrt(g.sum(d2) / n) / h0;
        const double dm = d1 > d2 ? d1 : d2;
        const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
        h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
        if (h > span) h = span;
    }

    bool rejected_before = false;
    while (j < a.n_t) {
        if (t_end - t <= 4.0 * 2.220446049250313e-16 * fabs(t_end)) {
            b = L.xnext();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) b[row] = psi[row];
            }
            g.sync();
            for (; j < a.n_t; ++j) record_outputs<Ar, G, R>(a, g, si, sv, b, j, out, obs);
            break;
        }
        if (attempts >= a.max_steps) {
            status = 4;
            break;
        }
        bool last = false;
        if (t + 1.01 * h >= t_end) {
            h = t_end - t;
            last = true;
        }
        if (h < 1e-14 * fmax(1.0, fabs(t))) {
            status = 5;
            break;
        }
        if constexpr (PROP) {
            proposed = false;
            const double hp = prop_propose<G>(a, g, P, hscratch, il, n_acc, t, h);
            if (hp > 0.0) {
                if (gl == 0) P->h_ctrl = h;
                h = hp;
                last = false;
                proposed = true;
            }
        }

        // (B): one Dormand-Prince attempt; K_6 = M ynew
        const typename Ar::coef hc = Ar::coef_of(h);
#pragma unroll 1
        for (int s = 1; s < 7; ++s) {
            b = L.xnext();
            if constexpr (Ar::kRowChains) {
                // the lane's R rows advance together: R independent accumulation chains
                typename Ar::acc acc[R];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = Ar::zero();
#pragma unroll 1
                for (int q = 0; q < s; ++q) {
                    const typename Ar::coef c = C.a[s][q];
                    const cplx *kq = L.kq(q);
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (gl + G * r < n) Ar::axpy(acc[r], c, kq[gl + G * r]);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int row = gl + G * r;
                    if (row < n) {
                        const cplx y = Ar::add_scaled(psi[row], hc, acc[r]);
                        b[row] = y;
                        if (s == 6) yn[row] = y;
                    }
                }
            } else {
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    const int row = gl + G * r;
                    if (row < n) {
                        typename Ar::acc acc = Ar::zero();
#pragma unroll 1
                        for (int q = 0; q < s; ++q) Ar::axpy(acc, C.a[s][q], L.kq(q)[row]);
                        const cplx y = Ar::add_scaled(psi[row], hc, acc);
                        b[row] = y;
                        if (s == 6) yn[row] = y;
                    }
                }
            }
            g.sync();
            spmv_rows<Ar, G, R>(M, b, L.kq(s), gl, n);
            if constexpr (DRIVE) drive_rows<Ar, G, R>(a, si, sv, b, L.kq(s), gl, t + DP5::c(s) * h);
        }
        n_rhs += 6;
        ++attempts;

        typename Ar::errt esum = 0;
        typename Ar::red nr = Ar::rzero();
        if constexpr (!Ar::kRowChains) {
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) {
                    typename Ar::acc e = Ar::zero();
#pragma unroll 1
                    for (int q = 0; q < 7; ++q)
                        if (q != 1) Ar::axpy(e, C.e[q], L.kq(q)[row]);
                    esum += Ar::err_term(e, h, psi[row], yn[row], rtol, atol);
                    nr = Ar::radd(nr, Ar::abs2(yn[row]));
                }
            }
        } else {
            typename Ar::acc e[R];
#pragma unroll
            for (int r = 0; r < R; ++r) e[r] = Ar::zero();
#pragma unroll 1
            for (int q = 0; q < 7; ++q) {
                if (q == 1) continue;
                const typename Ar::coef c = C.e[q];
                const cplx *kq = L.kq(q);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (gl + G * r < n) Ar::axpy(e[r], c, kq[gl + G * r]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) {
                    esum += Ar::err_term(e[r], h, psi[row], yn[row], rtol, atol);
                    nr = Ar::radd(nr, Ar::abs2(yn[row]));
                }
            }
        }
        const double err = Ar::err_final(Ar::err_sum(g, esum), n);

        if (!(err <= 1.0)) {
            if (!isfinite(err)) {
                status = 6;
                break;
            }
            double fac = Ar::controller(err);
            if (fac < kFacMin) fac = kFacMin;
            h *= fac;
            rejected_before = true;
            ++n_rej;
            continue;
        }
        ++n_acc;
        const double t_new = last ? t_end : t + h;
        const double nn = Ar::rval(Ar::rsum(g, nr));

        if (nn < rk) {
            // (C): the norm reached r inside this step
            const double th = locate_crossing<Ar, G, R>(C, L, g, h, rk, root_iters);
            double tau = t + th * h;
            if (tau > t_new) tau = t_new;
            for (; j < a.n_t && a.t[j] <= tau; ++j) {
                double thj = (a.t[j] - t) / h;
                if (thj > 1.0) thj = 1.0;
                b = L.xnext();
                dense_rows<Ar, G, R>(C, L, h, thj, b);
                g.sync();
                record_outputs<Ar, G, R>(a, g, si, sv, b, j, out, obs);
            }
            b = L.xnext();
            dense_rows<Ar, G, R>(C, L, h, th, b);
            g.sync();
            // ynew (in K_1's slot) is dead after a crossing: it serves as scratch
            const int ch = apply_jump<Ar, G, R>(a, g, si, sv, L.slot(kPsi), L.slot(kYn), b, ck);
            if (ch < 0) {
                status = 7;
                break;
            }
            if (gl == 0 && (long long)n_jump < a.max_jumps) {
                a.jump_t[(size_t)il * a.max_jumps + n_jump] = tau;
                a.jump_ch[(size_t)il * a.max_jumps + n_jump] = ch;
            }
            ++n_jump;

            if constexpr (PROP)
                if (proposed) h = P->h_ctrl;  // a proposed step was shortened on purpose

            // (D)
            ++k;
            jump_draws(a.seed, traj, k, rk, ck);
            if constexpr (PROP)
                if (gl == 0) prop_jumped(a, P, il, tau, rk);
            t = tau;
            b = L.xnext();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) b[row] = psi[row];
            }
            g.sync();
            spmv_rows<Ar, G, R>(M, b, L.kq(0), gl, n);
            if constexpr (DRIVE) drive_rows<Ar, G, R>(a, si, sv, b, L.kq(0), gl, t);
            ++n_rhs;
            rejected_before = false;
            continue;
        }

        for (; j < a.n_t && a.t[j] <= t_new; ++j) {
            double thj = (a.t[j] - t) / h;
            if (thj > 1.0) thj = 1.0;
            b = L.xnext();
            dense_rows<Ar, G, R>(C, L, h, thj, b);
            g.sync();
            record_outputs<Ar, G, R>(a, g, si, sv, b, j, out, obs);
        }
        double fac = (err == 0.0) ? kFacMax : Ar::controller(err);
        if (fac > kFacMax) fac = kFacMax;
        if (fac < kFacMin) fac = kFacMin;
        if (rejected_before && fac > 1.0) fac = 1.0;
        rejected_before = false;
        if constexpr (PROP) {
            if (gl == 0) prop_accepted(P, nn, t, h);
            if (proposed) {
                if (fac < 1.0) fac = 1.0;  // a shortened step says nothing about accuracy
                h = P->h_ctrl / fac;       // resume the controller's own step size below
            }
        }
        t = t_new;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                psi[row] = yn[row];
                L.kq(0)[row] = L.kq(6)[row];
            }
        }
        h *= fac;
    }

    if (gl == 0) {
        if (status != 0) {
            for (; j < a.n_t; ++j)
                for (int q = 0; q < a.n_obs; ++q)
                    out[(size_t)j * a.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
            atomicCAS(a.first_error, 0, status);
            atomicAdd(&a.counters[kFailed], 1ULL);
        }
        if (a.max_jumps > 0) a.n_jumps[il] = (int)n_jump;
        atomicAdd(&a.counters[kAccepted], n_acc);
        atomicAdd(&a.counters[kRejected], n_rej);
        atomicAdd(&a.counters[kRhs], n_rhs);
        atomicAdd(&a.counters[kJumps], n_jump);
        atomicAdd(&a.counters[kRootIters], (unsigned long long)root_iters);
    }
}

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4) in Krylov form, for a constant operator
// ---------------------------------------------------------------------------
//
// For dpsi/dt = M psi with a constant M every stage of an explicit Runge-Kutta
// step is a polynomial in hM applied to psi: h K_j = sum_k kappa_jk (hM)^k psi with
// kappa_j1 = 1 and kappa_j,k+1 = sum_l a_jl kappa_lk.  Hence the 5th-order solution
// is sum_{k<=6} beta_k (hM)^k psi (beta_k = sum_j b_j kappa_jk, beta_0 = 1), the
// local error estimate sum_{k=5..7} gamma_k (hM)^k psi (gamma_k = sum_j (b_j -
// bhat_j) kappa_jk; gamma_0..4 vanish because both weights are exact to 4th
// order), and the continuous extension psi + sum_m theta^m sum_k Q_mk (hM)^k psi
// (Q_mk = sum_j W_jm kappa_jk).  A step therefore needs the Krylov vectors
// M^k psi, k <= 7 -- the same six products per step as the stage form, the first
// of them left over from the previous step -- and no stage combinations; the
// error estimate is a sum of three terms of the size of the error, with none of
// the stage form's cancellation, so FP32 forms it; and after a rejected step
// the vectors stay valid, only the coefficients change with h.  It is the same
// method with the same step sequence as the stage form, up to rounding.
//
// To keep the vectors in range whatever the size of M, the kernel holds
// wt_k = (2^-e M)^k psi with 2^e above ||M|| (a power of two, so the scaling is
// exact) and folds (h 2^e)^k into the coefficients.

// The Krylov-form coefficients in the policy's arithmetic, per CTA.
template <class Ar>
struct KCoefs {
    typename Ar::coef beta[7];  // 5th-order solution: beta_k, k = 0..6
    typename Ar::coef Q[5][8];  // continuous extension: Q[m - 1][k], theta^m, m = 1..5, k = 0..7
    float gam[3];               // error estimate: gamma_5, gamma_6, gamma_7
};

// kappa, beta, gamma and Q from the Dormand-Prince tableau (FP64; one thread per CTA)
template <class Ar>
__device__ __noinline__ void krylov_coefs(KCoefs<Ar> *K)
{
    double kap[7][8];
#pragma unroll 1
    for (int j = 0; j < 7; ++j) {
        for (int k = 0; k < 8; ++k) kap[j][k] = 0.0;
        kap[j][1] = 1.0;
        for (int k = 1; k < 7; ++k) {
            double v = 0.0;
            for (int l = 0; l < j; ++l) v += DP5::a(j, l) * kap[l][k];
            kap[j][k + 1] = v;
        }
    }
    for (int k = 0; k < 7; ++k) {
        double b = k == 0 ? 1.0 : 0.0;
        for (int j = 0; j < 7; ++j) b += DP5::b(j) * kap[j][k];
        K->beta[k] = Ar::coef_of(b);
    }
    for (int k = 5; k < 8; ++k) {
        double e = 0.0;
        for (int j = 0; j < 7; ++j) e += DP5::e(j) * kap[j][k];
        K->gam[k - 5] = (float)e;
    }
    for (int m = 1; m <= 5; ++m)
        for (int k = 0; k < 8; ++k) {
            double q = 0.0;
            for (int j = 0; j < 7; ++j) q += DP5::W(j, m) * kap[j][k];
            K->Q[m - 1][k] = Ar::coef_of(q);
        }
}

// The scalars of the current step size in shared memory, one copy per warp:
// formed by the warp's lanes in parallel (entry k by lane k mod the warp's share
// of the group) and read by them, so the step's rolled loops index them without
// local memory and only a warp-level synchronisation guards them.
template <class Ar>
struct KStep {
    typename Ar::coef hp[8];  // H^k, H = h 2^e
    typename Ar::coef c[8];   // beta_k H^k, k = 1..6 (5th-order solution and the next first stage)
    typename Ar::coef d[8];   // rho_k(theta) H^k, k = 1..7 (continuous extension at one theta)
    float ge[4];              // gamma_k H^k, k = 5..7 (error estimate)
};

// Slots of the Krylov form: psi, wt_1..wt_7, the candidate and a scratch vector.
enum KSlot { kKPsi = 0 /* wt_k in slot k, k = 1..7 */, kKYn = 8, kKScr = 9 };

// Lanes that share one KStep copy and the synchronisation among them.
template <int G>
__device__ __forceinline__ void kstep_sync(const Group<G> &g)
{
    if constexpr (G > 32)
        __syncwarp();
    else
        g.sync();
}
template <int G>
__host__ __device__ constexpr int kstep_lanes() { return G > 32 ? 32 : G; }

// KS->hp, c, ge for step size H (synchronised among the copy's lanes on return)
template <class Ar, int G>
__device__ __forceinline__ void krylov_step_coefs(const KCoefs<Ar> &KC, KStep<Ar> *KS, const Group<G> &g, double H)
{
    using coef = typename Ar::coef;
    constexpr int W = kstep_lanes<G>();
    kstep_sync(g);  // the previous step's readers are done
    const coef h1 = Ar::coef_of(H);
#pragma unroll 1
    for (int k = g.gl % W; k < 8; k += W) {
        coef p = Ar::coef_of(1.0);
#pragma unroll 1
        for (int i = 0; i < k; ++i) p = Ar::cmul(p, h1);
        KS->hp[k] = p;
        if (k >= 1 && k <= 6) KS->c[k] = Ar::cmul(KC.beta[k], p);
        if (k >= 5) KS->ge[k - 5] = KC.gam[k - 5] * Ar::coef32(p);
    }
    kstep_sync(g);
}

// KS->d for the continuous extension at theta (uses KS->hp; synchronised on return)
template <class Ar, int G>
__device__ __forceinline__ void krylov_dense_coefs(const KCoefs<Ar> &KC, KStep<Ar> *KS, const Group<G> &g, double th)
{
    using coef = typename Ar::coef;
    constexpr int W = kstep_lanes<G>();
    kstep_sync(g);
    const coef tc = Ar::coef_of(th);
#pragma unroll 1
    for (int k = 1 + g.gl % W; k < 8; k += W) {
        coef p = KC.Q[4][k];
#pragma unroll 1
        for (int m = 3; m >= 0; --m) p = Ar::cadd(Ar::cmul(p, tc), KC.Q[m][k]);
        KS->d[k] = Ar::cmul(Ar::cmul(p, tc), KS->hp[k]);
    }
    kstep_sync(g);
}

// body(r) for the lane's rows r < R: rolled for single-warp groups (a small hot
// loop), unrolled for multi-warp groups, whose threads then advance their R rows
// as independent chains
template <int G, int R, class F>
__device__ __forceinline__ void krylov_rows(F &&body)
{
    if constexpr (G > 32) {
#pragma unroll
        for (int r = 0; r < R; ++r) body(r);
    } else {
#pragma unroll 1
        for (int r = 0; r < R; ++r) body(r);
    }
}

// |e|^2 / sc^2 of one row in FP32, e = (ere, eim) formed directly
template <class Ar>
__device__ __forceinline__ float krylov_err_term(float ere, float eim, typename Ar::cplx y0, typename Ar::cplx y1,
                                                 double rtol, double atol)
{
    const float ay2 = Ar::re32(y0) * Ar::re32(y0) + Ar::im32(y0) * Ar::im32(y0);
    const float an2 = Ar::re32(y1) * Ar::re32(y1) + Ar::im32(y1) * Ar::im32(y1);
    const float sc = (float)atol + (float)rtol * sqrtf(ay2 > an2 ? ay2 : an2);
    return (ere * ere + eim * eim) / (sc * sc);
}

// dst = psi + sum_k d_k wt_k on the lane's rows (the continuous extension at the
// theta of KS->d); the caller synchronises before dst is gathered
template <class Ar, int G, int R>
__device__ __noinline__ void krylov_dense(const KStep<Ar> *KS, const Lanes<Ar, G, R> &L, typename Ar::cplx *dst)
{
    krylov_rows<G, R>([&](int r) {
        const int row = L.gl + G * r;
        if (row < L.n) {
            typename Ar::acc acc = Ar::acc_of(L.slot(kKPsi)[row]);
#pragma unroll 1
            for (int k = 1; k < 8; ++k) Ar::axpy(acc, KS->d[k], L.slot(k)[row]);
            dst[row] = Ar::get(acc);
        }
    });
}

// First theta in (0, 1] with ||y(theta)||^2 = r on the Krylov-form continuous
// extension: y(theta) = sum_m theta^m u_m, u_0 = psi, u_m = sum_k Q[m - 1][k] H^k wt_k.
template <class Ar, int G, int R>
__device__ __noinline__ double krylov_crossing(const KCoefs<Ar> &KC, const KStep<Ar> *KS, const Lanes<Ar, G, R> &L,
                                               const Group<G> &g, double r, int &iters)
{
    using cplx = typename Ar::cplx;
    typename Ar::red gram[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) gram[i] = Ar::rzero();
#pragma unroll 1
    for (int rr = 0; rr < R; ++rr) {
        const int row = L.gl + G * rr;
        if (row >= L.n) continue;
        cplx u[6];
        u[0] = L.slot(kKPsi)[row];
#pragma unroll
        for (int m = 1; m <= 5; ++m) {
            typename Ar::acc acc = Ar::zero();
#pragma unroll 1
            for (int k = 1; k < 8; ++k) Ar::axpy(acc, Ar::cmul(KC.Q[m - 1][k], KS->hp[k]), L.slot(k)[row]);
            u[m] = Ar::get(acc);
        }
        int i = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int m2 = m; m2 < 6; ++m2, ++i) gram[i] = Ar::radd(gram[i], Ar::dot_re(u[m], u[m2]));
    }
    double P[11];
#pragma unroll
    for (int s = 0; s < 11; ++s) P[s] = 0.0;
    {
        int i = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int m2 = m; m2 < 6; ++m2, ++i) {
                const double v = Ar::rval(Ar::rsum(g, gram[i]));
                P[m + m2] += (m == m2) ? v : 2.0 * v;
            }
    }
    P[0] -= r;
    return first_root(P, iters);
}

// out[row] = 2^-e (M x)[row] on the lane's rows (x synchronised)
template <class Ar, int G, int R>
__device__ __forceinline__ void krylov_product(const CsrView<Ar> &M, const typename Ar::cplx *x,
                                               typename Ar::cplx *out, int gl, int n, float down)
{
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const typename Ar::cplx v = spmv_row<Ar, G>(M, x, gl, r);
        const int row = gl + G * r;
        if (row < n) out[row] = Ar::mul_pow2(v, down);
    }
}

// The starting step (Hairer, Norsett & Wanner, Sec. II.4) from psi with
// f0 = M psi, in FP64 scalars; wt_1 = 2^-e M psi is left in slot 1 (synchronised).
template <class Ar, int G, int R>
__device__ __noinline__ double krylov_start(const KernelArgs &a, const Group<G> &g, const CsrView<Ar> &M,
                                            const Lanes<Ar, G, R> &L, double span, float down, double up)
{
    using cplx = typename Ar::cplx;
    const int n = a.n, gl = g.gl;
    const double rtol = a.rtol, atol = a.atol;
    cplx *psi = L.slot(kKPsi), *w1 = L.slot(1), *scr = L.slot(kKScr), *f1 = L.slot(kKYn);
    krylov_product<Ar, G, R>(M, psi, w1, gl, n, down);
    double d0 = 0.0, d1 = 0.0;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) {
            const double yr = Ar::re(psi[row]), yi = Ar::im(psi[row]);
            const double fr = up * Ar::re(w1[row]), fi = up * Ar::im(w1[row]);
            const double sc = atol + rtol * sqrt(yr * yr + yi * yi);
            d0 += (yr * yr + yi * yi) / (sc * sc);
            d1 += (fr * fr + fi * fi) / (sc * sc);
        }
    }
    d0 = sqrt(g.sum(d0) / n);
    d1 = sqrt(g.sum(d1) / n);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    if (h0 > span) h0 = span;
    const typename Ar::coef h0c = Ar::coef_of(h0 * up);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) {
            typename Ar::acc acc = Ar::acc_of(psi[row]);
            Ar::axpy(acc, h0c, w1[row]);
            scr[row] = Ar::get(acc);
        }
    }
    g.sync();
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const cplx v = spmv_row<Ar, G>(M, scr, gl, r);
        const int row = gl + G * r;
        if (row < n) f1[row] = v;
    }
    double d2 = 0.0;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) {
            const double yr = Ar::re(psi[row]), yi = Ar::im(psi[row]);
            const double sc = atol + rtol * sqrt(yr * yr + yi * yi);
            const double dre = Ar::re(f1[row]) - up * Ar::re(w1[row]);
            const double dim = Ar::im(f1[row]) - up * Ar::im(w1[row]);
            d2 += (dre * dre + dim * dim) / (sc * sc);
        }
    }
    d2 = sqrt(g.sum(d2) / n) / h0;
    g.sync();
    const double dm = d1 > d2 ? d1 : d2;
    const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
    double h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
    if (h > span) h = span;
    return h;
}

// Algorithm 1 for one trajectory with the Krylov form of the Dormand-Prince step
// (the plain double-float and complex64 kernels: constant M, no proposal).  The
// loops stay rolled and read their coefficients from KS, which keeps the step
// loop inside the instruction cache.
template <class Ar, int G, int R>
__device__ void run_trajectory_krylov(const KernelArgs &a, const Group<G> &g, const int *si,
                                      const typename Ar::real *sv, const KCoefs<Ar> &KC, KStep<Ar> *KS,
                                      Lanes<Ar, G, R> &L, long long il)
{
    using cplx = typename Ar::cplx;
    const int n = a.n;
    const int gl = g.gl;
    const long long traj = a.traj0 + il;
    const double t_end = a.t[a.n_t - 1];
    double *out = a.out + (size_t)il * a.n_t * a.n_obs;
    const CsrView<Ar> M = csr_view<Ar>(a.op[0], si, sv);
    const double rtol = a.rtol, atol = a.atol;
    const float down = __int_as_float((127 - a.krylov_shift) << 23);  // 2^-e
    const double up = ldexp(1.0, a.krylov_shift);                       // 2^e
    cplx *psi = L.slot(kKPsi);
    cplx *yn = L.slot(kKYn);
    cplx *scr = L.slot(kKScr);

    int status = 0;
    long long attempts = 0;
    unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0, n_jump = 0;
    int root_iters = 0;

    // (A)
    const cplx *psi0 = static_cast<const cplx *>(a.psi0);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) psi[row] = psi0[row];
    }
    g.sync();
    long long k = 0;
    double rk, ck;
    jump_draws(a.seed, traj, k, rk, ck);
    double t = a.t[0];
    record_outputs<Ar, G, R>(a, g, si, sv, psi, 0, out, nullptr);
    int j = 1;
    double h = krylov_start<Ar, G, R>(a, g, M, L, t_end - t, down, up);
    n_rhs += 2;

    static_assert(sizeof(typename Ar::errt) == sizeof(float), "the Krylov form's error norm is FP32");
    bool rejected_before = false;
    int kfrom = 2;  // wt_kfrom..wt_7 still to be formed for the current psi (8: none)
    // scalar control with as little FP64 as the method allows: the next output
    // time in a register, the end test against a precomputed threshold
    double t_next = a.t[j < a.n_t ? j : a.n_t - 1];
    const double t_stop = t_end - 4.0 * 2.220446049250313e-16 * fabs(t_end);
    while (j < a.n_t) {
        if (t >= t_stop) {
            g.sync();
            for (; j < a.n_t; ++j) record_outputs<Ar, G, R>(a, g, si, sv, psi, j, out, nullptr);
            break;
        }
        if (attempts >= a.max_steps) {
            status = 4;
            break;
        }
        bool last = false;
        if (t + 1.01 * h >= t_end) {
            h = t_end - t;
            last = true;
        }
        if (h < 1e-14 * fmax(1.0, fabs(t))) {
            status = 5;
            break;
        }
        // (B): the Krylov vectors of psi; after a rejection they are still valid
#pragma unroll 1
        for (int q = kfrom; q < 8; ++q) {
            g.sync();  // wt_{q-1} complete in every lane
            krylov_product<Ar, G, R>(M, L.slot(q - 1), L.slot(q), gl, n, down);
        }
        n_rhs += 8 - kfrom;
        kfrom = 8;
        ++attempts;
        krylov_step_coefs<Ar, G>(KC, KS, g, h * up);

        typename Ar::errt esum = 0;
        float nr32 = 0.f;  // ||ynew||^2 from the leading FP32 parts (the crossing pre-test)
        krylov_rows<G, R>([&](int r) {
            const int row = gl + G * r;
            if (row < n) {
                const cplx y0 = psi[row];
                typename Ar::acc acc = Ar::acc_of(y0);
#pragma unroll 1
                for (int q = 1; q < 7; ++q) Ar::axpy(acc, KS->c[q], L.slot(q)[row]);
                const cplx y1 = Ar::get(acc);
                yn[row] = y1;
                const cplx w5 = L.slot(5)[row], w6 = L.slot(6)[row], w7 = L.slot(7)[row];
                const float ere = fmaf(KS->ge[0], Ar::re32(w5),
                                       fmaf(KS->ge[1], Ar::re32(w6), KS->ge[2] * Ar::re32(w7)));
                const float eim = fmaf(KS->ge[0], Ar::im32(w5),
                                       fmaf(KS->ge[1], Ar::im32(w6), KS->ge[2] * Ar::im32(w7)));
                esum += krylov_err_term<Ar>(ere, eim, y0, y1, rtol, atol);
                nr32 = fmaf(Ar::re32(y1), Ar::re32(y1), fmaf(Ar::im32(y1), Ar::im32(y1), nr32));
            }
        });
        // error norm, acceptance and controller in FP32 (the double-float policy's choice)
        const float err = sqrtf(Ar::err_sum(g, esum) / (float)n);

        if (!(err <= 1.f)) {
            if (!isfinite(err)) {
                status = 6;
                break;
            }
            float fac = 0.9f * __powf(err, -0.2f);
            if (fac < (float)kFacMin) fac = (float)kFacMin;
            h *= (double)fac;
            rejected_before = true;
            ++n_rej;
            continue;
        }
        ++n_acc;
        const double t_new = last ? t_end : t + h;
        // (B) crossing test ||ynew||^2 < r: decided from the FP32 sum when it lies
        // outside r (1 +- 1e-4) -- its relative error is below 1e-6 (leading parts
        // good to 2^-24, a dozen FP32 roundings of positive terms) -- else from the
        // double-float norm, so the decision is the one the exact norm gives
        const float s32 = g.sum(nr32), rkf = (float)rk;
        bool crossed = s32 < 0.9999f * rkf;
        if (!crossed && !(s32 > 1.0001f * rkf)) {
            typename Ar::red nr = Ar::rzero();
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) nr = Ar::radd(nr, Ar::abs2(yn[row]));
            }
            crossed = Ar::rval(Ar::rsum(g, nr)) < rk;
        }

        if (crossed) {
            // (C): the norm reached r inside this step
            const double th = krylov_crossing<Ar, G, R>(KC, KS, L, g, rk, root_iters);
            double tau = t + th * h;
            if (tau > t_new) tau = t_new;
            const double inv_h = 1.0 / h;
            for (; j < a.n_t && t_next <= tau; t_next = a.t[++j < a.n_t ? j : a.n_t - 1]) {
                double thj = (t_next - t) * inv_h;
                if (thj > 1.0) thj = 1.0;
                krylov_dense_coefs<Ar, G>(KC, KS, g, thj);
                krylov_dense<Ar, G, R>(KS, L, scr);
                g.sync();
                record_outputs<Ar, G, R>(a, g, si, sv, scr, j, out, nullptr);
            }
            krylov_dense_coefs<Ar, G>(KC, KS, g, th);
            krylov_dense<Ar, G, R>(KS, L, scr);
            g.sync();
            // the candidate is dead after a crossing: its slot serves as scratch
            const int ch = apply_jump<Ar, G, R>(a, g, si, sv, psi, yn, scr, ck);
            if (ch < 0) {
                status = 7;
                break;
            }
            if (gl == 0 && (long long)n_jump < a.max_jumps) {
                a.jump_t[(size_t)il * a.max_jumps + n_jump] = tau;
                a.jump_ch[(size_t)il * a.max_jumps + n_jump] = ch;
            }
            ++n_jump;
            // (D): the Krylov vectors of the new psi, from wt_1, at the next attempt
            ++k;
            jump_draws(a.seed, traj, k, rk, ck);
            t = tau;
            kfrom = 1;
            rejected_before = false;
            continue;
        }

        if (t_next <= t_new) {
            const double inv_h = 1.0 / h;
            for (; j < a.n_t && t_next <= t_new; t_next = a.t[++j < a.n_t ? j : a.n_t - 1]) {
                double thj = (t_next - t) * inv_h;
                if (thj > 1.0) thj = 1.0;
                krylov_dense_coefs<Ar, G>(KC, KS, g, thj);
                krylov_dense<Ar, G, R>(KS, L, scr);
                g.sync();
                record_outputs<Ar, G, R>(a, g, si, sv, scr, j, out, nullptr);
            }
        }
        float fac = (err == 0.f) ? (float)kFacMax : 0.9f * __powf(err, -0.2f);
        if (fac > (float)kFacMax) fac = (float)kFacMax;
        if (fac < (float)kFacMin) fac = (float)kFacMin;
        if (rejected_before && fac > 1.f) fac = 1.f;
        rejected_before = false;
        t = t_new;
        // first same as last: wt_1 <- 2^-e M ynew = wt_1 + sum_{k=1..6} c_k wt_{k+1}; psi <- ynew
        krylov_rows<G, R>([&](int r) {
            const int row = gl + G * r;
            if (row < n) {
                typename Ar::acc acc = Ar::acc_of(L.slot(1)[row]);
#pragma unroll 1
                for (int q = 1; q < 7; ++q) Ar::axpy(acc, KS->c[q], L.slot(q + 1)[row]);
                L.slot(1)[row] = Ar::get(acc);
                psi[row] = yn[row];
            }
        });
        kfrom = 2;
        h *= (double)fac;
    }

    if (gl == 0) {
        if (status != 0) {
            for (; j < a.n_t; ++j)
                for (int q = 0; q < a.n_obs; ++q)
                    out[(size_t)j * a.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
            atomicCAS(a.first_error, 0, status);
            atomicAdd(&a.counters[kFailed], 1ULL);
        }
        if (a.max_jumps > 0) a.n_jumps[il] = (int)n_jump;
        atomicAdd(&a.counters[kAccepted], n_acc);
        atomicAdd(&a.counters[kRejected], n_rej);
        atomicAdd(&a.counters[kRhs], n_rhs);
        atomicAdd(&a.counters[kJumps], n_jump);
        atomicAdd(&a.counters[kRootIters], (unsigned long long)root_iters);
    }
}

// Threads per CTA for a group size: 4 warps for single-warp groups, 8 warps (one
// to four groups) for multi-warp groups.
template <int G>
__host__ __device__ constexpr int block_for_group() { return G <= 32 ? 128 : 256; }

// The step form of an instantiation: the Krylov form (constant operator) for the
// plain double-float kernels; the stage form for complex128 (the plain FP64 path,
// written as the oracle writes it), for every kernel with a time-dependent term
// or the learned proposal, and for complex64.  The Krylov form carries wt_1 from
// step to step by a combination, whose rounding error is never reset by a
// product: at double-float precision that drift stays far below the parity bars,
// with an FP32 state it doubled the complex64 path's ensemble error (measured
// 1.4e-4 -> 2.8e-4 on the JC benchmark).
template <class Ar, int FEAT>
__host__ __device__ constexpr bool use_krylov() { return FEAT == 0 && Ar::kId == ArDF::kId; }

// CTA size and the CTAs per SM the register budget is set for.  The single-warp
// Krylov kernels run ten warps per CTA and two CTAs per SM where the ten slots
// of that many groups stay near 100 KB (R x complex size <= 32 bytes): one
// operator copy per ten warps instead of per four leaves room for 20 resident
// warps (at most 102 registers) instead of 16, which hides more of the step's
// latency.
template <class Ar, int G, int R, int FEAT>
__host__ __device__ constexpr int trajectory_block()
{
    return (G <= 32 && use_krylov<Ar, FEAT>() && R * sizeof(typename Ar::cplx) <= 32) ? 10 * 32
                                                                                     : block_for_group<G>();
}
template <int G, int BLOCK>
__host__ __device__ constexpr int trajectory_min_ctas() { return G > 32 ? 1 : (BLOCK > 128 ? 2 : 4); }

// Operators are staged into shared memory for single-warp groups (small N); the
// operators of multi-warp groups (N > 64) are read from global memory, where
// they stay resident in L2 and the L1 read-only path.
template <int G>
__host__ __device__ constexpr bool ops_in_shared() { return G <= 32; }

template <class Ar, int G, int R, int BLOCK, int FEAT>
__global__ void __launch_bounds__(BLOCK, (trajectory_min_ctas<G, BLOCK>())) mcwf_kernel(const __grid_constant__ KernelArgs a)
{
    using cplx = typename Ar::cplx;
    using real = typename Ar::real;
    extern __shared__ __align__(16) unsigned char smem[];
    const int *si;
    const real *sv;
    if constexpr (ops_in_shared<G>()) {
        int *ints = reinterpret_cast<int *>(smem);
        real *vals = reinterpret_cast<real *>(smem + a.smem_vals_offset);
        for (int i = threadIdx.x; i < a.n_ints; i += BLOCK) ints[i] = a.ints[i];
        const real *gv = static_cast<const real *>(a.vals);
        for (int i = threadIdx.x; i < a.n_vals; i += BLOCK) vals[i] = gv[i];
        si = ints;
        sv = vals;
    } else {
        si = a.ints;
        sv = static_cast<const real *>(a.vals);
    }
    // the plain double-float and complex64 kernels take the Krylov form of the step
    constexpr bool KRYLOV = use_krylov<Ar, FEAT>();
    Coefs<Ar> *C = reinterpret_cast<Coefs<Ar> *>(smem + a.smem_coef_offset);
    KCoefs<Ar> *KC = reinterpret_cast<KCoefs<Ar> *>(smem + a.smem_coef_offset);
    if constexpr (KRYLOV) {
        if (threadIdx.x == 0) krylov_coefs<Ar>(KC);
    } else {
        for (int i = threadIdx.x; i < 42 + 7 + 35; i += BLOCK) {
            if (i < 42)
                C->a[i / 6][i % 6] = Ar::coef_of(DP5::a(i / 6, i % 6));
            else if (i < 49)
                C->e[i - 42] = Ar::coef_of(DP5::e(i - 42));
            else
                C->W[(i - 49) / 5][(i - 49) % 5] = Ar::coef_of(DP5::W((i - 49) / 5, (i - 49) % 5 + 1));
        }
    }
    __syncthreads();

    const Group<G> g(threadIdx.x, reinterpret_cast<unsigned long long *>(smem + a.smem_scratch_offset));
    Lanes<Ar, G, R> L{reinterpret_cast<cplx *>(smem + a.smem_ybuf_offset) + (threadIdx.x / G) * kNumSlots * (G * R),
                      g.gl, a.n, 0};
    unsigned char *pbase = smem + a.smem_mlp_offset + (size_t)(threadIdx.x / G) * kPropStride;
    constexpr bool PROP = (FEAT & kFeatProposal) != 0;
    float *hscratch = PROP ? reinterpret_cast<float *>(pbase) : nullptr;
    KStep<Ar> *KS = reinterpret_cast<KStep<Ar> *>(smem + a.smem_mlp_offset) + threadIdx.x / kstep_lanes<G>();
    PropState *P = PROP ? reinterpret_cast<PropState *>(pbase + kMlpHidden * sizeof(float)) : nullptr;
    for (;;) {
        unsigned long long i = 0;
        if (g.gl == 0) i = atomicAdd(a.queue, 1ULL);
        i = g.bcast0(i);
        if ((long long)i >= a.ntraj) break;
        if constexpr (KRYLOV)
            run_trajectory_krylov<Ar, G, R>(a, g, si, sv, *KC, KS, L, (long long)i);
        else
            run_trajectory<Ar, G, R, FEAT>(a, g, si, sv, *C, L, hscratch, P, (long long)i);
    }
}

// Shared-memory layout and occupancy-sized persistent launch of one instantiation.
template <class Ar, int G, int R, int FEAT = 0>
cudaError_t launch_instance(const KernelArgs &a0, cudaStream_t stream, LaunchInfo *info)
{
    using cplx = typename Ar::cplx;
    constexpr int BLOCK = trajectory_block<Ar, G, R, FEAT>();
    constexpr int GROUPS = BLOCK / G;
    KernelArgs a = a0;
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t ib = ops_in_shared<G>() ? al16((size_t)a.n_ints * sizeof(int)) : 0;
    const size_t vb = ops_in_shared<G>() ? al16((size_t)a.n_vals * sizeof(typename Ar::real)) : 0;
    const size_t cb = al16(sizeof(Coefs<Ar>) > sizeof(KCoefs<Ar>) ? sizeof(Coefs<Ar>) : sizeof(KCoefs<Ar>));
    const size_t sb = al16((size_t)GROUPS * (Group<G>::kWarps + 1) * 8);
    const size_t mb = (FEAT & kFeatProposal) ? (size_t)GROUPS * kPropStride
                      : use_krylov<Ar, FEAT>() ? al16((size_t)(BLOCK / kstep_lanes<G>()) * sizeof(KStep<Ar>)) : 0;
    a.smem_vals_offset = (int)ib;
    a.smem_coef_offset = (int)(ib + vb);
    a.smem_scratch_offset = (int)(ib + vb + cb);
    a.smem_mlp_offset = (int)(ib + vb + cb + sb);
    a.smem_ybuf_offset = (int)(ib + vb + cb + sb + mb);
    const size_t smem = ib + vb + cb + sb + mb + (size_t)GROUPS * kNumSlots * G * R * sizeof(cplx);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = mcwf_kernel<Ar, G, R, BLOCK, FEAT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the trajectory state lives in shared memory: ask for the largest carveout
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem)) != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    const long long need = (a.ntraj + GROUPS - 1) / GROUPS;
    long long grid = (long long)nb * sms;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, BLOCK, smem, stream>>>(a);
    if (info) {
        info->group = G;
        info->rows = R;
        info->grid = (int)grid;
        info->block = BLOCK;
        info->smem = smem;
    }
    return cudaGetLastError();
}

// The instantiation for the layout the operators were packed with (a.G, a.R):
// single-warp groups here, multi-warp groups in launch_large.  The layouts are
// those of layout_candidates.
template <class Ar, int FEAT = 0>
cudaError_t launch_small(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    if (a.G == 1 && a.R == 2) return launch_instance<Ar, 1, 2, FEAT>(a, stream, info);
    if (a.G == 4 && a.R == 2) return launch_instance<Ar, 4, 2, FEAT>(a, stream, info);
    if (a.G == 4 && a.R == 4) return launch_instance<Ar, 4, 4, FEAT>(a, stream, info);
    if (a.G == 8 && a.R == 2) return launch_instance<Ar, 8, 2, FEAT>(a, stream, info);
    if (a.G == 8 && a.R == 4) return launch_instance<Ar, 8, 4, FEAT>(a, stream, info);
    if (a.G == 16 && a.R == 2) return launch_instance<Ar, 16, 2, FEAT>(a, stream, info);
    if (a.G == 16 && a.R == 4) return launch_instance<Ar, 16, 4, FEAT>(a, stream, info);
    if (a.G == 32 && a.R == 2) return launch_instance<Ar, 32, 2, FEAT>(a, stream, info);
    if (a.G == 32 && a.R == 4) return launch_instance<Ar, 32, 4, FEAT>(a, stream, info);
    return cudaErrorInvalidValue;
}

template <class Ar, int FEAT = 0>
cudaError_t launch_large(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    if (a.G == 64 && a.R == 2) return launch_instance<Ar, 64, 2, FEAT>(a, stream, info);
    if (a.G == 64 && a.R == 4) return launch_instance<Ar, 64, 4, FEAT>(a, stream, info);
    if (a.G == 128 && a.R == 2) return launch_instance<Ar, 128, 2, FEAT>(a, stream, info);
    if (a.G == 128 && a.R == 4) return launch_instance<Ar, 128, 4, FEAT>(a, stream, info);
    if (a.G == 256 && a.R == 2) return launch_instance<Ar, 256, 2, FEAT>(a, stream, info);
    if (a.G == 256 && a.R == 4) return launch_instance<Ar, 256, 4, FEAT>(a, stream, info);
    return cudaErrorInvalidValue;
}

}  // namespace qtm
