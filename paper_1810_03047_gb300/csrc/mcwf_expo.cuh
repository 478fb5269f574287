// mcwf_expo.cuh -- Algorithm 1 (Sec. 2.2) with the no-jump evolution applied
// exactly: between two jumps d psi/dt = M psi with a constant M = -i H_eff, so
// psi(t) = exp(M (t - t_k)) psi_k.  This is the library's method for stiff
// problems (Sec. 2.1: the paper switches ZVODE to BDF there), where an explicit
// integrator's step is set by the largest decay rate rather than by accuracy.
//
// The host precomputes a ladder of propagators P_l = exp(M delta 2^l),
// l = 0..L, with delta chosen so that nu delta <= 1/16 (nu >= ||M||_2) and
// delta 2^L = the output spacing.  A group of G lanes (R rows per lane, vectors
// in shared memory as in mcwf_kernel.cuh) carries T trajectories in lock step
// from output to output (T = 1 in every instantiation, see expo_batch; the code
// is written for general T):
//   * between outputs: psi_t(t_j) = P_L psi_t(t_{j-1}) for the group's
//     trajectories in one pass over P_L on a uniform grid; otherwise, per
//     trajectory, the duration d is split into its binary digits in
//     units of delta (one product per digit) and a remainder s < delta, which
//     takes a degree-9 Taylor polynomial of exp(s M) (9 products with M; the
//     truncation error is below 3e-19 relative);
//   * (B) d||psi||^2/dt = -sum_n ||C_n psi||^2 <= 0, so the norm cannot rise: if
//     ||psi(t_j)||^2 >= r no jump happened before t_j.  Otherwise the crossing is
//     found by a binary descent over the ladder from psi(t_{j-1}): level l is
//     applied when the norm after it is still >= r, which brackets the crossing
//     within one delta; there, ||psi(s)||^2 with psi(s) = sum_m s^m u_m
//     (u_m = M^m psi / m!) is solved for r by Newton's method with a bisection
//     safeguard;
//   * (C), (D) as in the Dormand-Prince kernel (apply_jump, new draws), and the
//     propagation restarts at tau and continues to t_j; a trajectory's crossings
//     are handled one trajectory at a time with the group's shared scratch
//     vectors, so after each output step every trajectory of the group is at t_j.
// No step-size control and no interpolation are involved: a trajectory differs
// from the exact one by rounding and by the root tolerance only, whatever the
// stiffness of M.
#pragma once

#include "mcwf_kernel.cuh"

namespace qtm {

constexpr int kExpoTaylor = 9;  // largest degree of the Taylor polynomial of exp(s M), s <= delta

// The degree used by an arithmetic.  The ladder's delta keeps ||s M|| <= 1/16, so
// the truncation is below (1/16)^(K+1) / (K+1)!: 2.4e-19 at K = 9 for the
// FP64-class arithmetics, 8.3e-11 at K = 5 -- far below FP32 rounding -- for
// complex64, whose crossing search and remainders thus take four products
// fewer each.
template <class Ar>
__host__ __device__ constexpr int expo_degree() { return Ar::kId == ArF32::kId ? 5 : kExpoTaylor; }

// Vector slots of a group of T trajectories: psi_t and the batched product y_t
// per trajectory, then the shared scratch (two product buffers and the Taylor
// vectors u_1..u_9, used by one trajectory at a time; u_1 doubles as the jump's
// scratch, since it is dead once the jump time is known).
template <int T>
struct ExpoSlots {
    static constexpr int kPsi = 0, kY = T, kA = 2 * T, kB = 2 * T + 1, kU = 2 * T + 2;
    static constexpr int kCount = kU + kExpoTaylor;
};
// apply_jump's dense path keeps every channel's product in u_1, u_2, ...
static_assert(kJumpKeep <= kExpoTaylor, "the kept channel products fit the Taylor slots");

// out_t = P x_t for t < T (x_t = x + t NP, out_t = out + t NP) on the lane's rows;
// P is column-major with NP = G R rows per column (zero below n), so every
// column is loaded once for the T products.  nn[t] = the lane's part of
// ||out_t||^2.  The x_t are synchronised.
template <class Ar, int G, int R, int T, int U = 0>
__device__ __forceinline__ void level_apply(const typename Ar::cplx *__restrict__ P, const typename Ar::cplx *x,
                                            typename Ar::cplx *out, int gl, int n, typename Ar::red (&nn)[T])
{
    constexpr int NP = G * R;
    typename Ar::acc acc[T][R];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[t][r] = Ar::zero();
    const typename Ar::cplx *col = P + gl;
    // columns in flight: four; two where the accumulators already fill the
    // registers (double-float, batches); eight for complex64 on multi-warp
    // groups, whose large P_L streams from L2 (dense N = 256: +6 %; on the
    // single-warp layouts eight measured 3-4 % slower)
    constexpr int kUnroll = U > 0 ? U : (T > 1 || Ar::kId == ArDF::kId) ? 2 : (Ar::kId == ArF32::kId && G >= 64 ? 8 : 4);
#pragma unroll(kUnroll)
    for (int c = 0; c < n; ++c) {
        typename Ar::cplx p[R];
#pragma unroll
        for (int r = 0; r < R; ++r) p[r] = col[G * r];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const typename Ar::cplx xc = x[t * NP + c];
#pragma unroll
            for (int r = 0; r < R; ++r) Ar::mac(acc[t][r], p[r], xc);
        }
        col += NP;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        nn[t] = Ar::rzero();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                const typename Ar::cplx v = Ar::get(acc[t][r]);
                out[t * NP + row] = v;
                nn[t] = Ar::radd(nn[t], Ar::abs2(v));
            }
        }
    }
}

// One trajectory's propagation and crossing search with the group's shared
// scratch vectors A, B and U (u_m at U + (m - 1) NP).
template <class Ar, int G, int R, bool DENSE = false>
struct Expo {
    using cplx = typename Ar::cplx;
    static constexpr int K = expo_degree<Ar>();
    static constexpr int NP = G * R;
    const KernelArgs &a;
    const Group<G> &g;
    CsrView<Ar> M;
    cplx *A, *B, *U;
    const typename Ar::coef *inv;  // inv[m] = 1/m in the coefficient type (shared memory)
    unsigned long long n_rhs = 0, n_rej = 0, n_miss = 0;
    int root_iters = 0;

    __device__ const cplx *level(int l) const
    {
        return static_cast<const cplx *>(a.expo) + (size_t)l * a.n * NP;
    }
    __device__ cplx *u(int m) const { return U + (m - 1) * NP; }

    // lane-summed ||y||^2 (y written by this lane on its rows)
    __device__ double norm2(const cplx *y) const
    {
        typename Ar::red nn = Ar::rzero();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = g.gl + G * r;
            if (row < a.n) nn = Ar::radd(nn, Ar::abs2(y[row]));
        }
        return Ar::rval(Ar::rsum(g, nn));
    }

    // dst = x + s (M src) (x given) or s (M src) on the lane's rows, no
    // synchronisation: the M product of the Taylor remainder and of the
    // crossing's u_m (out of line for double-float, like level_part)
    __device__ __forceinline__ void m_times(const cplx *src, cplx *dst, typename Ar::coef s, const cplx *x) const
    {
        if constexpr (Ar::kId == ArDF::kId)
            m_times_ool(src, dst, s, x);
        else
            m_times_inl(src, dst, s, x);
    }
    __device__ __noinline__ void m_times_ool(const cplx *src, cplx *dst, typename Ar::coef s, const cplx *x) const
    {
        m_times_inl(src, dst, s, x);
    }
    __device__ __forceinline__ void m_times_inl(const cplx *src, cplx *dst, typename Ar::coef s, const cplx *x) const
    {
        if constexpr (DENSE) {  // the dense FP32 copy of M, when it has one
            if (a.dense_off[0] >= 0) {
                cpx<float> v[R];
                dense_rows_f32<G, R>(a.dense + a.dense_off[0], a.dense_ld, src, g.gl, a.n, v);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int row = g.gl + G * r;
                    if (row < a.n) {
                        typename Ar::acc acc = Ar::zero();
                        Ar::axpy(acc, s, v[r]);
                        dst[row] = x ? Ar::add_scaled(x[row], Ar::coef_of(1.0), acc) : Ar::get(acc);
                    }
                }
                return;
            }
        }
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            const cplx mv = spmv_row<Ar, G>(M, src, g.gl, r);
            const int row = g.gl + G * r;
            if (row < a.n) {
                typename Ar::acc acc = Ar::zero();
                Ar::axpy(acc, s, mv);
                dst[row] = x ? Ar::add_scaled(x[row], Ar::coef_of(1.0), acc) : Ar::get(acc);
            }
        }
    }

    // out = P_l x on the lane's rows; returns the lane's part of ||out||^2 (no
    // synchronisation).  Double-float: out of line, so every propagation,
    // descent and bracket check runs one copy of the product loop, which keeps
    // the kernel's hot code inside the instruction cache (inlined at each call
    // site, the long double-float copies evicted one another: instruction-fetch
    // stalls were the largest stall; +23 % on Jaynes-Cummings).  The shorter
    // FP32 and FP64 loops stay inline (out of line measured 3-12 % slower in
    // complex64).
    __device__ __forceinline__ typename Ar::red level_part_inl(int l, const cplx *x, cplx *out) const
    {
        typename Ar::red p[1];
        // the lock-step kernel keeps sixteen columns in flight (its catch-ups are
        // bound by the loads in flight: +4.5 % over eight)
        level_apply<Ar, G, R, 1, DENSE ? 16 : 0>(level(l), x, out, g.gl, a.n, p);
        return p[0];
    }
    __device__ __noinline__ typename Ar::red level_part_ool(int l, const cplx *x, cplx *out) const
    {
        return level_part_inl(l, x, out);
    }
    __device__ __forceinline__ typename Ar::red level_part(int l, const cplx *x, cplx *out) const
    {
        if constexpr (Ar::kId == ArDF::kId)
            return level_part_ool(l, x, out);
        else
            return level_part_inl(l, x, out);
    }

    // out = P_l x, synchronised; returns ||out||^2
    __device__ double apply_level(int l, const cplx *x, cplx *out)
    {
        const double nn = Ar::rval(Ar::rsum(g, level_part(l, x, out)));
        g.sync();
        ++n_rhs;
        return nn;
    }

    // exp(s M) x for 0 < s <= delta by Horner's rule, v <- x + (s/m) M v for
    // m = 9..1, alternating between w0 and w1; returns the buffer with the result
    __device__ cplx *taylor(const cplx *x, cplx *w0, cplx *w1, double s)
    {
        const cplx *src = x;
        cplx *dst = w0;
        const typename Ar::coef sc = Ar::coef_of(s);
#pragma unroll 1
        for (int m = K; m >= 1; --m) {
            m_times(src, dst, Ar::cmul(sc, inv[m]), x);
            g.sync();
            ++n_rhs;
            src = dst;
            dst = (dst == w0) ? w1 : w0;
        }
        return const_cast<cplx *>(src);
    }

    // exp(d M) psi: the binary digits of d / delta on the ladder, then the
    // remainder by Taylor.  Returns the buffer holding the result (A, B, u_1 or
    // u_2; never psi).
    __device__ cplx *propagate(double d, const cplx *psi)
    {
        const int L = a.expo_levels - 1;
        const double delta = a.expo_delta;
        double qd = floor(d / delta);
        const double qmax = ldexp(1.0, L + 1) - 1.0;
        if (!(qd >= 0.0)) qd = 0.0;
        if (qd > qmax) qd = qmax;
        double rem = fma(-qd, delta, d);
        if (rem < 0.0) {
            if (qd > 0.0) {
                qd -= 1.0;
                rem += delta;
            } else {
                rem = 0.0;
            }
        }
        const unsigned long long q = (unsigned long long)qd;
        const cplx *cur = psi;
#pragma unroll 1
        for (int l = L; l >= 0; --l)
            if ((q >> l) & 1ULL) {
                cplx *out = (cur == A) ? B : A;
                apply_level(l, cur, out);
                cur = out;
            }
        if (rem > 0.0) return taylor(cur, u(1), u(2), rem);
        if (cur == psi) {  // d == 0: a copy
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = g.gl + G * r;
                if (row < a.n) A[row] = psi[row];
            }
            g.sync();
            return A;
        }
        return const_cast<cplx *>(cur);
    }

    // The bracket [m delta, (m + 1) delta) holding the predicted crossing time
    // s_hat, formed from the binary digits of m (the levels the descent would keep,
    // in its order) and checked with one more product.  True on a hit (base, cur,
    // nb describe the bracket's start); otherwise base, cur, nb are where the
    // descent has to continue from (psi and 0 when the crossing lies earlier).
    // Out of line: the crossing search is rare and its registers stay out of the
    // propagation loop.
    __device__ __noinline__ bool predicted_bracket(double d, const cplx *psi, double r, double s_hat, const cplx *&base,
                                                   double &cur, double &nb)
    {
        const int L = a.expo_levels - 1;
        const double delta = a.expo_delta;
        const double mmax = ceil(d / delta) - 1.0;
        double md = floor(s_hat / delta);
        if (md > mmax) md = mmax;
        if (md < 0.0) md = 0.0;
        const unsigned long long m = (unsigned long long)md;
        double nm = nb;
        base = psi;
#pragma unroll 1
        for (int l = L; l >= 0; --l)
            if ((m >> l) & 1ULL) {
                cplx *o = (base == A) ? B : A;
                nm = apply_level(l, base, o);
                base = o;
            }
        if (!(nm >= r)) {  // the crossing lies earlier: descend from psi
            base = psi;
            cur = 0.0;
            ++n_miss;
            return false;
        }
        cur = md * delta;
        nb = nm;
        if (cur + delta >= d) return true;  // the interval ends inside the last delta
        cplx *o = (base == A) ? B : A;
        const double n1 = apply_level(0, base, o);
        if (n1 < r) {
            ++n_rej;
            return true;
        }
        base = o;  // the crossing lies later: descend from the end of this delta
        cur += delta;
        nb = n1;
        ++n_miss;
        return false;
    }

    // (B) with ||psi||^2 = nb >= r now and ||exp(d M) psi||^2 < r: the time s in
    // (0, d] of the crossing; psi(s) is left in *out (A or B, synchronised).
    // s_hat >= 0 is a predicted crossing time (the learned proposal): the bracket
    // [m delta, (m + 1) delta) holding it is formed directly from the binary digits
    // of m -- the same products, in the same order, as the levels the descent keeps
    // for that bracket -- and checked with one more product; on a miss the descent
    // takes over.  The crossing itself is found as without a prediction.
    __device__ double crossing(double d, const cplx *psi, double nb, double r, double t0, cplx **out,
                              double s_hat = -1.0)
    {
        const int L = a.expo_levels - 1;
        const double delta = a.expo_delta;
        const cplx *base = psi;
        double cur = 0.0;
        const bool bracketed = s_hat >= 0.0 && predicted_bracket(d, psi, r, s_hat, base, cur, nb);
        // binary descent: keep level l when the norm after it is still >= r (a
        // level ending at d would not be kept: the norm there is below r)
        if (!bracketed) {
#pragma unroll 1
            for (int l = L; l >= 0; --l) {
                const double step = ldexp(delta, l);
                if (cur + step >= d) continue;
                cplx *o = (base == A) ? B : A;
                const double nn = apply_level(l, base, o);
                if (nn >= r) {
                    base = o;
                    cur += step;
                    nb = nn;
                } else {
                    ++n_rej;
                }
            }
        }
        double smax = d - cur;
        if (smax > delta) smax = delta;
        if (smax < 0.0) smax = 0.0;
        // u_m = M u_{m-1} / m, u_0 = base
        const cplx *prev = base;
#pragma unroll 1
        for (int m = 1; m <= K; ++m) {
            cplx *um = u(m);
            m_times(prev, um, inv[m], nullptr);
            g.sync();
            ++n_rhs;
            prev = um;
        }
        // f(s) = ||sum_m s^m u_m||^2 - r and f'(s) = 2 Re<psi(s), psi'(s)>; the
        // powers are formed once per evaluation in the arithmetic's coefficient
        // type (FP32 pairs or floats on the FP32 pipe, doubles for complex128)
        auto eval = [&](double s, double &fp) {
            typename Ar::coef pw[K + 1], dpw[K + 1];
            const typename Ar::coef sc = Ar::coef_of(s);
            pw[0] = Ar::coef_of(1.0);
#pragma unroll
            for (int m = 1; m <= K; ++m) {
                dpw[m] = Ar::cmul(Ar::cconst((double)m), pw[m - 1]);
                pw[m] = Ar::cmul(pw[m - 1], sc);
            }
            typename Ar::red nn = Ar::rzero(), dd = Ar::rzero();
#pragma unroll 1
            for (int r2 = 0; r2 < R; ++r2) {
                const int row = g.gl + G * r2;
                if (row < a.n) {
                    typename Ar::acc y = Ar::zero(), yp = Ar::zero();
#pragma unroll
                    for (int m = 1; m <= K; ++m) {
                        const cplx um = u(m)[row];
                        Ar::axpy(yp, dpw[m], um);
                        Ar::axpy(y, pw[m], um);
                    }
                    const cplx yv = Ar::add_scaled(base[row], Ar::coef_of(1.0), y);
                    const cplx ypv = Ar::get(yp);
                    nn = Ar::radd(nn, Ar::abs2(yv));
                    dd = Ar::radd(dd, Ar::dot_re(yv, ypv));
                }
            }
            fp = 2.0 * Ar::rval(Ar::rsum(g, dd));
            return Ar::rval(Ar::rsum(g, nn)) - r;
        };
        double fp = 0.0;
        const double flo = nb - r, fhi = eval(smax, fp);
        double s = smax;
        if (fhi < 0.0 && flo > 0.0) {
            double lo = 0.0, hi = smax;
            s = smax * flo / (flo - fhi);
            const double tol = 1e-15 * fmax(1.0, fabs(t0 + cur));
#pragma unroll 1
            for (int it = 0; it < 60; ++it) {
                ++root_iters;
                const double f = eval(s, fp);
                if (f == 0.0) break;
                if (f > 0.0)
                    lo = s;
                else
                    hi = s;
                double sn = s - f / fp;
                if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
                if (fabs(sn - s) <= tol || hi - lo <= tol) {
                    s = sn;
                    break;
                }
                s = sn;
            }
        } else if (!(flo > 0.0)) {
            s = 0.0;  // the norm was already at r (rounding)
        }
        // psi(s) into the product buffer that does not hold the base
        cplx *o = (base == A) ? B : A;
        typename Ar::coef pw[K + 1];
        {
            const typename Ar::coef sc = Ar::coef_of(s);
            pw[0] = Ar::coef_of(1.0);
#pragma unroll
            for (int m = 1; m <= K; ++m) pw[m] = Ar::cmul(pw[m - 1], sc);
        }
#pragma unroll 1
        for (int r2 = 0; r2 < R; ++r2) {
            const int row = g.gl + G * r2;
            if (row < a.n) {
                typename Ar::acc y = Ar::zero();
#pragma unroll
                for (int m = 1; m <= K; ++m) Ar::axpy(y, pw[m], u(m)[row]);
                o[row] = Ar::add_scaled(base[row], Ar::coef_of(1.0), y);
            }
        }
        g.sync();
        *out = o;
        return cur + s;
    }
};

// The learned proposal in the exponential method (instantiations with
// kFeatProposal; single-warp groups, one trajectory per group).  When an output
// interval (t_{j-1}, t_j] is found to contain the crossing, the features are the
// decay rate over that interval from the norms at its ends, Gamma = log(nb/nn)/d,
// its change since the previous interval's rate (per unit time), the norm nb at
// t_{j-1}, log r, and the latest outputs of the first two observables; the network
// corrects the constant-rate estimate log(nb/r)/Gamma of the time to the crossing
// (the same parametrisation as the Dormand-Prince proposal), and the prediction
// selects the bracket the crossing search tries first.  In collection mode
// (rec_stride > 0) every rec_stride-th crossing stores its features and, once the
// crossing is found, its time from t_{j-1}.
struct ExpoProp {
    float h[kMlpHidden];  // the network's hidden-layer scratch
    float f[kMlpIn];      // features of the current crossing
    float gam_prev;       // decay rate of the last jump-free interval (< 0: none yet)
    int rec_n;            // records stored for this trajectory
};
constexpr int kExpoPropStride = (int)((sizeof(ExpoProp) + 15) & ~size_t(15));

// The proposal's work at a crossing, out of line so that it adds no register
// pressure to the propagation loop: the features of the interval (x.t, x.t + d]
// with norms nb and nn at its ends, a training record (collection mode; *rec is
// left pointing at it so that the caller can store the crossing's time), and the
// predicted time of the crossing from x.t (-1 without a network).
template <int G>
__device__ __noinline__ double expo_predict(const KernelArgs &a, const Group<G> &g, ExpoProp *PS, double nb,
                                            double nn, double d, double r, unsigned long long n_jump, long long il,
                                            float **rec)
{
    // FP32 features (like the network), so the narrow FP64 pipe is not used for them
    const float gam = __logf((float)nb / (float)nn) / (float)d;
    *rec = nullptr;
    if (g.gl == 0) {
        PS->f[0] = gam;
        PS->f[1] = PS->gam_prev > 0.f ? (gam - PS->gam_prev) / (float)d : 0.f;
        PS->f[2] = (float)nb;
        PS->f[3] = __logf((float)r);
        if (a.rec_stride > 0 && (long long)(n_jump % a.rec_stride) == 0 && PS->rec_n < a.rec_max) {
            float *q = a.rec + ((size_t)il * a.rec_max + PS->rec_n++) * kRecFloats;
            for (int i = 0; i < kMlpIn; ++i) q[i] = PS->f[i];
            q[6] = 0.f;
            *rec = q;
        }
    }
    if (!a.mlp) return -1.0;
    const float y = mlp_eval<G>(g, a.mlp, PS->f, PS->h);  // synchronises before reading f
    const float est = (__logf((float)nb) - __logf((float)r)) / gam;
    double s_hat = (double)(est * __expf(y));
    if (!(s_hat >= 0.0)) s_hat = 0.0;
    if (s_hat > d) s_hat = d;
    return s_hat;
}

// Per-trajectory scalars of a group (indexed at run time; they live in local memory).
struct ExpoTraj {
    double t, r, c, nb;
    long long k, steps;
    int status, jdone;
    unsigned long long n_jump;
};

// The rest of output interval j of trajectory il (Algorithm 1 (B)-(D) inside the
// interval, then the outputs at t_j), given y = exp(M (t_j - x.t)) psi and
// nn = ||y||^2: every crossing of the threshold is found, the jump applied and
// the state propagated on to t_j.  Returns true with psi = psi(t_j) (x.t = t_j,
// x.nb its squared norm), or false with x.status set (x.jdone = j).
template <class Ar, int G, int R, int FEAT, bool DENSE = false>
__device__ bool expo_interval(const KernelArgs &a, const Group<G> &g, const int *si, const typename Ar::real *sv,
                              Expo<Ar, G, R, DENSE> &E, ExpoTraj &x, typename Ar::cplx *psi, typename Ar::cplx *y,
                              double nn, int j, long long il, ExpoProp *PS, unsigned long long &n_acc)
{
    constexpr bool PROP = (FEAT & kFeatProposal) != 0;
    using cplx = typename Ar::cplx;
    const int gl = g.gl;
    for (;;) {
        if (!isfinite(nn)) {
            x.status = 6;
            break;
        }
        if (nn >= x.r) break;
        if (++x.steps > a.max_steps) {
            x.status = 4;
            break;
        }
        // (B): the norm reaches r inside (x.t, t_j]
        cplx *ytau = nullptr;
        const double d = a.t[j] - x.t;
        double s_hat = -1.0;
        float *rec = nullptr;
        if constexpr (PROP) s_hat = expo_predict<G>(a, g, PS, x.nb, nn, d, x.r, x.n_jump, il, &rec);
        const double s = E.crossing(d, psi, x.nb, x.r, x.t, &ytau, s_hat);
        if constexpr (PROP)
            if (rec) rec[7] = (float)s;
        double tau = x.t + s;
        if (tau > a.t[j]) tau = a.t[j];
        // (C)
        const int ch = apply_jump<Ar, G, R, DENSE>(a, g, si, sv, psi, E.u(1), ytau, x.c);
        if (ch < 0) {
            x.status = 7;
            break;
        }
        g.sync();
        if (gl == 0 && (long long)x.n_jump < a.max_jumps) {
            a.jump_t[(size_t)il * a.max_jumps + x.n_jump] = tau;
            a.jump_ch[(size_t)il * a.max_jumps + x.n_jump] = ch;
        }
        ++x.n_jump;
        ++n_acc;
        // (D), then on to t_j
        ++x.k;
        jump_draws(a.seed, a.traj0 + il, x.k, x.r, x.c);
        x.t = tau;
        x.nb = 1.0;
        if constexpr (PROP)
            if (gl == 0) PS->gam_prev = -1.f;
        y = E.propagate(a.t[j] - tau, psi);
        nn = E.norm2(y);
    }
    if (x.status != 0) {
        x.jdone = j;
        return false;
    }
    if constexpr (PROP)  // the decay rate over this (jump-free) stretch, for the next crossing's features
        if (gl == 0) PS->gam_prev = __logf((float)x.nb / (float)nn) / (float)(a.t[j] - x.t);
    record_outputs<Ar, G, R>(a, g, si, sv, y, j, a.out + (size_t)il * a.n_t * a.n_obs, PROP ? PS->f + 4 : nullptr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < a.n) psi[row] = y[row];
    }
    g.sync();
    x.nb = nn;
    x.t = a.t[j];
    ++n_acc;
    return true;
}

// Trajectories il0 .. il0 + live - 1 (live <= T) of the launch, in lock step.
template <class Ar, int G, int R, int T, int FEAT>
__device__ void run_group_expo(const KernelArgs &a, const Group<G> &g, const int *si, const typename Ar::real *sv,
                               const typename Ar::coef *inv, typename Ar::cplx *slots, long long il0, int live,
                               ExpoProp *PS)
{
    constexpr bool PROP = (FEAT & kFeatProposal) != 0;
    static_assert(!PROP || T == 1, "the proposal takes one trajectory per group");
    using cplx = typename Ar::cplx;
    using S = ExpoSlots<T>;
    constexpr int NP = G * R;
    const int n = a.n, gl = g.gl;
    Expo<Ar, G, R> E{a, g, csr_view<Ar>(a.op[0], si, sv), slots + S::kA * NP, slots + S::kB * NP,
                     slots + S::kU * NP, inv};
    cplx *psi_all = slots + S::kPsi * NP;
    cplx *y_all = slots + S::kY * NP;
    ExpoTraj tr[T];
    unsigned long long n_acc = 0;

    // (A): psi0 for the live trajectories, zero in the unused slots
    const cplx *psi0 = static_cast<const cplx *>(a.psi0);
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) psi_all[t * NP + row] = t < live ? psi0[row] : Ar::czero();
        }
    g.sync();
#pragma unroll 1
    for (int t = 0; t < live; ++t) {
        ExpoTraj &x = tr[t];
        x.k = 0;
        jump_draws(a.seed, a.traj0 + il0 + t, 0, x.r, x.c);
        x.t = a.t[0];
        x.steps = 0;
        x.status = 0;
        x.jdone = a.n_t;
        x.n_jump = 0;
        record_outputs<Ar, G, R>(a, g, si, sv, psi_all + t * NP, 0, a.out + (size_t)(il0 + t) * a.n_t * a.n_obs,
                                 PROP ? PS->f + 4 : nullptr);
        x.nb = E.norm2(psi_all + t * NP);
    }
    if constexpr (PROP) {
        if (gl == 0) {
            PS->gam_prev = -1.f;
            PS->rec_n = 0;
        }
    }
#pragma unroll 1
    for (int j = 1; j < a.n_t; ++j) {
        typename Ar::red part[T];
        if (a.expo_uniform) {
            if constexpr (T == 1)
                part[0] = E.level_part(a.expo_levels - 1, psi_all, y_all);
            else
                level_apply<Ar, G, R, T>(E.level(a.expo_levels - 1), psi_all, y_all, gl, n, part);
            g.sync();
        }
        bool any = false;
#pragma unroll 1
        for (int t = 0; t < live; ++t) {
            ExpoTraj &x = tr[t];
            if (x.status != 0) continue;
            any = true;
            cplx *psi = psi_all + t * NP;
            cplx *y;
            double nn;
            ++x.steps;
            if (a.expo_uniform) {
                y = y_all + t * NP;
                typename Ar::red p = Ar::rzero();
#pragma unroll
                for (int q = 0; q < T; ++q)
                    if (q == t) p = part[q];
                nn = Ar::rval(Ar::rsum(g, p));
                ++E.n_rhs;
            } else {
                y = E.propagate(a.t[j] - x.t, psi);
                nn = E.norm2(y);
            }
            expo_interval<Ar, G, R, FEAT>(a, g, si, sv, E, x, psi, y, nn, j, il0 + t, PS, n_acc);
        }
        if (!any) break;
    }

    if (gl == 0) {
        unsigned long long jumps = 0;
        for (int t = 0; t < live; ++t) {
            const ExpoTraj &x = tr[t];
            const long long il = il0 + t;
            if (x.status != 0) {
                double *out = a.out + (size_t)il * a.n_t * a.n_obs;
                for (int j = x.jdone; j < a.n_t; ++j)
                    for (int q = 0; q < a.n_obs; ++q)
                        out[(size_t)j * a.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
                atomicCAS(a.first_error, 0, x.status);
                atomicAdd(&a.counters[kFailed], 1ULL);
            }
            if (a.max_jumps > 0) a.n_jumps[il] = (int)x.n_jump;
            jumps += x.n_jump;
        }
        atomicAdd(&a.counters[kAccepted], n_acc);
        atomicAdd(&a.counters[kRejected], E.n_rej);
        atomicAdd(&a.counters[kRhs], E.n_rhs);
        atomicAdd(&a.counters[kJumps], jumps);
        atomicAdd(&a.counters[kRootIters], (unsigned long long)E.root_iters);
        if constexpr (PROP) atomicAdd(&a.counters[kPropMiss], E.n_miss);
    }
}

// Trajectories per group.  Lock-step batches (one pass over P_L for T
// trajectories) were measured with T = 4 (two rows per lane) and T = 2 (four):
// 8 % faster on dense N = 256 in double-float, but slower everywhere else
// (dense complex64 -43 %, the stiff system -24 %, Jaynes-Cummings -8 to -21 %),
// because each trajectory's outputs, reductions and jumps then run one after
// another inside the group while fewer groups share an SM.  With two CTAs per
// SM restored, T = 2 for complex64 on the multi-warp layouts (dense N = 256)
// measured the same as one trajectory per group (106k trajectories/s).  One
// trajectory per group is kept.
template <int R>
__host__ __device__ constexpr int expo_batch() { return 1; }

// Multi-warp groups: two CTAs per SM (the register bound keeps a second CTA
// resident; one CTA per SM halved the dense complex64 throughput).
template <class Ar, int G, int R, int BLOCK, int FEAT>
__global__ void __launch_bounds__(BLOCK, (G <= 32 ? 4 : 2)) mcwf_expo_kernel(const __grid_constant__ KernelArgs a)
{
    using cplx = typename Ar::cplx;
    using real = typename Ar::real;
    constexpr int T = expo_batch<R>();
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
    using coef = typename Ar::coef;
    coef *inv = reinterpret_cast<coef *>(smem + a.smem_coef_offset);
    if (threadIdx.x <= kExpoTaylor) inv[threadIdx.x] = Ar::coef_of(threadIdx.x ? 1.0 / threadIdx.x : 0.0);
    __syncthreads();
    const Group<G> g(threadIdx.x, reinterpret_cast<unsigned long long *>(smem + a.smem_scratch_offset));
    cplx *slots = reinterpret_cast<cplx *>(smem + a.smem_ybuf_offset) +
                  (size_t)(threadIdx.x / G) * ExpoSlots<T>::kCount * (G * R);
    ExpoProp *PS = (FEAT & kFeatProposal)
                       ? reinterpret_cast<ExpoProp *>(smem + a.smem_mlp_offset + (size_t)(threadIdx.x / G) * kExpoPropStride)
                       : nullptr;
    for (;;) {
        unsigned long long i = 0;
        if (g.gl == 0) i = atomicAdd(a.queue, (unsigned long long)T);
        i = g.bcast0(i);
        if ((long long)i >= a.ntraj) break;
        const long long left = a.ntraj - (long long)i;
        run_group_expo<Ar, G, R, T, FEAT>(a, g, si, sv, inv, slots, (long long)i, left < T ? (int)left : T, PS);
    }
}

template <class Ar, int G, int R, int FEAT = 0>
cudaError_t launch_expo_instance(const KernelArgs &a0, cudaStream_t stream, LaunchInfo *info)
{
    using cplx = typename Ar::cplx;
    constexpr int BLOCK = block_for_group<G>();
    constexpr int GROUPS = BLOCK / G;
    constexpr int T = expo_batch<R>();
    KernelArgs a = a0;
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t ib = ops_in_shared<G>() ? al16((size_t)a.n_ints * sizeof(int)) : 0;
    const size_t vb = ops_in_shared<G>() ? al16((size_t)a.n_vals * sizeof(typename Ar::real)) : 0;
    const size_t sb = al16((size_t)GROUPS * (Group<G>::kWarps + 1) * 8);
    const size_t cb = al16((kExpoTaylor + 1) * sizeof(typename Ar::coef));
    const size_t mb = (FEAT & kFeatProposal) ? (size_t)GROUPS * kExpoPropStride : 0;
    a.smem_vals_offset = (int)ib;
    a.smem_scratch_offset = (int)(ib + vb);
    a.smem_coef_offset = (int)(ib + vb + sb);
    a.smem_mlp_offset = (int)(ib + vb + sb + cb);
    a.smem_ybuf_offset = (int)(ib + vb + sb + cb + mb);
    const size_t smem = ib + vb + sb + cb + mb + (size_t)GROUPS * ExpoSlots<T>::kCount * G * R * sizeof(cplx);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = mcwf_expo_kernel<Ar, G, R, BLOCK, FEAT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem)) != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    const long long need = (a.ntraj + (long long)GROUPS * T - 1) / ((long long)GROUPS * T);
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

// The instantiation for the layout the operators were packed with (a.G, a.R),
// dimension <= 256 (the layouts of layout_candidates up to that size).
template <class Ar>
cudaError_t launch_expo(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    if (a.G == 1 && a.R == 2) return launch_expo_instance<Ar, 1, 2>(a, stream, info);
    if (a.G == 4 && a.R == 2) return launch_expo_instance<Ar, 4, 2>(a, stream, info);
    if (a.G == 8 && a.R == 2) return launch_expo_instance<Ar, 8, 2>(a, stream, info);
    if (a.G == 4 && a.R == 4) return launch_expo_instance<Ar, 4, 4>(a, stream, info);
    if (a.G == 16 && a.R == 2) return launch_expo_instance<Ar, 16, 2>(a, stream, info);
    if (a.G == 8 && a.R == 4) return launch_expo_instance<Ar, 8, 4>(a, stream, info);
    if (a.G == 32 && a.R == 2) return launch_expo_instance<Ar, 32, 2>(a, stream, info);
    if (a.G == 16 && a.R == 4) return launch_expo_instance<Ar, 16, 4>(a, stream, info);
    if (a.G == 64 && a.R == 2) return launch_expo_instance<Ar, 64, 2>(a, stream, info);
    if (a.G == 32 && a.R == 4) return launch_expo_instance<Ar, 32, 4>(a, stream, info);
    if (a.G == 128 && a.R == 2) return launch_expo_instance<Ar, 128, 2>(a, stream, info);
    if (a.G == 64 && a.R == 4) return launch_expo_instance<Ar, 64, 4>(a, stream, info);
    return cudaErrorInvalidValue;
}

// The same with the learned proposal compiled in (single-warp layouts, dimension <= 64).
template <class Ar>
cudaError_t launch_expo_prop(const KernelArgs &a, cudaStream_t stream, LaunchInfo *info)
{
    constexpr int F = kFeatProposal;
    if (a.G == 1 && a.R == 2) return launch_expo_instance<Ar, 1, 2, F>(a, stream, info);
    if (a.G == 4 && a.R == 2) return launch_expo_instance<Ar, 4, 2, F>(a, stream, info);
    if (a.G == 8 && a.R == 2) return launch_expo_instance<Ar, 8, 2, F>(a, stream, info);
    if (a.G == 4 && a.R == 4) return launch_expo_instance<Ar, 4, 4, F>(a, stream, info);
    if (a.G == 16 && a.R == 2) return launch_expo_instance<Ar, 16, 2, F>(a, stream, info);
    if (a.G == 8 && a.R == 4) return launch_expo_instance<Ar, 8, 4, F>(a, stream, info);
    if (a.G == 32 && a.R == 2) return launch_expo_instance<Ar, 32, 2, F>(a, stream, info);
    if (a.G == 16 && a.R == 4) return launch_expo_instance<Ar, 16, 4, F>(a, stream, info);
    if (a.G == 32 && a.R == 4) return launch_expo_instance<Ar, 32, 4, F>(a, stream, info);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Lock-step form (tensor-core products).  On a uniform output grid every output
// interval starts with the same product P_L psi, so all trajectories of a run
// advance together: one launch of the tensor-core engine forms (P_L - I) psi for
// every column (a GEMM; y = psi + that, added here in FP32), then this kernel
// finishes interval lock_j of every column with the code above -- outputs, or
// the crossing search, the jump and the propagation to t_j on the ladder -- one
// group per column.  Complex64 arithmetic (FP32 state and propagators,
// double-float norms); the operators are read from device memory (L1/L2), so
// every layout fits, dense ones (M, C_n) from their column-major FP32 copies:
// the packed form of a dense operator, read row by row from L2 with one
// dependent load chain per entry, made each crossing take milliseconds.
// ---------------------------------------------------------------------------

struct LockCol {
    ExpoTraj x;
    unsigned long long n_acc, n_rhs, n_rej;
    int root_iters;
    int jdef;  // >= 0: the crossing found in interval jdef waits for the catch-up (psi still at t_{jdef-1})
};
static_assert(sizeof(LockCol) == kLockColBytes, "lock-step column record");

// One group's column il in the three modes of the lock-step launch sequence:
//   kLockInterval  interval lock_j (0: start): y = psi + (P_L - I) psi from the
//                  tensor cores; without a crossing in the interval the outputs
//                  at t_j, psi <- y; with one the column is deferred (appended to
//                  the catch-up list, psi kept at t_{j-1})
//   kLockCatchUp   a deferred column (taken from the list): its crossing search,
//                  jump and propagation, then the intervals up to lock_j with the
//                  ladder's P_L (SIMT), so it rejoins the lock step
//   kLockFinish    the column's totals, jump count and failure outputs
template <int G, int R>
__device__ void lockstep_column(const KernelArgs &a, const Group<G> &g, const int *si, const ArF32::real *sv,
                                const ArF32::coef *inv, ArF32::cplx *slots, long long il)
{
    using Ar = ArF32;
    using cplx = Ar::cplx;
    using S = ExpoSlots<1>;
    constexpr int NP = G * R;
    cplx *psi = slots + S::kPsi * NP, *ybuf = slots + S::kY * NP;
    const int n = a.n, gl = g.gl, j = a.lock_j, half = a.lock_ld / 2;
    LockCol *lc = static_cast<LockCol *>(a.lock_col) + il;
    float *gpsi = a.lock_psi + (size_t)il * a.lock_ld;
    Expo<Ar, G, R, true> E{a, g, csr_view<Ar>(a.op[0], si, sv), slots + S::kA * NP, slots + S::kB * NP,
                           slots + S::kU * NP, inv};
    ExpoTraj x;
    int jdef = -1;
    unsigned long long n_acc = 0;
    bool write_psi = false;
    if (a.lock_mode == kLockFinish) {
        if (gl == 0) {
            const LockCol c = *lc;
            if (c.x.status != 0) {
                double *out = a.out + (size_t)il * a.n_t * a.n_obs;
                for (int jj = c.x.jdone; jj < a.n_t; ++jj)
                    for (int q = 0; q < a.n_obs; ++q)
                        out[(size_t)jj * a.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
                atomicCAS(a.first_error, 0, c.x.status);
                atomicAdd(&a.counters[kFailed], 1ULL);
            }
            if (a.max_jumps > 0) a.n_jumps[il] = (int)c.x.n_jump;
            atomicAdd(&a.counters[kAccepted], c.n_acc);
            atomicAdd(&a.counters[kRejected], c.n_rej);
            atomicAdd(&a.counters[kRhs], c.n_rhs);
            atomicAdd(&a.counters[kJumps], c.x.n_jump);
            atomicAdd(&a.counters[kRootIters], (unsigned long long)c.root_iters);
        }
        return;
    }
    if (a.lock_mode == kLockInterval && j == 0) {
        // (A): psi0, the first draws, output 0
        const cplx *psi0 = static_cast<const cplx *>(a.psi0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) psi[row] = psi0[row];
        }
        g.sync();
        x.k = 0;
        jump_draws(a.seed, a.traj0 + il, 0, x.r, x.c);
        x.t = a.t[0];
        x.steps = 0;
        x.status = 0;
        x.jdone = a.n_t;
        x.n_jump = 0;
        record_outputs<Ar, G, R>(a, g, si, sv, psi, 0, a.out + (size_t)il * a.n_t * a.n_obs, nullptr);
        x.nb = E.norm2(psi);
        write_psi = true;
    } else {
        x = lc->x;
        jdef = lc->jdef;
        if (x.status != 0) return;
        if (a.lock_mode == kLockInterval) {
            if (jdef >= 0) return;  // waiting for the catch-up
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) {  // y = psi + (P_L - I) psi
                    const float pr = gpsi[row], pi = gpsi[half + row];
                    psi[row] = cplx{pr, pi};
                    ybuf[row] = cplx{pr + a.lock_y[(size_t)il * a.lock_ld + row],
                                     pi + a.lock_y[(size_t)il * a.lock_ld + half + row]};
                }
            }
            g.sync();
            ++E.n_rhs;  // the tensor cores' product
            const double nn = E.norm2(ybuf);
            if (nn < x.r) {  // a crossing: deferred to the catch-up
                jdef = j;
                if (gl == 0) a.lock_list[atomicAdd(&a.queue[0], 1ULL)] = (int)il;
            } else {
                ++x.steps;
                write_psi = expo_interval<Ar, G, R, 0, true>(a, g, si, sv, E, x, psi, ybuf, nn, j, il, nullptr, n_acc);
            }
        } else {  // kLockCatchUp: intervals jdef .. lock_j on the ladder
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) psi[row] = cplx{gpsi[row], gpsi[half + row]};
            }
            g.sync();
            bool ok = true;
#pragma unroll 1
            for (int jj = jdef; jj <= j && ok; ++jj) {
                const double nn = E.apply_level(a.expo_levels - 1, psi, ybuf);
                ++x.steps;
                ok = expo_interval<Ar, G, R, 0, true>(a, g, si, sv, E, x, psi, ybuf, nn, jj, il, nullptr, n_acc);
            }
            jdef = -1;
            write_psi = ok;
        }
    }
    if (write_psi) {  // psi(t_j) back to its column
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                gpsi[row] = psi[row].re;
                gpsi[half + row] = psi[row].im;
            }
        }
    }
    const bool fresh = a.lock_mode == kLockInterval && j == 0;
    const unsigned long long acc_tot = n_acc + (fresh ? 0 : lc->n_acc);
    const unsigned long long rhs_tot = E.n_rhs + (fresh ? 0 : lc->n_rhs);
    const unsigned long long rej_tot = E.n_rej + (fresh ? 0 : lc->n_rej);
    const int root_tot = E.root_iters + (fresh ? 0 : lc->root_iters);
    g.sync();  // every lane has read the record before lane 0 rewrites it
    if (gl == 0) {
        lc->x = x;
        lc->jdef = jdef;
        lc->n_acc = acc_tot;
        lc->n_rhs = rhs_tot;
        lc->n_rej = rej_tot;
        lc->root_iters = root_tot;
    }
}

// kLockInterval in a light instantiation of its own (the interval and start
// launches): the same work as lockstep_column's interval mode, with one vector
// slot per group and none of the crossing code, so that many more groups fit
// per SM than in the catch-up's instantiation (13 slots, 128 registers).
template <int G, int R>
__device__ void lockstep_interval(const KernelArgs &a, const Group<G> &g, const int *si, const ArF32::real *sv,
                                  ArF32::cplx *ybuf, long long il)
{
    using Ar = ArF32;
    using cplx = Ar::cplx;
    const int n = a.n, gl = g.gl, j = a.lock_j, half = a.lock_ld / 2;
    LockCol *lc = static_cast<LockCol *>(a.lock_col) + il;
    float *gpsi = a.lock_psi + (size_t)il * a.lock_ld;
    auto norm2 = [&]() {
        Ar::red nn = Ar::rzero();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) nn = Ar::radd(nn, Ar::abs2(ybuf[row]));
        }
        return Ar::rval(Ar::rsum(g, nn));
    };
    ExpoTraj x;
    int jdef = -1;
    unsigned long long acc = 0, rhs = 0;
    bool write_psi = false;
    if (j == 0) {
        // (A): psi0, the first draws, output 0
        const cplx *psi0 = static_cast<const cplx *>(a.psi0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) ybuf[row] = psi0[row];
        }
        g.sync();
        x.k = 0;
        jump_draws(a.seed, a.traj0 + il, 0, x.r, x.c);
        x.t = a.t[0];
        x.steps = 0;
        x.status = 0;
        x.jdone = a.n_t;
        x.n_jump = 0;
        record_outputs<Ar, G, R>(a, g, si, sv, ybuf, 0, a.out + (size_t)il * a.n_t * a.n_obs, nullptr);
        x.nb = norm2();
        write_psi = true;
    } else {
        x = lc->x;
        jdef = lc->jdef;
        if (x.status != 0 || jdef >= 0) return;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n)  // y = psi + (P_L - I) psi
                ybuf[row] = cplx{gpsi[row] + a.lock_y[(size_t)il * a.lock_ld + row],
                                 gpsi[half + row] + a.lock_y[(size_t)il * a.lock_ld + half + row]};
        }
        g.sync();
        rhs = 1;  // the tensor cores' product
        const double nn = norm2();
        if (nn < x.r) {  // a crossing: deferred to the catch-up
            jdef = j;
            if (gl == 0) a.lock_list[atomicAdd(&a.queue[0], 1ULL)] = (int)il;
        } else {
            ++x.steps;
            if (!isfinite(nn)) {
                x.status = 6;
                x.jdone = j;
            } else {
                record_outputs<Ar, G, R>(a, g, si, sv, ybuf, j, a.out + (size_t)il * a.n_t * a.n_obs, nullptr);
                x.nb = nn;
                x.t = a.t[j];
                acc = 1;
                write_psi = true;
            }
        }
    }
    if (write_psi) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = gl + G * r;
            if (row < n) {
                gpsi[row] = ybuf[row].re;
                gpsi[half + row] = ybuf[row].im;
            }
        }
    }
    const unsigned long long acc_tot = acc + (j == 0 ? 0 : lc->n_acc);
    const unsigned long long rhs_tot = rhs + (j == 0 ? 0 : lc->n_rhs);
    const unsigned long long rej_tot = j == 0 ? 0 : lc->n_rej;
    const int root_tot = j == 0 ? 0 : lc->root_iters;
    g.sync();  // every lane has read the record before lane 0 rewrites it
    if (gl == 0) {
        lc->x = x;
        lc->jdef = jdef;
        lc->n_acc = acc_tot;
        lc->n_rhs = rhs_tot;
        lc->n_rej = rej_tot;
        lc->root_iters = root_tot;
    }
}

template <int G, int R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (G <= 32 ? 6 : 3)) mcwf_expo_interval_kernel(const __grid_constant__ KernelArgs a)
{
    using Ar = ArF32;
    using cplx = Ar::cplx;
    constexpr int NP = G * R;
    constexpr int GROUPS = BLOCK / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const Group<G> g(threadIdx.x, reinterpret_cast<unsigned long long *>(smem + a.smem_scratch_offset));
    cplx *ybuf = reinterpret_cast<cplx *>(smem + a.smem_ybuf_offset) + (size_t)(threadIdx.x / G) * NP;
    const int *si = a.ints;
    const Ar::real *sv = static_cast<const Ar::real *>(a.vals);
    for (long long il = (long long)blockIdx.x * GROUPS + threadIdx.x / G; il < a.ntraj;
         il += (long long)gridDim.x * GROUPS) {
        lockstep_interval<G, R>(a, g, si, sv, ybuf, il);
        g.sync();
    }
}

template <int G, int R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (G <= 32 ? 4 : 2)) mcwf_expo_lockstep_kernel(const __grid_constant__ KernelArgs a)
{
    using Ar = ArF32;
    using cplx = Ar::cplx;
    using real = Ar::real;
    constexpr int NP = G * R;
    constexpr int GROUPS = BLOCK / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const int *si = a.ints;
    const real *sv = static_cast<const real *>(a.vals);
    Ar::coef *inv = reinterpret_cast<Ar::coef *>(smem + a.smem_coef_offset);
    if (threadIdx.x <= kExpoTaylor) inv[threadIdx.x] = Ar::coef_of(threadIdx.x ? 1.0 / threadIdx.x : 0.0);
    __syncthreads();
    const Group<G> g(threadIdx.x, reinterpret_cast<unsigned long long *>(smem + a.smem_scratch_offset));
    cplx *slots = reinterpret_cast<cplx *>(smem + a.smem_ybuf_offset) +
                  (size_t)(threadIdx.x / G) * ExpoSlots<1>::kCount * NP;
    if (a.lock_mode == kLockCatchUp) {
        // the deferred columns, one at a time per group from the shared list
        const long long count = (long long)a.queue[0];
        for (;;) {
            unsigned long long i = 0;
            if (g.gl == 0) i = atomicAdd(&a.queue[1], 1ULL);
            i = g.bcast0(i);
            if ((long long)i >= count) break;
            lockstep_column<G, R>(a, g, si, sv, inv, slots, (long long)a.lock_list[i]);
            g.sync();
        }
        return;
    }
    for (long long il = (long long)blockIdx.x * GROUPS + threadIdx.x / G; il < a.ntraj;
         il += (long long)gridDim.x * GROUPS) {
        lockstep_column<G, R>(a, g, si, sv, inv, slots, il);
        g.sync();
    }
}

template <int G, int R>
cudaError_t launch_expo_lockstep_instance(const KernelArgs &a0, cudaStream_t stream, LaunchInfo *info)
{
    using cplx = ArF32::cplx;
    constexpr int BLOCK = block_for_group<G>();
    constexpr int GROUPS = BLOCK / G;
    KernelArgs a = a0;
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const bool light = a.lock_mode == kLockInterval;
    const size_t sb = al16((size_t)GROUPS * (Group<G>::kWarps + 1) * 8);
    const size_t cb = light ? 0 : al16((kExpoTaylor + 1) * sizeof(ArF32::coef));
    a.smem_vals_offset = 0;
    a.smem_scratch_offset = 0;
    a.smem_coef_offset = (int)sb;
    a.smem_mlp_offset = (int)(sb + cb);
    a.smem_ybuf_offset = (int)(sb + cb);
    const size_t smem = sb + cb + (size_t)GROUPS * (light ? 1 : ExpoSlots<1>::kCount) * G * R * sizeof(cplx);
    if (smem > 227 * 1024 || a.lock_ld < 2 * a.n) return cudaErrorInvalidValue;
    auto kern = light ? mcwf_expo_interval_kernel<G, R, BLOCK> : mcwf_expo_lockstep_kernel<G, R, BLOCK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

}  // namespace qtm
