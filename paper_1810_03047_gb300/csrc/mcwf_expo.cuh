// mcwf_expo.cuh -- Algorithm 1 (Sec. 2.2) with the no-jump evolution applied
// exactly: between two jumps d psi/dt = M psi with a constant M = -i H_eff, so
// psi(t) = exp(M (t - t_k)) psi_k.  This is the library's method for stiff
// problems (Sec. 2.1: the paper switches ZVODE to BDF there), where an explicit
// integrator's step is set by the largest decay rate rather than by accuracy.
//
// The host precomputes a ladder of propagators P_l = exp(M delta 2^l),
// l = 0..L, with delta chosen so that nu delta <= 1/16 (nu >= ||M||_2) and
// delta 2^L = the output spacing.  Per trajectory (G lanes, R rows per lane,
// vectors in shared memory as in mcwf_kernel.cuh):
//   * between outputs: psi(t_j) = P_L psi(t_{j-1}) on a uniform grid (one dense
//     product); otherwise the duration d is split into its binary digits in
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
//     propagation restarts at tau.
// No step-size control and no interpolation are involved: a trajectory differs
// from the exact one by rounding and by the root tolerance only, whatever the
// stiffness of M.
#pragma once

#include "mcwf_kernel.cuh"

namespace qtm {

constexpr int kExpoTaylor = 9;  // degree of the Taylor polynomial of exp(s M), s <= delta

// Vector slots of one trajectory group: the state, two product buffers and the
// Taylor vectors u_1..u_9.  u_1 sits in the slot apply_jump uses as scratch (it
// is dead once the jump time is known).
enum ExpoSlot { kEPsi = 0, kEA = 1, kEU = 2, kEB = kEU + kExpoTaylor, kNumExpoSlots = kEB + 1 };
static_assert(kEU == kYn && kEPsi == kPsi, "apply_jump writes slot kPsi and uses slot kYn as scratch");

// out = P x on the lane's rows; P is column-major with G R rows per column (zero
// below n).  Returns the lane's part of ||out||^2.  x is synchronised.
template <class Ar, int G, int R>
__device__ __forceinline__ typename Ar::red level_apply(const typename Ar::cplx *__restrict__ P,
                                                        const typename Ar::cplx *x, typename Ar::cplx *out,
                                                        int gl, int n)
{
    constexpr int NP = G * R;
    typename Ar::acc acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = Ar::zero();
    const typename Ar::cplx *col = P + gl;
#pragma unroll 4
    for (int c = 0; c < n; ++c) {
        const typename Ar::cplx xc = x[c];
#pragma unroll
        for (int r = 0; r < R; ++r) Ar::mac(acc[r], col[G * r], xc);
        col += NP;
    }
    typename Ar::red nn = Ar::rzero();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) {
            const typename Ar::cplx v = Ar::get(acc[r]);
            out[row] = v;
            nn = Ar::radd(nn, Ar::abs2(v));
        }
    }
    return nn;
}

template <class Ar, int G, int R>
struct Expo {
    using cplx = typename Ar::cplx;
    static constexpr int NP = G * R;
    const KernelArgs &a;
    const Group<G> &g;
    CsrView<Ar> M;
    cplx *v;  // the group's slots
    unsigned long long n_rhs = 0, n_rej = 0;
    int root_iters = 0;

    __device__ cplx *slot(int s) const { return v + s * NP; }
    __device__ const cplx *level(int l) const
    {
        return static_cast<const cplx *>(a.expo) + (size_t)l * a.n * NP;
    }

    // lane-summed ||y||^2 of a synchronised buffer
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

    // out = P_l x, synchronised; returns ||out||^2
    __device__ double apply_level(int l, const cplx *x, cplx *out)
    {
        const typename Ar::red p = level_apply<Ar, G, R>(level(l), x, out, g.gl, a.n);
        const double nn = Ar::rval(Ar::rsum(g, p));
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
#pragma unroll 1
        for (int m = kExpoTaylor; m >= 1; --m) {
            const typename Ar::coef sm = Ar::coef_of(s / m);
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const cplx mv = spmv_row<Ar, G>(M, src, g.gl, r);
                const int row = g.gl + G * r;
                if (row < a.n) {
                    typename Ar::acc acc = Ar::zero();
                    Ar::axpy(acc, sm, mv);
                    dst[row] = Ar::add_scaled(x[row], Ar::coef_of(1.0), acc);
                }
            }
            g.sync();
            ++n_rhs;
            src = dst;
            dst = (dst == w0) ? w1 : w0;
        }
        return const_cast<cplx *>(src);
    }

    // exp(d M) psi: the binary digits of d / delta on the ladder, then the
    // remainder by Taylor.  Returns the buffer holding the result (never psi).
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
        cplx *A = slot(kEA), *B = slot(kEB);
        const cplx *cur = psi;
#pragma unroll 1
        for (int l = L; l >= 0; --l)
            if ((q >> l) & 1ULL) {
                cplx *out = (cur == A) ? B : A;
                apply_level(l, cur, out);
                cur = out;
            }
        if (rem > 0.0) return taylor(cur, slot(kEU), slot(kEU + 1), rem);
        if (cur == psi) {  // d == 0: a copy, so that the caller may overwrite psi
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

    // (B) with ||psi||^2 = nb >= r now and ||exp(d M) psi||^2 < r: the time s in
    // (0, d] of the crossing; psi(s) is left in *out (synchronised).
    __device__ double crossing(double d, const cplx *psi, double nb, double r, double t0, cplx **out)
    {
        const int L = a.expo_levels - 1;
        const double delta = a.expo_delta;
        cplx *A = slot(kEA), *B = slot(kEB);
        const cplx *base = psi;
        double cur = 0.0;
        // binary descent: keep level l when the norm after it is still >= r
#pragma unroll 1
        for (int l = L; l >= 0; --l) {
            const double step = ldexp(delta, l);
            if (cur + step > d) continue;
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
        double smax = d - cur;
        if (smax > delta) smax = delta;
        if (smax < 0.0) smax = 0.0;
        // u_m = M u_{m-1} / m, u_0 = base
        const cplx *prev = base;
#pragma unroll 1
        for (int m = 1; m <= kExpoTaylor; ++m) {
            cplx *um = slot(kEU + m - 1);
            const typename Ar::coef inv = Ar::coef_of(1.0 / m);
#pragma unroll 1
            for (int r2 = 0; r2 < R; ++r2) {
                const cplx mv = spmv_row<Ar, G>(M, prev, g.gl, r2);
                const int row = g.gl + G * r2;
                if (row < a.n) {
                    typename Ar::acc acc = Ar::zero();
                    Ar::axpy(acc, inv, mv);
                    um[row] = Ar::get(acc);
                }
            }
            g.sync();
            ++n_rhs;
            prev = um;
        }
        // f(s) = ||sum_m s^m u_m||^2 - r and f'(s) = 2 Re<psi(s), psi'(s)>
        auto eval = [&](double s, double &fp) {
            typename Ar::red nn = Ar::rzero(), dd = Ar::rzero();
#pragma unroll 1
            for (int r2 = 0; r2 < R; ++r2) {
                const int row = g.gl + G * r2;
                if (row < a.n) {
                    typename Ar::acc y = Ar::zero(), yp = Ar::zero();
                    double sp = 1.0;  // s^(m-1)
#pragma unroll
                    for (int m = 1; m <= kExpoTaylor; ++m) {
                        const cplx um = slot(kEU + m - 1)[row];
                        Ar::axpy(yp, Ar::coef_of(m * sp), um);
                        sp *= s;
                        Ar::axpy(y, Ar::coef_of(sp), um);
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
#pragma unroll 1
        for (int r2 = 0; r2 < R; ++r2) {
            const int row = g.gl + G * r2;
            if (row < a.n) {
                typename Ar::acc y = Ar::zero();
                double sp = 1.0;
#pragma unroll
                for (int m = 1; m <= kExpoTaylor; ++m) {
                    sp *= s;
                    Ar::axpy(y, Ar::coef_of(sp), slot(kEU + m - 1)[row]);
                }
                o[row] = Ar::add_scaled(base[row], Ar::coef_of(1.0), y);
            }
        }
        g.sync();
        *out = o;
        return cur + s;
    }
};

template <class Ar, int G, int R>
__device__ void run_trajectory_expo(const KernelArgs &a, const Group<G> &g, const int *si,
                                    const typename Ar::real *sv, typename Ar::cplx *slots, long long il)
{
    using cplx = typename Ar::cplx;
    constexpr int NP = G * R;
    const int n = a.n, gl = g.gl;
    const long long traj = a.traj0 + il;
    double *out = a.out + (size_t)il * a.n_t * a.n_obs;
    Expo<Ar, G, R> E{a, g, csr_view<Ar>(a.op[0], si, sv), slots};
    Lanes<Ar, G, R> L{slots, gl, n, 0};
    cplx *psi = slots + kEPsi * NP;
    cplx *A = slots + kEA * NP;

    int status = 0;
    unsigned long long n_acc = 0, n_jump = 0;
    long long steps = 0;

    // (A)
    const cplx *psi0 = static_cast<const cplx *>(a.psi0);
#pragma unroll
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
    double nb = E.norm2(psi);
    bool at_grid = true;
    int j = 1;
    while (j < a.n_t) {
        if (++steps > a.max_steps) {
            status = 4;
            break;
        }
        const double d = a.t[j] - t;
        cplx *y;
        double nn;
        if (a.expo_uniform && at_grid) {
            y = A;
            nn = E.apply_level(a.expo_levels - 1, psi, A);
        } else {
            y = E.propagate(d, psi);
            nn = E.norm2(y);
        }
        if (!isfinite(nn)) {
            status = 6;
            break;
        }
        if (nn >= rk) {
            record_outputs<Ar, G, R>(a, g, si, sv, y, j, out, nullptr);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = gl + G * r;
                if (row < n) psi[row] = y[row];
            }
            g.sync();
            nb = nn;
            t = a.t[j];
            ++j;
            ++n_acc;
            at_grid = true;
            continue;
        }
        // (B): the norm reaches r inside (t, t_j]
        cplx *ytau = nullptr;
        const double s = E.crossing(d, psi, nb, rk, t, &ytau);
        double tau = t + s;
        if (tau > a.t[j]) tau = a.t[j];
        // (C)
        const int ch = apply_jump<Ar, G, R>(a, g, si, sv, L, ytau, ck);
        if (ch < 0) {
            status = 7;
            break;
        }
        g.sync();
        if (gl == 0 && (long long)n_jump < a.max_jumps) {
            a.jump_t[(size_t)il * a.max_jumps + n_jump] = tau;
            a.jump_ch[(size_t)il * a.max_jumps + n_jump] = ch;
        }
        ++n_jump;
        ++n_acc;
        // (D)
        ++k;
        jump_draws(a.seed, traj, k, rk, ck);
        t = tau;
        nb = 1.0;
        at_grid = false;
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
        atomicAdd(&a.counters[kRejected], E.n_rej);
        atomicAdd(&a.counters[kRhs], E.n_rhs);
        atomicAdd(&a.counters[kJumps], n_jump);
        atomicAdd(&a.counters[kRootIters], (unsigned long long)E.root_iters);
    }
}

template <class Ar, int G, int R, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (G <= 32 ? 4 : 1)) mcwf_expo_kernel(const __grid_constant__ KernelArgs a)
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
    __syncthreads();
    const Group<G> g(threadIdx.x, reinterpret_cast<unsigned long long *>(smem + a.smem_scratch_offset));
    cplx *slots = reinterpret_cast<cplx *>(smem + a.smem_ybuf_offset) + (threadIdx.x / G) * kNumExpoSlots * (G * R);
    for (;;) {
        unsigned long long i = 0;
        if (g.gl == 0) i = atomicAdd(a.queue, 1ULL);
        i = g.bcast0(i);
        if ((long long)i >= a.ntraj) break;
        run_trajectory_expo<Ar, G, R>(a, g, si, sv, slots, (long long)i);
    }
}

template <class Ar, int G, int R>
cudaError_t launch_expo_instance(const KernelArgs &a0, cudaStream_t stream, LaunchInfo *info)
{
    using cplx = typename Ar::cplx;
    constexpr int BLOCK = block_for_group<G>();
    constexpr int GROUPS = BLOCK / G;
    KernelArgs a = a0;
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t ib = ops_in_shared<G>() ? al16((size_t)a.n_ints * sizeof(int)) : 0;
    const size_t vb = ops_in_shared<G>() ? al16((size_t)a.n_vals * sizeof(typename Ar::real)) : 0;
    const size_t sb = al16((size_t)GROUPS * (Group<G>::kWarps + 1) * 8);
    a.smem_vals_offset = (int)ib;
    a.smem_scratch_offset = (int)(ib + vb);
    a.smem_ybuf_offset = (int)(ib + vb + sb);
    const size_t smem = ib + vb + sb + (size_t)GROUPS * kNumExpoSlots * G * R * sizeof(cplx);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = mcwf_expo_kernel<Ar, G, R, BLOCK>;
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

}  // namespace qtm
