// mcwf_kernel.cuh -- the trajectory kernel: Algorithm 1 (Sec. 2.2) of the QTM
// paper for a whole ensemble in one persistent launch.
//
// Mapping onto the GPU.  G consecutive lanes of a warp own one trajectory; lane
// gl keeps rows gl, gl+G, ... (R of them) of every Dormand-Prince vector -- the
// state psi, the seven stage derivatives K_0..K_6 and the candidate ynew -- in
// registers for the trajectory's whole life.  The only data that crosses lanes is
// the stage vector entering each product M y: the lanes write their rows into a
// small shared-memory exchange buffer (two alternating halves, one warp-level
// barrier per product) and read back the entries their CSR rows need.  All
// operators (M = -i H_eff, the C_n and the A_k) are staged once per CTA into
// shared memory.  Groups pull trajectory ids from a global counter and start the
// next trajectory as soon as theirs ends, so uneven trajectory lifetimes do not
// idle lanes.  Every decision (accept/reject, crossing, output times, channel) is
// taken from values reduced with a butterfly, which leaves the bitwise-identical
// value in every lane of the group, so control flow is uniform per group.
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

#include "qtm_device.cuh"
#include "qtm_launch.h"

namespace qtm {

template <class V>
struct CsrView {
    const int *rp;
    const int *ci;
    const cpx<V> *val;
};

template <class V>
__device__ __forceinline__ CsrView<V> csr_view(const OpOffsets &o, const int *si, const cpx<V> *sv)
{
    return CsrView<V>{si + o.rp, si + o.ci, sv + o.val};
}

// Two alternating halves of the group's exchange buffer.  Each write is followed
// by a group barrier before any lane reads, so a half is never rewritten while a
// lane may still read it (that lane has passed the barrier of the write in between).
template <class V>
struct XBuf {
    cpx<V> *base;
    int np;
    int cur;
    __device__ __forceinline__ cpx<V> *next()
    {
        cur ^= 1;
        return base + cur * np;
    }
};

template <class V, int G, int R>
__device__ __forceinline__ void put_rows(cpx<V> *buf, const cpx<V> (&y)[R], int gl, int n)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        if (row < n) buf[row] = y[r];
    }
}

// out = A buf on the lane's rows
template <class V, int G, int R>
__device__ __forceinline__ void spmv_rows(const CsrView<V> &A, const cpx<V> *buf, cpx<V> (&out)[R],
                                          int gl, int n)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        cpx<V> acc = czero<V>();
        if (row < n) {
            const int k1 = A.rp[row + 1];
            for (int k = A.rp[row]; k < k1; ++k) acc = cmac(acc, A.val[k], buf[A.ci[k]]);
        }
        out[r] = acc;
    }
}

// y(t + theta h) = psi + h sum_j w_j(theta) K_j with w_j in monomial form
template <class V, int R>
__device__ __forceinline__ void dense_output(const cpx<V> (&psi)[R], const cpx<V> (&K)[7][R],
                                             double h, double th, cpx<V> (&y)[R])
{
    double w[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const double p = (((DP5::W(j, 5) * th + DP5::W(j, 4)) * th + DP5::W(j, 3)) * th
                          + DP5::W(j, 2)) * th + DP5::W(j, 1);
        w[j] = h * p * th;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cpx<V> acc = psi[r];
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if (j != 1) acc = caxpy(acc, (V)w[j], K[j][r]);
        y[r] = acc;
    }
}

// Output j: Re<y|A_k|y>/<y|y> for every observable, written by lane 0.
template <class V, int G, int R>
__device__ void record_outputs(const KernelArgs &a, const Group<G> &g, const int *si,
                               const cpx<V> *sv, XBuf<V> &xb, const cpx<V> (&y)[R], int j,
                               double *out)
{
    cpx<V> *b = xb.next();
    put_rows<V, G, R>(b, y, g.gl, a.n);
    g.sync();
    double nn = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) nn += (double)cabs2(y[r]);
    nn = g.sum(nn);
    for (int k = 0; k < a.n_obs; ++k) {
        const CsrView<V> A = csr_view<V>(a.op[1 + a.n_c + k], si, sv);
        cpx<V> ay[R];
        spmv_rows<V, G, R>(A, b, ay, g.gl, a.n);
        double ev = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) ev += (double)y[r].re * ay[r].re + (double)y[r].im * ay[r].im;
        ev = g.sum(ev);
        if (g.gl == 0) out[(size_t)j * a.n_obs + k] = ev / nn;
    }
}

// First theta in (0, 1] where ||y(theta)||^2 = r.  ||y(theta)||^2 = sum_s P_s theta^s
// with y(theta) = sum_m theta^m u_m, u_0 = psi, u_m = h sum_j W(j, m) K_j, and
// P_s = sum_{m + m' = s} Re<u_m, u_m'>.
template <class V, int G, int R>
__device__ double locate_crossing(const Group<G> &g, const cpx<V> (&psi)[R],
                                  const cpx<V> (&K)[7][R], double h, double r, int &iters)
{
    double gram[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) gram[q] = 0.0;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        cpx<V> u[6];
        u[0] = psi[rr];
#pragma unroll
        for (int m = 1; m <= 5; ++m) {
            cpx<V> acc = czero<V>();
#pragma unroll
            for (int j = 0; j < 7; ++j)
                if (DP5::W(j, m) != 0.0) acc = caxpy(acc, (V)(h * DP5::W(j, m)), K[j][rr]);
            u[m] = acc;
        }
        int q = 0;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int m2 = m; m2 < 6; ++m2, ++q)
                gram[q] += (double)u[m].re * u[m2].re + (double)u[m].im * u[m2].im;
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
                const double v = g.sum(gram[q]);
                P[m + m2] += (m == m2) ? v : 2.0 * v;
            }
    }
    P[0] -= r;
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

template <class V, int G, int R>
__device__ void run_trajectory(const KernelArgs &a, const Group<G> &g, const int *si,
                               const cpx<V> *sv, XBuf<V> &xb, long long il)
{
    const int n = a.n;
    const int gl = g.gl;
    const long long traj = a.traj0 + il;
    const double t_end = a.t[a.n_t - 1];
    double *out = a.out + (size_t)il * a.n_t * a.n_obs;
    const CsrView<V> M = csr_view<V>(a.op[0], si, sv);
    const double rtol = a.rtol, atol = a.atol;

    cpx<V> psi[R], K[7][R];
    int status = 0;
    long long attempts = 0;
    unsigned long long n_acc = 0, n_rej = 0, n_rhs = 0, n_jump = 0;
    int root_iters = 0;

    const cpx<V> *psi0 = static_cast<const cpx<V> *>(a.psi0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = gl + G * r;
        psi[r] = row < n ? psi0[row] : czero<V>();
    }

    // (A)
    long long k = 0;
    double rk, ck;
    jump_draws(a.seed, traj, k, rk, ck);
    double t = a.t[0];
    record_outputs<V, G, R>(a, g, si, sv, xb, psi, 0, out);
    int j = 1;

    {
        cpx<V> *b = xb.next();
        put_rows<V, G, R>(b, psi, gl, n);
        g.sync();
        spmv_rows<V, G, R>(M, b, K[0], gl, n);
        ++n_rhs;
    }

    // starting step (Hairer, Norsett & Wanner, Sec. II.4)
    double h;
    {
        const double span = t_end - t;
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double ay = sqrt((double)cabs2(psi[r]));
            const double sc = atol + rtol * ay;
            d0 += (double)cabs2(psi[r]) / (sc * sc);
            d1 += (double)cabs2(K[0][r]) / (sc * sc);
        }
        d0 = sqrt(g.sum(d0) / n);
        d1 = sqrt(g.sum(d1) / n);
        double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        if (h0 > span) h0 = span;
        cpx<V> y1[R], f1[R];
#pragma unroll
        for (int r = 0; r < R; ++r) y1[r] = caxpy(psi[r], (V)h0, K[0][r]);
        cpx<V> *b = xb.next();
        put_rows<V, G, R>(b, y1, gl, n);
        g.sync();
        spmv_rows<V, G, R>(M, b, f1, gl, n);
        ++n_rhs;
        double d2 = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double ay = sqrt((double)cabs2(psi[r]));
            const double sc = atol + rtol * ay;
            const double dre = (double)f1[r].re - K[0][r].re, dim = (double)f1[r].im - K[0][r].im;
            d2 += (dre * dre + dim * dim) / (sc * sc);
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
            for (; j < a.n_t; ++j) record_outputs<V, G, R>(a, g, si, sv, xb, psi, j, out);
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

        // (B): one Dormand-Prince attempt; K[6] = M ynew
        cpx<V> yn[R];
#pragma unroll
        for (int s = 1; s < 7; ++s) {
            cpx<V> ys[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                cpx<V> acc = czero<V>();
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    if (q < s && DP5::a(s, q) != 0.0) acc = caxpy(acc, (V)DP5::a(s, q), K[q][r]);
                ys[r] = caxpy(psi[r], (V)h, acc);
            }
            if (s == 6) {
#pragma unroll
                for (int r = 0; r < R; ++r) yn[r] = ys[r];
            }
            cpx<V> *b = xb.next();
            put_rows<V, G, R>(b, ys, gl, n);
            g.sync();
            spmv_rows<V, G, R>(M, b, K[s], gl, n);
        }
        n_rhs += 6;
        ++attempts;

        double esum = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (gl + G * r < n) {
                cpx<V> e = czero<V>();
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    if (DP5::e(q) != 0.0) e = caxpy(e, (V)DP5::e(q), K[q][r]);
                const double ere = h * (double)e.re, eim = h * (double)e.im;
                const double ay = sqrt((double)cabs2(psi[r]));
                const double an = sqrt((double)cabs2(yn[r]));
                const double sc = atol + rtol * (ay > an ? ay : an);
                esum += (ere * ere + eim * eim) / (sc * sc);
            }
        }
        const double err = sqrt(g.sum(esum) / n);

        if (!(err <= 1.0)) {
            if (!isfinite(err)) {
                status = 6;
                break;
            }
            double fac = kSafety * pow(err, -0.2);
            if (fac < kFacMin) fac = kFacMin;
            h *= fac;
            rejected_before = true;
            ++n_rej;
            continue;
        }
        ++n_acc;
        const double t_new = last ? t_end : t + h;
        double nn = 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) nn += (double)cabs2(yn[r]);
        nn = g.sum(nn);

        if (nn < rk) {
            // (C): the norm reached r inside this step
            const double th = locate_crossing<V, G, R>(g, psi, K, h, rk, root_iters);
            double tau = t + th * h;
            if (tau > t_new) tau = t_new;
            for (; j < a.n_t && a.t[j] <= tau; ++j) {
                double thj = (a.t[j] - t) / h;
                if (thj > 1.0) thj = 1.0;
                cpx<V> yd[R];
                dense_output<V, R>(psi, K, h, thj, yd);
                record_outputs<V, G, R>(a, g, si, sv, xb, yd, j, out);
            }
            cpx<V> yd[R];
            dense_output<V, R>(psi, K, h, th, yd);
            cpx<V> *b = xb.next();
            put_rows<V, G, R>(b, yd, gl, n);
            g.sync();
            double wq[kMaxChannels];
            double wsum = 0.0;
            for (int q = 0; q < a.n_c; ++q) {
                cpx<V> cy[R];
                spmv_rows<V, G, R>(csr_view<V>(a.op[1 + q], si, sv), b, cy, gl, n);
                double part = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r) part += (double)cabs2(cy[r]);
                wq[q] = g.sum(part);
                wsum += wq[q];
            }
            if (!(wsum > 0.0)) {
                status = 7;
                break;
            }
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
            cpx<V> cy[R];
            spmv_rows<V, G, R>(csr_view<V>(a.op[1 + ch], si, sv), b, cy, gl, n);
            const double nc = sqrt(wq[ch]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                psi[r].re = (V)((double)cy[r].re / nc);
                psi[r].im = (V)((double)cy[r].im / nc);
            }
            if (gl == 0 && (long long)n_jump < a.max_jumps) {
                a.jump_t[(size_t)il * a.max_jumps + n_jump] = tau;
                a.jump_ch[(size_t)il * a.max_jumps + n_jump] = ch;
            }
            ++n_jump;

            // (D)
            ++k;
            jump_draws(a.seed, traj, k, rk, ck);
            t = tau;
            b = xb.next();
            put_rows<V, G, R>(b, psi, gl, n);
            g.sync();
            spmv_rows<V, G, R>(M, b, K[0], gl, n);
            ++n_rhs;
            rejected_before = false;
            continue;
        }

        for (; j < a.n_t && a.t[j] <= t_new; ++j) {
            double thj = (a.t[j] - t) / h;
            if (thj > 1.0) thj = 1.0;
            cpx<V> yd[R];
            dense_output<V, R>(psi, K, h, thj, yd);
            record_outputs<V, G, R>(a, g, si, sv, xb, yd, j, out);
        }
        double fac = (err == 0.0) ? kFacMax : kSafety * pow(err, -0.2);
        if (fac > kFacMax) fac = kFacMax;
        if (fac < kFacMin) fac = kFacMin;
        if (rejected_before && fac > 1.0) fac = 1.0;
        rejected_before = false;
        t = t_new;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            psi[r] = yn[r];
            K[0][r] = K[6][r];
        }
        h *= fac;
    }

    if (gl == 0) {
        if (status != 0) {
            for (; j < a.n_t; ++j)
                for (int q = 0; q < a.n_obs; ++q) out[(size_t)j * a.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
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

template <class V, int G, int R, int BLOCK>
__global__ void __launch_bounds__(BLOCK) mcwf_kernel(const __grid_constant__ KernelArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int *si = reinterpret_cast<int *>(smem);
    cpx<V> *sv = reinterpret_cast<cpx<V> *>(smem + a.smem_vals_offset);
    for (int i = threadIdx.x; i < a.n_ints; i += BLOCK) si[i] = a.ints[i];
    const cpx<V> *gv = static_cast<const cpx<V> *>(a.vals);
    for (int i = threadIdx.x; i < a.n_vals; i += BLOCK) sv[i] = gv[i];
    __syncthreads();

    const Group<G> g(threadIdx.x & 31);
    XBuf<V> xb{reinterpret_cast<cpx<V> *>(smem + a.smem_ybuf_offset) + (threadIdx.x / G) * 2 * (G * R),
               G * R, 0};
    for (;;) {
        unsigned long long i = 0;
        if (g.gl == 0) i = atomicAdd(a.queue, 1ULL);
        i = g.bcast0(i);
        if ((long long)i >= a.ntraj) break;
        run_trajectory<V, G, R>(a, g, si, sv, xb, (long long)i);
    }
}

// Shared-memory layout and occupancy-sized persistent launch of one instantiation.
template <class V, int G, int R>
cudaError_t launch_instance(const KernelArgs &a0, cudaStream_t stream, LaunchInfo *info)
{
    constexpr int BLOCK = 128;
    KernelArgs a = a0;
    auto al16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t ib = al16((size_t)a.n_ints * sizeof(int));
    const size_t vb = al16((size_t)a.n_vals * sizeof(cpx<V>));
    a.smem_vals_offset = (int)ib;
    a.smem_ybuf_offset = (int)(ib + vb);
    const size_t smem = ib + vb + (size_t)(BLOCK / G) * 2 * G * R * sizeof(cpx<V>);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = mcwf_kernel<V, G, R, BLOCK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem)) != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    const long long per_cta = BLOCK / G;
    const long long need = (a.ntraj + per_cta - 1) / per_cta;
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
