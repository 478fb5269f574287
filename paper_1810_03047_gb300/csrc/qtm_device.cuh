// qtm_device.cuh -- device building blocks of the trajectory kernels (sm_103a).
//
//  * complex arithmetic on interleaved (re, im) pairs;
//  * Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
//    "Parallel random numbers: as easy as 1, 2, 3", SC'11), replacing the
//    LFSR113 generator of Sec. 2.3 so that the draws of Algorithm 1 are
//    addressable by (seed, trajectory, jump index);
//  * the Dormand-Prince 5(4) tableau (Dormand & Prince 1980) and its 4th-order
//    continuous extension (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.6),
//    the latter re-expanded into monomials theta^1..theta^5 so that the squared
//    norm of the interpolant is a degree-10 polynomial in theta;
//  * reductions over the lanes that share one trajectory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qtm {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------

template <class V> struct cpx;
template <> struct __align__(16) cpx<double> { double re, im; };
template <> struct __align__(8) cpx<float> { float re, im; };

template <class V>
__device__ __forceinline__ cpx<V> czero() { return cpx<V>{V(0), V(0)}; }

// acc + a * b
template <class V>
__device__ __forceinline__ cpx<V> cmac(cpx<V> acc, cpx<V> a, cpx<V> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
    return acc;
}

// acc + s * a for a real scalar s
template <class V>
__device__ __forceinline__ cpx<V> caxpy(cpx<V> acc, V s, cpx<V> a)
{
    acc.re = fma(s, a.re, acc.re);
    acc.im = fma(s, a.im, acc.im);
    return acc;
}

template <class V>
__device__ __forceinline__ V cabs2(cpx<V> a) { return fma(a.re, a.re, a.im * a.im); }

// ---------------------------------------------------------------------------
// Philox4x64-10
// ---------------------------------------------------------------------------

struct Philox4x64 {
    static constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ULL;
    static constexpr uint64_t kMul1 = 0xCA5A826395121157ULL;
    static constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ULL;  // golden ratio
    static constexpr uint64_t kWeyl1 = 0xBB67AE8584CAA73BULL;  // sqrt(3) - 1

    // Ten rounds; key schedule k_i = k_0 + i * Weyl.
    __device__ static void block(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                 uint64_t k1, uint64_t out[4])
    {
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            const uint64_t lo0 = kMul0 * c0, hi0 = __umul64hi(kMul0, c0);
            const uint64_t lo1 = kMul1 * c2, hi1 = __umul64hi(kMul1, c2);
            const uint64_t n0 = hi1 ^ c1 ^ k0;
            const uint64_t n2 = hi0 ^ c3 ^ k1;
            c0 = n0;
            c1 = lo1;
            c2 = n2;
            c3 = lo0;
            k0 += kWeyl0;
            k1 += kWeyl1;
        }
        out[0] = c0;
        out[1] = c1;
        out[2] = c2;
        out[3] = c3;
    }
};

// 53 random bits -> (0, 1), never 0 or 1
__device__ __forceinline__ double open_unit(uint64_t w)
{
    return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

// r_k (norm threshold, Algorithm 1 (A)/(D)) and c_k (channel draw, step (C))
__device__ __forceinline__ void jump_draws(uint64_t seed, long long traj, long long k, double &r,
                                           double &c)
{
    uint64_t w[4];
    Philox4x64::block((uint64_t)k, (uint64_t)traj, 0, 0, seed, 0, w);
    r = open_unit(w[0]);
    c = open_unit(w[1]);
}

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4)
// ---------------------------------------------------------------------------

struct DP5 {
    // stage coupling a_sj (row s uses K_0..K_{s-1}); row 6 is the 5th-order
    // solution (first same as last)
    __host__ __device__ static constexpr double a(int s, int j)
    {
        return s == 1 ? (j == 0 ? 1.0 / 5.0 : 0.0)
             : s == 2 ? (j == 0 ? 3.0 / 40.0 : j == 1 ? 9.0 / 40.0 : 0.0)
             : s == 3 ? (j == 0 ? 44.0 / 45.0 : j == 1 ? -56.0 / 15.0 : j == 2 ? 32.0 / 9.0 : 0.0)
             : s == 4 ? (j == 0 ? 19372.0 / 6561.0 : j == 1 ? -25360.0 / 2187.0
                         : j == 2 ? 64448.0 / 6561.0 : j == 3 ? -212.0 / 729.0 : 0.0)
             : s == 5 ? (j == 0 ? 9017.0 / 3168.0 : j == 1 ? -355.0 / 33.0
                         : j == 2 ? 46732.0 / 5247.0 : j == 3 ? 49.0 / 176.0
                         : j == 4 ? -5103.0 / 18656.0 : 0.0)
             : s == 6 ? b(j)
             : 0.0;
    }
    // 5th-order weights
    __host__ __device__ static constexpr double b(int j)
    {
        return j == 0 ? 35.0 / 384.0 : j == 2 ? 500.0 / 1113.0 : j == 3 ? 125.0 / 192.0
             : j == 4 ? -2187.0 / 6784.0 : j == 5 ? 11.0 / 84.0 : 0.0;
    }
    // nodes: stage s is evaluated at t + c_s h (c_s = sum_j a_sj)
    __host__ __device__ static constexpr double c(int s)
    {
        return s == 1 ? 1.0 / 5.0 : s == 2 ? 3.0 / 10.0 : s == 3 ? 4.0 / 5.0 : s == 4 ? 8.0 / 9.0
             : (s == 5 || s == 6) ? 1.0 : 0.0;
    }
    // embedded 4th-order weights
    __host__ __device__ static constexpr double bhat(int j)
    {
        return j == 0 ? 5179.0 / 57600.0 : j == 2 ? 7571.0 / 16695.0 : j == 3 ? 393.0 / 640.0
             : j == 4 ? -92097.0 / 339200.0 : j == 5 ? 187.0 / 2100.0 : j == 6 ? 1.0 / 40.0 : 0.0;
    }
    // error weights b - bhat (the local error estimate is h sum_j e_j K_j)
    __host__ __device__ static constexpr double e(int j) { return b(j) - bhat(j); }

    // Continuous extension: y(t + theta h) = y + h sum_j w_j(theta) K_j with
    //   w_j(theta) = theta^2 (3 - 2 theta) b_j + theta^2 (theta - 1)^2 g_j (beta_j - gamma_j theta)
    // plus theta (theta - 1)^2 for j = 0 and theta^2 (theta - 1) for j = 6, where
    // (g_j, beta_j, gamma_j) are the published constants of the DOPRI5 dense output.
    __host__ __device__ static constexpr double dg(int j)
    {
        return j == 0 ? -5.0 / 11282082432.0 : j == 2 ? 100.0 / 32700410799.0
             : j == 3 ? -25.0 / 1880347072.0 : j == 4 ? 32805.0 / 199316789632.0
             : j == 5 ? -55.0 / 822651844.0 : j == 6 ? 10.0 / 29380423.0 : 0.0;
    }
    __host__ __device__ static constexpr double dbeta(int j)
    {
        return j == 0 ? 2558722523.0 : j == 2 ? 882725551.0 : j == 3 ? 443332067.0
             : j == 4 ? 23143187.0 : j == 5 ? 29972135.0 : j == 6 ? 7414447.0 : 0.0;
    }
    __host__ __device__ static constexpr double dgamma(int j)
    {
        return j == 0 ? 31403016.0 : j == 2 ? 15701508.0 : j == 3 ? 31403016.0
             : j == 4 ? 3489224.0 : j == 5 ? 7076736.0 : j == 6 ? 829305.0 : 0.0;
    }
    // Monomial coefficient W[j][m] of theta^m (m = 1..5) in w_j(theta).  Expanding
    // theta^2 (theta-1)^2 (beta - gamma theta) = -gamma theta^5 + (beta + 2 gamma) theta^4
    //   - (2 beta + gamma) theta^3 + beta theta^2 and theta^2 (3 - 2 theta) = 3 theta^2 - 2 theta^3.
    __host__ __device__ static constexpr double W(int j, int m)
    {
        return m == 1 ? (j == 0 ? 1.0 : 0.0)
             : m == 2 ? 3.0 * b(j) + dg(j) * dbeta(j) + (j == 0 ? -2.0 : j == 6 ? -1.0 : 0.0)
             : m == 3 ? -2.0 * b(j) - dg(j) * (2.0 * dbeta(j) + dgamma(j))
                            + (j == 0 ? 1.0 : j == 6 ? 1.0 : 0.0)
             : m == 4 ? dg(j) * (dbeta(j) + 2.0 * dgamma(j))
             : m == 5 ? -dg(j) * dgamma(j)
             : 0.0;
    }
};

// Step-size controller (Hairer, Norsett & Wanner, Sec. II.4): safety 0.9, growth
// factor in [0.2, 10], exponent 1/5, no growth right after a rejection.
constexpr double kSafety = 0.9;
constexpr double kFacMin = 0.2;
constexpr double kFacMax = 10.0;

// ---------------------------------------------------------------------------
// lanes sharing one trajectory
// ---------------------------------------------------------------------------

// G consecutive threads integrate one trajectory; thread gl of the group owns
// state rows gl, gl + G, gl + 2G, ...  G is a power of two: 1..32 lanes of one
// warp, or 64..256 threads spanning G/32 warps.  Within a warp the group
// synchronises with __syncwarp and reduces with a butterfly of shuffles, which
// leaves the bitwise-identical total in every lane.  A multi-warp group
// synchronises with the named barrier (1 + its index in the CTA) and reduces
// each warp by butterfly, then adds the per-warp totals through a small
// shared-memory scratch in warp order -- again identical in every thread.
template <int G>
struct Group {
    static constexpr bool kMulti = G > 32;
    static constexpr int kWarps = kMulti ? G / 32 : 1;
    unsigned mask;
    int gl;
    int bar;                   // named barrier id (multi-warp groups)
    unsigned long long *scr;   // kWarps + 1 eight-byte slots (multi-warp groups)

    // tid: thread index in the CTA; scratch: the CTA's group scratch area
    __device__ Group(int tid, unsigned long long *scratch)
    {
        if constexpr (kMulti) {
            gl = tid & (G - 1);
            mask = 0xffffffffu;
            bar = 1 + tid / G;
            scr = scratch + (size_t)(tid / G) * (kWarps + 1);
        } else {
            const int lane = tid & 31;
            gl = lane & (G - 1);
            mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
            bar = 0;
            scr = nullptr;
        }
    }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (kMulti)
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(G) : "memory");
        else if (G > 1)
            __syncwarp(mask);
    }
    template <class T>
    __device__ __forceinline__ T sum(T v) const
    {
        constexpr int W = kMulti ? 32 : G;
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, W);
        if constexpr (kMulti) {
            static_assert(sizeof(T) <= 8, "scratch slots hold 8 bytes");
            T *s = reinterpret_cast<T *>(scr);
            if ((gl & 31) == 0) s[gl >> 5] = v;
            sync();
            T t = s[0];
#pragma unroll
            for (int w = 1; w < kWarps; ++w) t += s[w];
            sync();
            return t;
        } else {
            return v;
        }
    }
    template <class T>
    __device__ __forceinline__ T bcast0(T v) const
    {
        if constexpr (kMulti) {
            static_assert(sizeof(T) <= 8, "scratch slots hold 8 bytes");
            T *s = reinterpret_cast<T *>(scr + kWarps);
            if (gl == 0) *s = v;
            sync();
            const T t = *s;
            sync();
            return t;
        } else {
            if (G == 1) return v;
            return __shfl_sync(mask, v, 0, G);
        }
    }
};

}  // namespace qtm
