// moments.h -- exact ensemble sums of bounded observables (host and device).
//
// The ensemble average of Sec. 3 (each node averages its trajectories, the
// master averages the node results) is a sum over trajectories whose value must
// not depend on how the trajectories were split over launches or GPUs.  A sum
// of doubles does: floating-point addition is not associative.  So the library
// sums on a fixed-point grid instead.  Every recorded value of observable k is
// Re<psi|A_k|psi>/<psi|psi>, bounded by ||A_k||_2 <= max_i sum_j |A_ij|; with
// 2^(E_k - 1) above that bound (the scale exponent E_k), each value x is
// truncated to an integer number of quanta 2^(E_k - 100), and x^2 (formed
// exactly as p + e by an FMA) to quanta 2^(2 E_k - 100).  Integers add exactly
// in any order, so the totals -- and the mean and standard error computed from
// them -- are the same bits for one launch, for any split into shards, and for
// any order in which the shards' totals are added.  The truncation moves each
// value by less than 2^-99 of the observable's bound, far below FP64 rounding
// of the value itself.
//
// Representation ("moment words", kMomentWords int64 per output value):
//   w[0..2]  sum of the quanta of x    as d0 + d1 2^48 + d2 2^96
//   w[3..5]  sum of the quanta of x^2  in the same digits
//   w[6]     number of values that could not be represented (NaN, Inf or not
//            below 2^E_k: a failed trajectory), which makes the mean NaN
// Digits are signed int64; after normalize() d0 and d1 lie in [0, 2^48) and
// d2 carries the rest, so up to 2^14 normalised word sets add digit by digit
// without overflow (e.g. in an integer all-reduce across GPUs).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cmath>

#ifdef __CUDACC__
#define QTM_HD __host__ __device__ __forceinline__
#else
#define QTM_HD inline
#endif

namespace qtm {

constexpr int kMomentWords = 7;
constexpr int kQuantBits = 100;    // quanta per value: 2^(E - kQuantBits)
constexpr int kDigitBits = 48;
constexpr int kMinScaleExp = -400;
constexpr int kMaxScaleExp = 400;
constexpr int kNormalizeEvery = 1024;  // values added between two normalisations

// 2^k as a double for k in [-1022, 1023] (built from its bits: exact)
QTM_HD double pow2(int k)
{
    const unsigned long long bits = (unsigned long long)(k + 1023) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
#endif
}

// Scale exponent of an observable whose values are bounded by `bound` in
// magnitude: the smallest power of two above twice the bound (head-room for the
// rounding of a value computed next to the bound), clamped to a range where
// every scaling below stays a normal double.
inline int scale_exponent(double bound)
{
    if (!(bound > 0.0)) return kMinScaleExp;
    int e = std::ilogb(bound) + 2;  // 2^(ilogb + 1) > bound
    if (e < kMinScaleExp) e = kMinScaleExp;
    if (e > kMaxScaleExp) e = kMaxScaleExp;
    return e;
}

// d += sign(y) trunc(|y|) in digits, for |y| < 2^100.  Every operation is exact:
// scaling by powers of two, floor/trunc, and differences whose result has no
// more significant bits than the operand.
QTM_HD void add_quanta(long long d[3], double y)
{
    const double a = trunc(fabs(y));
    const double h2 = floor(a * 0x1p-96);
    const double r = a - h2 * 0x1p96;
    const double h1 = floor(r * 0x1p-48);
    const double h0 = r - h1 * 0x1p48;
    if (y < 0.0) {
        d[0] -= (long long)h0;
        d[1] -= (long long)h1;
        d[2] -= (long long)h2;
    } else {
        d[0] += (long long)h0;
        d[1] += (long long)h1;
        d[2] += (long long)h2;
    }
}

// Carries so that d[0], d[1] lie in [0, 2^48) (floor division by 2^48).
QTM_HD void normalize_digits(long long d[3])
{
    const long long base = 1LL << kDigitBits;
    long long c = d[0] >> kDigitBits;  // arithmetic shift: floor for negative digits
    d[0] -= c * base;
    d[1] += c;
    c = d[1] >> kDigitBits;
    d[1] -= c * base;
    d[2] += c;
}

// Per-output-value accumulator of the moment words.
struct MomentAcc {
    long long s1[3], s2[3], bad;
    int pending;

    QTM_HD void clear()
    {
        s1[0] = s1[1] = s1[2] = 0;
        s2[0] = s2[1] = s2[2] = 0;
        bad = 0;
        pending = 0;
    }
    // adds one value x with scale exponent E (sc1 = 2^(100 - E), sc2 = 2^(100 - 2E), lim = 2^E)
    QTM_HD void add(double x, double sc1, double sc2, double lim)
    {
        if (!(fabs(x) < lim)) {
            ++bad;
            return;
        }
        add_quanta(s1, x * sc1);
        const double p = x * x;
        const double e = fma(x, x, -p);  // x^2 = p + e exactly
        add_quanta(s2, p * sc2);
        add_quanta(s2, e * sc2);
        if (++pending == kNormalizeEvery) normalize();
    }
    QTM_HD void normalize()
    {
        normalize_digits(s1);
        normalize_digits(s2);
        pending = 0;
    }
    QTM_HD void store(long long *w, long long stride) const
    {
        w[0] = s1[0];
        w[stride] = s1[1];
        w[2 * stride] = s1[2];
        w[3 * stride] = s2[0];
        w[4 * stride] = s2[1];
        w[5 * stride] = s2[2];
        w[6 * stride] = bad;
    }
};

// Host: mean, standard error (sample variance, n - 1 divisor), sum and sum of
// squares of one output value from its normalised moment words, n values and
// scale exponent E.  Any output pointer may be NULL.  Defined in moments.cpp.
void moments_finish(const long long *w, long long n, int E, double *mean, double *se, double *sum, double *sumsq);

}  // namespace qtm
