// moments.h -- exact ensemble sums of bounded observables (host and device).
//
// The ensemble average of Sec. 3 (each node averages its trajectories, the
// master averages the node results) is a sum over trajectories whose value must
// not depend on how the trajectories were split over launches or GPUs.  A sum
// of doubles does: floating-point addition is not associative.  So the library
// sums on a fixed-point grid instead.  Every recorded value of observable k is
// Re<psi|A_k|psi>/<psi|psi>, bounded by ||A_k||_2 <= max_i sum_j |A_ij|; with
// 2^(E_k - 1) above that bound (the scale exponent E_k), each value x is
// truncated to an integer q(x) of quanta 2^(E_k - 100), and the library sums
// q(x) and q(x)^2 as integers.  Integer sums are exact in any order, so the
// totals -- and the mean and the sample variance of the quantised values formed
// from them exactly -- are the same bits for one launch, for any split into
// shards, and for any order in which the shards' totals are added.  The
// truncation moves each value by less than 2^-99 of the observable's bound, far
// below FP64 rounding of the value itself.
//
// Representation ("moment words", kMomentWords int64 per output value):
//   w[0..2]  S1 = sum q(x)    as d0 + d1 2^48 + d2 2^96
//   w[3..7]  S2 = sum q(x)^2  as d0 + d1 2^48 + ... + d4 2^192
//   w[8]     number of values that could not be represented (NaN, Inf or not
//            below 2^E_k: a failed trajectory), which makes the mean NaN
// Digits are signed int64; after normalisation every digit but the last lies in
// [0, 2^48) and the last carries the rest, so up to 2^14 normalised word sets
// add digit by digit without overflow (e.g. in an integer all-reduce across GPUs).
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

constexpr int kMomentWords = 9;
constexpr int kS1 = 0, kS1Digits = 3, kS2 = 3, kS2Digits = 5, kBad = 8;
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

// Digits of trunc(|y|) in base 2^48, for |y| < 2^100 (so d[2] < 2^4).  Every
// operation is exact: scaling by powers of two, floor/trunc, and differences
// whose result has no more significant bits than the operand.
QTM_HD void quanta_digits(double y, unsigned long long d[3])
{
    const double a = trunc(fabs(y));
    const double h2 = floor(a * 0x1p-96);
    const double r = a - h2 * 0x1p96;
    const double h1 = floor(r * 0x1p-48);
    const double h0 = r - h1 * 0x1p48;
    d[0] = (unsigned long long)h0;
    d[1] = (unsigned long long)h1;
    d[2] = (unsigned long long)h2;
}

// Carries so that every digit but the last lies in [0, 2^48) (floor division).
QTM_HD void normalize_digits(long long *d, int count)
{
    const long long base = 1LL << kDigitBits;
    for (int i = 0; i + 1 < count; ++i) {
        const long long c = d[i] >> kDigitBits;  // arithmetic shift: floor for negative digits
        d[i] -= c * base;
        d[i + 1] += c;
    }
}

// d[i] += low 48 bits of v, d[i + 1] += the rest (v < 2^112)
QTM_HD void add_wide(long long *d, int i, unsigned __int128 v)
{
    d[i] += (long long)(unsigned long long)(v & ((1ULL << kDigitBits) - 1));
    d[i + 1] += (long long)(unsigned long long)(v >> kDigitBits);
}

// Per-output-value accumulator of the moment words.
struct MomentAcc {
    long long s1[kS1Digits], s2[kS2Digits], bad;
    int pending;

    QTM_HD void clear()
    {
        for (int i = 0; i < kS1Digits; ++i) s1[i] = 0;
        for (int i = 0; i < kS2Digits; ++i) s2[i] = 0;
        bad = 0;
        pending = 0;
    }
    // adds one value x with scale exponent E (sc = 2^(100 - E), lim = 2^E)
    QTM_HD void add(double x, double sc, double lim)
    {
        if (!(fabs(x) < lim)) {
            ++bad;
            return;
        }
        unsigned long long d[3];
        quanta_digits(x * sc, d);
        if (x < 0.0) {
            s1[0] -= (long long)d[0];
            s1[1] -= (long long)d[1];
            s1[2] -= (long long)d[2];
        } else {
            s1[0] += (long long)d[0];
            s1[1] += (long long)d[1];
            s1[2] += (long long)d[2];
        }
        // q^2 = d0^2 + 2 d0 d1 B + (2 d0 d2 + d1^2) B^2 + 2 d1 d2 B^3 + d2^2 B^4, B = 2^48
        using u128 = unsigned __int128;
        add_wide(s2, 0, (u128)d[0] * d[0]);
        add_wide(s2, 1, (u128)(2 * d[0]) * d[1]);
        add_wide(s2, 2, (u128)(2 * d[0]) * d[2] + (u128)d[1] * d[1]);
        add_wide(s2, 3, (u128)(2 * d[1]) * d[2]);
        s2[4] += (long long)(d[2] * d[2]);
        if (++pending == kNormalizeEvery) normalize();
    }
    QTM_HD void normalize()
    {
        normalize_digits(s1, kS1Digits);
        normalize_digits(s2, kS2Digits);
        pending = 0;
    }
    QTM_HD void store(long long *w, long long stride) const
    {
        for (int i = 0; i < kS1Digits; ++i) w[(kS1 + i) * stride] = s1[i];
        for (int i = 0; i < kS2Digits; ++i) w[(kS2 + i) * stride] = s2[i];
        w[kBad * stride] = bad;
    }
};

// Host: mean, standard error (sample variance, n - 1 divisor), sum and sum of
// squares of one output value from its moment words, n values and scale
// exponent E.  Any output pointer may be NULL.  Defined in moments.cpp.
void moments_finish(const long long *w, long long n, int E, double *mean, double *se, double *sum, double *sumsq);

}  // namespace qtm
