// moments.cpp -- host side of the exact ensemble sums (moments.h): the mean and
// standard error from the integer totals, the same totals from host values, and
// the combination of shards (the master's average of the node averages, Sec. 3).
//
// Compiled without floating-point contraction, so every operation here rounds
// as written and the results are the same bits on every host architecture.

#include <climits>
#include <cmath>
#include <cstdint>

#include "../../include/qtm.h"
#include "moments.h"
#include "qtm_launch.h"

namespace {

// Signed integer of 6 x 64 bits (sign and magnitude), enough for the exact
// variance numerator n S2 - S1^2 (below 2^282 for up to 2^40 values).
struct Big {
    bool neg = false;
    uint64_t m[6] = {0, 0, 0, 0, 0, 0};
};

using u128 = unsigned __int128;

int cmp_mag(const Big &a, const Big &b)
{
    for (int i = 5; i >= 0; --i)
        if (a.m[i] != b.m[i]) return a.m[i] < b.m[i] ? -1 : 1;
    return 0;
}

bool is_zero(const Big &a)
{
    for (int i = 0; i < 6; ++i)
        if (a.m[i]) return false;
    return true;
}

Big add_mag(const Big &a, const Big &b)
{
    Big r;
    u128 c = 0;
    for (int i = 0; i < 6; ++i) {
        c += (u128)a.m[i] + b.m[i];
        r.m[i] = (uint64_t)c;
        c >>= 64;
    }
    return r;
}

// |a| - |b| for |a| >= |b|
Big sub_mag(const Big &a, const Big &b)
{
    Big r;
    uint64_t borrow = 0;
    for (int i = 0; i < 6; ++i) {
        const uint64_t x = a.m[i], y = b.m[i];
        const uint64_t d = x - y - borrow;
        borrow = (x < y || (x == y && borrow)) ? 1 : 0;
        r.m[i] = d;
    }
    return r;
}

Big add(const Big &a, const Big &b)
{
    Big r;
    if (a.neg == b.neg) {
        r = add_mag(a, b);
        r.neg = a.neg;
    } else if (cmp_mag(a, b) >= 0) {
        r = sub_mag(a, b);
        r.neg = a.neg;
    } else {
        r = sub_mag(b, a);
        r.neg = b.neg;
    }
    if (is_zero(r)) r.neg = false;
    return r;
}

Big negate(Big a)
{
    if (!is_zero(a)) a.neg = !a.neg;
    return a;
}

Big from_i64(long long v)
{
    Big r;
    r.neg = v < 0;
    r.m[0] = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    return r;
}

Big shl(const Big &a, int bits)
{
    Big r;
    r.neg = a.neg;
    const int q = bits / 64, s = bits % 64;
    for (int i = 5; i >= 0; --i) {
        const int src = i - q;
        if (src < 0) continue;
        uint64_t v = a.m[src] << s;
        if (s && src > 0) v |= a.m[src - 1] >> (64 - s);
        r.m[i] = v;
    }
    return r;
}

// product, truncated to 6 limbs (callers stay below 2^384)
Big mul(const Big &a, const Big &b)
{
    Big r;
    for (int i = 0; i < 6; ++i) {
        if (!a.m[i]) continue;
        u128 c = 0;
        for (int j = 0; i + j < 6; ++j) {
            c += (u128)a.m[i] * b.m[j] + r.m[i + j];
            r.m[i + j] = (uint64_t)c;
            c >>= 64;
        }
    }
    r.neg = a.neg != b.neg;
    if (is_zero(r)) r.neg = false;
    return r;
}

// sum_i d[i] 2^(48 i)
Big from_digits(const long long *d, int count)
{
    Big r;
    for (int i = 0; i < count; ++i) r = add(r, shl(from_i64(d[i]), i * qtm::kDigitBits));
    return r;
}

// Round to nearest double: the top 64 bits, with any lower set bit folded into
// bit 0 (a sticky bit 11 places below the rounding position), converted once.
double to_double(const Big &a)
{
    int top = -1;
    for (int i = 5; i >= 0; --i)
        if (a.m[i]) {
            top = i;
            break;
        }
    if (top < 0) return 0.0;
    const int hb = 63 - __builtin_clzll(a.m[top]);
    const int len = 64 * top + hb + 1;  // bit length
    uint64_t u;
    int shift = 0;
    if (len <= 64) {
        u = a.m[0];
    } else {
        shift = len - 64;
        const int q = shift / 64, s = shift % 64;
        u = a.m[q] >> s;
        if (s && q + 1 < 6) u |= a.m[q + 1] << (64 - s);
        bool sticky = s ? (a.m[q] & ((1ULL << s) - 1)) != 0 : false;
        for (int i = 0; i < q && !sticky; ++i) sticky = a.m[i] != 0;
        if (sticky) u |= 1;
    }
    const double d = std::ldexp((double)u, shift);
    return a.neg ? -d : d;
}

}  // namespace

namespace qtm {

void moments_finish(const long long *w, long long n, int E, double *mean, double *se, double *sum, double *sumsq)
{
    if (w[kBad] > 0) {
        const double nan = std::nan("");
        if (mean) *mean = nan;
        if (se) *se = nan;
        if (sum) *sum = nan;
        if (sumsq) *sumsq = nan;
        return;
    }
    const Big S1 = from_digits(w + kS1, kS1Digits);  // quanta 2^(E - 100)
    const Big S2 = from_digits(w + kS2, kS2Digits);  // quanta 2^(2E - 200)
    const double s1 = std::ldexp(to_double(S1), E - kQuantBits);
    if (sum) *sum = s1;
    if (sumsq) *sumsq = std::ldexp(to_double(S2), 2 * (E - kQuantBits));
    if (mean) *mean = n > 0 ? s1 / (double)n : 0.0;
    if (!se) return;
    if (n < 2) {
        *se = 0.0;
        return;
    }
    // n sum q^2 - (sum q)^2 = n (n - 1) times the sample variance of the q, exact (quanta 2^(2E - 200))
    const Big D = add(mul(S2, from_i64(n)), negate(mul(S1, S1)));
    if (D.neg || is_zero(D)) {
        *se = 0.0;
        return;
    }
    const double num = std::ldexp(to_double(D), 2 * (E - kQuantBits));
    const double den = (double)n * (double)n * (double)(n - 1);
    *se = std::sqrt(num / den);
}

}  // namespace qtm

extern "C" {

qtm_status qtm_moments_of_values(const double *values, int64_t ntraj, int32_t n_values, int32_t n_obs,
                                 const int32_t *scale_exp, int64_t *words)
{
    if (ntraj < 0 || n_values < 0 || n_obs < 1 || (n_values % n_obs) != 0) {
        qtm::set_last_error("qtm_moments_of_values: need ntraj >= 0, n_obs >= 1, n_values a multiple of n_obs");
        return QTM_ERR_ARG;
    }
    if ((ntraj > 0 && n_values > 0 && !values) || !scale_exp || (n_values > 0 && !words)) {
        qtm::set_last_error("qtm_moments_of_values: NULL buffer");
        return QTM_ERR_ARG;
    }
    for (int k = 0; k < n_obs; ++k)
        if (scale_exp[k] < qtm::kMinScaleExp || scale_exp[k] > qtm::kMaxScaleExp) {
            qtm::set_last_error("qtm_moments_of_values: scale exponent out of range");
            return QTM_ERR_ARG;
        }
    for (int p = 0; p < n_values; ++p) {
        const int E = scale_exp[p % n_obs];
        const double sc = qtm::pow2(qtm::kQuantBits - E), lim = qtm::pow2(E);
        qtm::MomentAcc acc;
        acc.clear();
        for (int64_t i = 0; i < ntraj; ++i) acc.add(values[(size_t)i * n_values + p], sc, lim);
        acc.normalize();
        acc.store(reinterpret_cast<long long *>(words) + (size_t)p * qtm::kMomentWords, 1);
    }
    return QTM_OK;
}

qtm_status qtm_combine_moments(int32_t n_shards, int32_t n_values, int32_t n_obs, const int32_t *scale_exp,
                               const int64_t *words, const int64_t *counts, double *mean, double *stderr_out,
                               double *sum, double *sumsq)
{
    if (n_shards < 1 || n_shards > (1 << 14) || n_values < 0 || n_obs < 1 || (n_values % n_obs) != 0) {
        qtm::set_last_error("qtm_combine_moments: need 1 <= n_shards <= 16384, n_obs >= 1, "
                            "n_values a multiple of n_obs");
        return QTM_ERR_ARG;
    }
    if (!scale_exp || !counts || (n_values > 0 && (!words || !mean))) {
        qtm::set_last_error("qtm_combine_moments: NULL buffer");
        return QTM_ERR_ARG;
    }
    long long n = 0;
    for (int r = 0; r < n_shards; ++r) {
        if (counts[r] < 0 || counts[r] > ((int64_t)1 << 40) - n) {
            qtm::set_last_error("qtm_combine_moments: counts must be >= 0 and total at most 2^40");
            return QTM_ERR_ARG;
        }
        n += counts[r];
    }
    for (int k = 0; k < n_obs; ++k)
        if (scale_exp[k] < qtm::kMinScaleExp || scale_exp[k] > qtm::kMaxScaleExp) {
            qtm::set_last_error("qtm_combine_moments: scale exponent out of range");
            return QTM_ERR_ARG;
        }
    const size_t W = qtm::kMomentWords;
    for (int p = 0; p < n_values; ++p) {
        long long w[qtm::kMomentWords] = {};
        // shards in rank order; integer digits, so the order does not change the result
        for (int r = 0; r < n_shards; ++r) {
            const int64_t *s = words + ((size_t)r * n_values + p) * W;
            for (size_t q = 0; q < W; ++q) w[q] += s[q];
            qtm::normalize_digits(w + qtm::kS1, qtm::kS1Digits);
            qtm::normalize_digits(w + qtm::kS2, qtm::kS2Digits);
        }
        qtm::moments_finish(w, n, scale_exp[p % n_obs], mean + p, stderr_out ? stderr_out + p : nullptr,
                            sum ? sum + p : nullptr, sumsq ? sumsq + p : nullptr);
    }
    return QTM_OK;
}

}  // extern "C"
