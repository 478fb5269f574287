// qtm_arith.cuh -- arithmetic policies of the trajectory kernel.
//
// The trajectory kernel is written once; its vector arithmetic (stage products,
// stage combinations, norms, inner products) goes through one of three policies:
//
//   ArF64  complex128 throughout: FP64 state, operators and accumulation.
//   ArDF   "double-float": every real is an unevaluated sum hi + lo of two FP32
//          numbers (|lo| <= ulp(hi)/2, about 48 significant bits).  Products and
//          sums use the error-free transformations TwoProd (FMA based) and
//          TwoSum (Knuth), so the state carries FP64-class precision while
//          every instruction runs on the FP32 pipe -- on GB300 the FP64 pipe has
//          1/63 of the FP32 rate.
//   ArF32  complex64 state and stage products, with double-float accumulation of
//          norms and inner products (the mixed-precision form).
//
// The step-size controller of ArDF/ArF32 runs in FP32 (the error norm only
// decides accept/reject and the next step size), while time, step size and the
// jump-time root find stay in FP64 scalars.
#pragma once

#include "qtm_device.cuh"

namespace qtm {

// ---------------------------------------------------------------------------
// double-float primitives
// ---------------------------------------------------------------------------

struct df {
    float hi, lo;
};

// a + b = s + e exactly (Knuth's TwoSum; no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a * b = p + e exactly (FMA-based TwoProd)
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ df df_renorm(float s, float c)
{
    float h, l;
    two_sum(s, c, h, l);
    return df{h, l};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_renorm(s, e);
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_renorm(p, e);
}

__device__ __forceinline__ df df_from_double(double x)
{
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}

__host__ __device__ constexpr df df_const(double x)
{
    return df{(float)x, (float)(x - (double)(float)x)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// a / b: one FP32 quotient, its exact residual, and a correction quotient
__device__ __forceinline__ df df_div(df a, df b)
{
    const float q1 = a.hi / b.hi;
    float p, e;
    two_prod(q1, b.hi, p, e);
    e = fmaf(q1, b.lo, e);
    float s, t;
    two_sum(a.hi, -p, s, t);
    t += a.lo - e;
    const float q2 = (s + t) / b.hi;
    return df_renorm(q1, q2);
}

// Lazy double-float accumulator: value = s + c, where c collects the exact
// rounding errors of the running sum and the low-order product terms.
struct dacc {
    float s, c;
};

__device__ __forceinline__ void dacc_add_prod(dacc &a, df x, df y)
{
    float p, e;
    two_prod(x.hi, y.hi, p, e);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.c += t + e;
}

// a fresh accumulator holding x y: TwoProd with the cross terms.  Bitwise the
// same as dacc_add_prod into {0, 0} (TwoSum(0, p) = (p, 0) exactly), in 4 FP32
// instructions instead of 12.
__device__ __forceinline__ dacc dacc_prod(df x, df y)
{
    float p, e;
    two_prod(x.hi, y.hi, p, e);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return dacc{p, 0.f + e};
}

__device__ __forceinline__ void dacc_add(dacc &a, df x)
{
    float s, t;
    two_sum(a.s, x.hi, s, t);
    a.s = s;
    a.c += t + x.lo;
}

__device__ __forceinline__ df dacc_get(dacc a) { return df_renorm(a.s, a.c); }

// Group sum of double-float values: every thread ends with the same bits
// (TwoSum's exact error does not depend on operand order and the low parts are
// combined symmetrically; per-warp totals of a multi-warp group are added in
// warp order).
template <int G>
__device__ __forceinline__ df group_sum_df(const Group<G> &g, df v)
{
    constexpr int W = Group<G>::kMulti ? 32 : G;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(g.mask, v.hi, o, W);
        const float ol = __shfl_xor_sync(g.mask, v.lo, o, W);
        float s, e;
        two_sum(v.hi, oh, s, e);
        e += v.lo + ol;
        v = df_renorm(s, e);
    }
    if constexpr (Group<G>::kMulti) {
        df *s = reinterpret_cast<df *>(g.scr);
        if ((g.gl & 31) == 0) s[g.gl >> 5] = v;
        g.sync();
        df t = s[0];
#pragma unroll
        for (int w = 1; w < Group<G>::kWarps; ++w) t = df_add(t, s[w]);
        g.sync();
        return t;
    } else {
        return v;
    }
}

// ---------------------------------------------------------------------------
// complex128 policy
// ---------------------------------------------------------------------------

struct ArF64 {
    static constexpr int kId = 0;
    // Stage and error sums advance the lane's rows together (independent
    // accumulation chains); measured faster than row by row for this arithmetic.
    static constexpr bool kRowChains = true;
    using cplx = cpx<double>;
    using real = double;
    using coef = double;
    struct acc {
        double re, im;
    };
    using red = double;

    __host__ __device__ static constexpr coef cconst(double x) { return x; }
    __device__ static coef coef_of(double x) { return x; }
    __device__ static coef cmul(coef x, coef y) { return x * y; }
    __device__ static coef cadd(coef x, coef y) { return x + y; }
    __device__ static acc zero() { return acc{0.0, 0.0}; }
    __device__ static cplx czero() { return cplx{0.0, 0.0}; }
    __device__ static void mac(acc &a, cplx x, cplx y)
    {
        a.re = fma(x.re, y.re, a.re);
        a.re = fma(-x.im, y.im, a.re);
        a.im = fma(x.re, y.im, a.im);
        a.im = fma(x.im, y.re, a.im);
    }
    __device__ static void axpy(acc &a, coef s, cplx x)
    {
        a.re = fma(s, x.re, a.re);
        a.im = fma(s, x.im, a.im);
    }
    // a += v x and a += i v x for a real matrix entry v
    __device__ static void mac_re(acc &a, real v, cplx x)
    {
        a.re = fma(v, x.re, a.re);
        a.im = fma(v, x.im, a.im);
    }
    __device__ static void mac_im(acc &a, real v, cplx x)
    {
        a.re = fma(-v, x.im, a.re);
        a.im = fma(v, x.re, a.im);
    }
    // a fresh accumulator holding v x (the same value as zero() then mac_re)
    __device__ static acc first_re(real v, cplx x) { return acc{v * x.re, v * x.im}; }
    __device__ static cplx get(const acc &a) { return cplx{a.re, a.im}; }
    // y + h * a
    __device__ static cplx add_scaled(cplx y, coef h, const acc &a)
    {
        return cplx{fma(h, a.re, y.re), fma(h, a.im, y.im)};
    }
    __device__ static red abs2(cplx z) { return fma(z.re, z.re, z.im * z.im); }
    __device__ static red dot_re(cplx a, cplx b) { return a.re * b.re + a.im * b.im; }
    __device__ static red rzero() { return 0.0; }
    __device__ static red radd(red a, red b) { return a + b; }
    __device__ static double rval(red a) { return a; }
    template <int G>
    __device__ static red rsum(const Group<G> &g, red v) { return g.sum(v); }
    __device__ static double re(cplx z) { return z.re; }
    __device__ static double im(cplx z) { return z.im; }
    __device__ static cplx from_double(double re, double im) { return cplx{re, im}; }
    // z / d for a real d > 0, componentwise
    __device__ static cplx div(cplx z, double d) { return cplx{z.re / d, z.im / d}; }

    // Error-norm term |e|^2 / sc^2 of one row, e = h * a
    __device__ static double err_term(const acc &a, double h, cplx y0, cplx y1, double rtol, double atol)
    {
        const double ere = h * a.re, eim = h * a.im;
        const double ay = sqrt(abs2(y0)), an = sqrt(abs2(y1));
        const double sc = atol + rtol * (ay > an ? ay : an);
        return (ere * ere + eim * eim) / (sc * sc);
    }
    using errt = double;
    template <int G>
    __device__ static errt err_sum(const Group<G> &g, errt v) { return g.sum(v); }
    __device__ static double err_final(errt s, int n) { return sqrt(s / n); }
    // growth factor 0.9 err^(-1/5)
    __device__ static double controller(double err) { return kSafety * pow(err, -0.2); }
    // Re<y|A|y> / <y|y>
    __device__ static double ratio(red a, red b) { return a / b; }
    // continuous-extension weights w_j(theta), monomial coefficients W[j][m-1]
    __device__ static void weights(double th, const coef *W, coef (&w)[7])
    {
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const coef *c = W + 5 * j;
            w[j] = ((((c[4] * th + c[3]) * th + c[2]) * th + c[1]) * th + c[0]) * th;
        }
    }
};

// ---------------------------------------------------------------------------
// double-float policy
// ---------------------------------------------------------------------------

struct __align__(16) cdf {
    df re, im;
};

struct ArDF {
    static constexpr int kId = 1;
    // Stage sums row by row (rolled): interleaving the lane's rows into
    // independent chains measured 7 % slower for this arithmetic.
    static constexpr bool kRowChains = false;
    using cplx = cdf;
    using real = df;
    using coef = df;
    struct acc {
        dacc re, im;
    };
    using red = df;

    __host__ __device__ static constexpr coef cconst(double x) { return df_const(x); }
    __device__ static coef coef_of(double x) { return df_from_double(x); }
    __device__ static coef cmul(coef x, coef y) { return df_mul(x, y); }
    __device__ static coef cadd(coef x, coef y) { return df_add(x, y); }
    __device__ static acc zero() { return acc{{0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static cplx czero() { return cplx{{0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static void mac(acc &a, cplx x, cplx y)
    {
        dacc_add_prod(a.re, x.re, y.re);
        dacc_add_prod(a.re, df{-x.im.hi, -x.im.lo}, y.im);
        dacc_add_prod(a.im, x.re, y.im);
        dacc_add_prod(a.im, x.im, y.re);
    }
    __device__ static void axpy(acc &a, coef s, cplx x)
    {
        dacc_add_prod(a.re, s, x.re);
        dacc_add_prod(a.im, s, x.im);
    }
    __device__ static void mac_re(acc &a, real v, cplx x)
    {
        dacc_add_prod(a.re, v, x.re);
        dacc_add_prod(a.im, v, x.im);
    }
    __device__ static void mac_im(acc &a, real v, cplx x)
    {
        dacc_add_prod(a.re, df{-v.hi, -v.lo}, x.im);
        dacc_add_prod(a.im, v, x.re);
    }
    __device__ static acc first_re(real v, cplx x) { return acc{dacc_prod(v, x.re), dacc_prod(v, x.im)}; }
    __device__ static cplx get(const acc &a) { return cplx{dacc_get(a.re), dacc_get(a.im)}; }
    // an accumulator holding y (the Krylov-form sums start from the state)
    __device__ static acc acc_of(cplx y) { return acc{{y.re.hi, y.re.lo}, {y.im.hi, y.im.lo}}; }
    // z 2^k for a power of two s = 2^k (exact)
    __device__ static cplx mul_pow2(cplx z, float s)
    {
        return cplx{{z.re.hi * s, z.re.lo * s}, {z.im.hi * s, z.im.lo * s}};
    }
    // leading FP32 parts (for the error estimate of the Krylov form, which needs no cancellation)
    __device__ static float re32(cplx z) { return z.re.hi; }
    __device__ static float im32(cplx z) { return z.im.hi; }
    __device__ static float coef32(coef c) { return c.hi + c.lo; }
    __device__ static cplx add_scaled(cplx y, coef h, const acc &a)
    {
        dacc r{y.re.hi, y.re.lo}, i{y.im.hi, y.im.lo};
        dacc_add_prod(r, h, dacc_get(a.re));
        dacc_add_prod(i, h, dacc_get(a.im));
        return cplx{dacc_get(r), dacc_get(i)};
    }
    __device__ static red abs2(cplx z)
    {
        dacc a{0.f, 0.f};
        dacc_add_prod(a, z.re, z.re);
        dacc_add_prod(a, z.im, z.im);
        return dacc_get(a);
    }
    __device__ static red dot_re(cplx a, cplx b)
    {
        dacc s{0.f, 0.f};
        dacc_add_prod(s, a.re, b.re);
        dacc_add_prod(s, a.im, b.im);
        return dacc_get(s);
    }
    __device__ static red rzero() { return df{0.f, 0.f}; }
    __device__ static red radd(red a, red b) { return df_add(a, b); }
    __device__ static double rval(red a) { return df_to_double(a); }
    template <int G>
    __device__ static red rsum(const Group<G> &g, red v) { return group_sum_df(g, v); }
    __device__ static double re(cplx z) { return df_to_double(z.re); }
    __device__ static double im(cplx z) { return df_to_double(z.im); }
    __device__ static cplx from_double(double re, double im) { return cplx{df_from_double(re), df_from_double(im)}; }
    __device__ static cplx div(cplx z, double d)
    {
        const df inv = df_from_double(1.0 / d);
        return cplx{df_mul(z.re, inv), df_mul(z.im, inv)};
    }

    // |e|^2 / sc^2 in FP32: e = h * a is already accurate to FP64 class (the
    // accumulator cancelled the nearly equal stage terms exactly); the scale only
    // needs FP32 accuracy.
    __device__ static float err_term(const acc &a, double h, cplx y0, cplx y1, double rtol, double atol)
    {
        const float hf = (float)h;
        const float ere = hf * (a.re.s + a.re.c), eim = hf * (a.im.s + a.im.c);
        const float ay2 = y0.re.hi * y0.re.hi + y0.im.hi * y0.im.hi;
        const float an2 = y1.re.hi * y1.re.hi + y1.im.hi * y1.im.hi;
        const float sc = (float)atol + (float)rtol * sqrtf(ay2 > an2 ? ay2 : an2);
        return (ere * ere + eim * eim) / (sc * sc);
    }
    using errt = float;
    template <int G>
    __device__ static errt err_sum(const Group<G> &g, errt v) { return g.sum(v); }
    __device__ static double err_final(errt s, int n) { return (double)sqrtf(s / (float)n); }
    __device__ static double controller(double err) { return (double)(0.9f * __powf((float)err, -0.2f)); }
    __device__ static double ratio(red a, red b) { return df_to_double(df_div(a, b)); }
    __device__ static void weights(double th, const coef *W, coef (&w)[7])
    {
        const df t = df_from_double(th);
#pragma unroll 1
        for (int j = 0; j < 7; ++j) {
            const coef *c = W + 5 * j;
            df p = c[4];
#pragma unroll 1
            for (int m = 3; m >= 0; --m) p = df_add(df_mul(p, t), c[m]);
            w[j] = df_mul(p, t);
        }
    }
};

// ---------------------------------------------------------------------------
// complex64 policy (mixed: FP32 state, double-float norms and inner products)
// ---------------------------------------------------------------------------

struct ArF32 {
    static constexpr int kId = 2;
    // Stage and error sums advance the lane's rows together (independent
    // accumulation chains); measured faster than row by row for this arithmetic.
    static constexpr bool kRowChains = true;
    using cplx = cpx<float>;
    using real = float;
    using coef = float;
    struct acc {
        float re, im;
    };
    using red = df;

    __host__ __device__ static constexpr coef cconst(double x) { return (float)x; }
    __device__ static coef coef_of(double x) { return (float)x; }
    __device__ static coef cmul(coef x, coef y) { return x * y; }
    __device__ static coef cadd(coef x, coef y) { return x + y; }
    __device__ static acc zero() { return acc{0.f, 0.f}; }
    __device__ static cplx czero() { return cplx{0.f, 0.f}; }
    __device__ static void mac(acc &a, cplx x, cplx y)
    {
        a.re = fmaf(x.re, y.re, a.re);
        a.re = fmaf(-x.im, y.im, a.re);
        a.im = fmaf(x.re, y.im, a.im);
        a.im = fmaf(x.im, y.re, a.im);
    }
    __device__ static void axpy(acc &a, coef s, cplx x)
    {
        a.re = fmaf(s, x.re, a.re);
        a.im = fmaf(s, x.im, a.im);
    }
    __device__ static void mac_re(acc &a, real v, cplx x)
    {
        a.re = fmaf(v, x.re, a.re);
        a.im = fmaf(v, x.im, a.im);
    }
    __device__ static void mac_im(acc &a, real v, cplx x)
    {
        a.re = fmaf(-v, x.im, a.re);
        a.im = fmaf(v, x.re, a.im);
    }
    __device__ static acc first_re(real v, cplx x) { return acc{v * x.re, v * x.im}; }
    __device__ static cplx get(const acc &a) { return cplx{a.re, a.im}; }
    __device__ static acc acc_of(cplx y) { return acc{y.re, y.im}; }
    __device__ static cplx mul_pow2(cplx z, float s) { return cplx{z.re * s, z.im * s}; }
    __device__ static float re32(cplx z) { return z.re; }
    __device__ static float im32(cplx z) { return z.im; }
    __device__ static float coef32(coef c) { return c; }
    __device__ static cplx add_scaled(cplx y, coef h, const acc &a)
    {
        return cplx{fmaf(h, a.re, y.re), fmaf(h, a.im, y.im)};
    }
    __device__ static red abs2(cplx z)
    {
        dacc a{0.f, 0.f};
        dacc_add_prod(a, df{z.re, 0.f}, df{z.re, 0.f});
        dacc_add_prod(a, df{z.im, 0.f}, df{z.im, 0.f});
        return dacc_get(a);
    }
    __device__ static red dot_re(cplx a, cplx b)
    {
        dacc s{0.f, 0.f};
        dacc_add_prod(s, df{a.re, 0.f}, df{b.re, 0.f});
        dacc_add_prod(s, df{a.im, 0.f}, df{b.im, 0.f});
        return dacc_get(s);
    }
    __device__ static red rzero() { return df{0.f, 0.f}; }
    __device__ static red radd(red a, red b) { return df_add(a, b); }
    __device__ static double rval(red a) { return df_to_double(a); }
    template <int G>
    __device__ static red rsum(const Group<G> &g, red v) { return group_sum_df(g, v); }
    __device__ static double re(cplx z) { return (double)z.re; }
    __device__ static double im(cplx z) { return (double)z.im; }
    __device__ static cplx from_double(double re, double im) { return cplx{(float)re, (float)im}; }
    __device__ static cplx div(cplx z, double d)
    {
        const float inv = (float)(1.0 / d);
        return cplx{z.re * inv, z.im * inv};
    }
    __device__ static float err_term(const acc &a, double h, cplx y0, cplx y1, double rtol, double atol)
    {
        const float hf = (float)h;
        const float ere = hf * a.re, eim = hf * a.im;
        const float ay2 = y0.re * y0.re + y0.im * y0.im;
        const float an2 = y1.re * y1.re + y1.im * y1.im;
        const float sc = (float)atol + (float)rtol * sqrtf(ay2 > an2 ? ay2 : an2);
        return (ere * ere + eim * eim) / (sc * sc);
    }
    using errt = float;
    template <int G>
    __device__ static errt err_sum(const Group<G> &g, errt v) { return g.sum(v); }
    __device__ static double err_final(errt s, int n) { return (double)sqrtf(s / (float)n); }
    __device__ static double controller(double err) { return (double)(0.9f * __powf((float)err, -0.2f)); }
    __device__ static double ratio(red a, red b) { return df_to_double(df_div(a, b)); }
    __device__ static void weights(double th, const coef *W, coef (&w)[7])
    {
        const float t = (float)th;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const coef *c = W + 5 * j;
            w[j] = ((((c[4] * t + c[3]) * t + c[2]) * t + c[1]) * t + c[0]) * t;
        }
    }
};

}  // namespace qtm
