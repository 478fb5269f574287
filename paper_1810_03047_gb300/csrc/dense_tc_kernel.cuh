// dense_tc_kernel.cuh -- Algorithm 1 (Sec. 2.2) for dense operators with the stage
// products on the tensor cores (the kernel template; one translation unit per
// padded dimension instantiates it, mcwf_dense_tc_<NP>.cu).
//
// One persistent CTA per SM owns 128 trajectory columns and keeps them busy for
// the whole launch (a finished column takes the next trajectory id from the
// device counter).  The columns advance in lock step, one Dormand-Prince attempt
// at a time, each column with its own t and h.  The step is taken in its Krylov
// form (mcwf_kernel.cuh, run_trajectory_krylov): with a constant M every stage is
// a polynomial in hM applied to psi, so an attempt needs the vectors
// wt_k = (2^-e M)^k psi, k <= 7, and nothing else:
//
//   for s = 1..7:  wt_s = 2^-e M wt_{s-1}, wt_0 = psi       (tcgen05, BF16x6 -> FP32;
//                                                            producers only split wt_{s-1})
//   control:       ynew = psi + sum_k beta_k H^k wt_k, the error estimate
//                  sum_k gamma_k H^k wt_k (H = h 2^e), accept/reject, outputs from
//                  the continuous extension, crossing root find, jump, refill
//                  (one warp per column)
//
// wt_1 is formed by a product every attempt (seven products, the stage form's six
// plus one): carried over from the last step by a combination instead, as the
// double-float SIMT kernel does, its FP32 rounding would drift from step to step
// (measured: median jump-time error 2.9e-5 against the oracle instead of < 1e-5).
//
// The product is D[col][i] = sum_k Y[col][k] Mr[i][k] with the real form
// Mr = [[Re M, -Im M], [Im M, Re M]] (2N x 2N) and Y = (Re y, Im y): M = 128 columns,
// N = 2N outputs (one or two MMAs of up to 256), K = 2N in k-blocks of 64.  Both
// operands are split into three bf16 terms, x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1): 24 significant bits, an FP32 value
// exactly), and the six products of combined order <= 2 (Y0M0, Y1M0, Y2M0, Y0M1,
// Y1M1, Y0M2) are accumulated in FP32: the dropped terms are of relative size
// 2^-24, so the product is as accurate as an FP32 one.  (Two terms and three
// products leave 2^-16, far above the 1e-8 tolerances, and the step-size control
// then shrinks the steps to chase the product's noise.)  Each k-block of the
// input wt_s is read once from device memory, split, and written straight into
// the 128-byte-swizzled K-major layout the tensor core reads (the operator's
// splits are scaled by 2^-e on the host, exactly); the operator's splits stream in by TMA, one 256-row
// chunk of one split per ring entry (three-deep ring, L2-resident).  The FP32
// accumulators (128 lanes x 2N columns) sit in tensor memory until the epilogue
// warps move them to wt_{s+1} in device memory.
//
// Warp roles (320 threads): warp 0 TMA, warp 1 tensor-memory owner and MMA
// issuer, warps 2..9 producers, epilogue and per-column control.  Every mbarrier
// wait is bounded; a timeout sets the launch's error status (8) and the CTA
// winds down, freeing its tensor memory.
#pragma once

#include <cuda_bf16.h>

#include "dense_tc.h"
#include "mcwf_kernel.cuh"
#include "tc_ptx.cuh"

namespace qtm {
namespace {

constexpr int kThreadsTc = 320;
constexpr int kProducers = 256;
constexpr int kKB = 64;               // k-block: 64 bf16 = one 128-byte row
constexpr int kYTile = 128 * 128;     // bytes of one bf16 Y tile (128 rows x 128 B)
constexpr int kCoefFloats = 50;  // KCoefs<ArF32>: beta[7], Q[5][8], gamma[3]
constexpr int kStatusTimeout = 8;  // QTM_ERR_TIMEOUT
constexpr int kSplits = 3;         // bf16 terms per operand
constexpr int kOpRing = 3;         // operator ring entries
constexpr unsigned kTmemCols = 512;

template <int NP>
struct TcShape {
    static constexpr int KD = 2 * NP;          // real dimension: GEMM K and N
    static constexpr int NKB = KD / kKB;       // k-blocks per product
    static constexpr int NCHUNK = (KD + 255) / 256;  // 256-row output chunks (one MMA each)
    static constexpr int OP_ENTRY = 256 * 128;       // bytes of one ring entry: a chunk of one split
    static constexpr int HALF = KD / 2;        // epilogue columns per warp half
    static constexpr int OFF_OP = 0;
    static constexpr int OFF_Y = OFF_OP + kOpRing * OP_ENTRY;
    static constexpr int OFF_SCR = OFF_Y + 2 * kSplits * kYTile;
    static constexpr int OFF_HF = OFF_SCR + 8 * KD * 4;
    static constexpr int OFF_SEL = OFF_HF + 128 * 4;
    static constexpr int OFF_COEF = OFF_SEL + 128 * 4;
    static constexpr int OFF_BAR = OFF_COEF + ((kCoefFloats * 4 + 63) / 64) * 64;
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;
    static constexpr int BYTES = OFF_MISC + 64 + 1024;  // + alignment slack of the dynamic base
    static_assert(NP % 64 == 0 && NP <= kTcMaxDim, "padded dimension");
    static_assert(HALF % 16 == 0, "epilogue loads 16 columns at a time");
};

// The coefficient table is the Krylov form's KCoefs<ArF32> (beta, Q, gamma).
__device__ __forceinline__ const KCoefs<ArF32> &kcoefs(const float *cf)
{
    return *reinterpret_cast<const KCoefs<ArF32> *>(cf);
}
// State-vector index of wt_k (k = 1..7): the seven slots after the two psi buffers
__device__ __forceinline__ int wvec(int k) { return kVK0 + k - 1; }

struct Ctl {
    const DenseArgs *a;
    int col;       // global column index
    int np, kd;
    __device__ __forceinline__ float *vec(int v) const
    {
        return a->state + ((size_t)v * a->cols + col) * kd;
    }
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// Three-term bf16 split of four FP32 values: t0 = bf16(y), t1 = bf16(y - t0),
// t2 = bf16(y - t0 - t1) (the differences are exact in FP32); two values per
// conversion.
__device__ __forceinline__ void split4(float4 y, uint2 (&t)[kSplits])
{
    float2 a = make_float2(y.x, y.y), b = make_float2(y.z, y.w);
#pragma unroll
    for (int q = 0; q < kSplits; ++q) {
        const __nv_bfloat162 ha = __float22bfloat162_rn(a), hb = __float22bfloat162_rn(b);
        t[q].x = *reinterpret_cast<const uint32_t *>(&ha);
        t[q].y = *reinterpret_cast<const uint32_t *>(&hb);
        if (q + 1 < kSplits) {
            const float2 fa = __bfloat1622float2(ha), fb = __bfloat1622float2(hb);
            a.x -= fa.x;
            a.y -= fa.y;
            b.x -= fb.x;
            b.y -= fb.y;
        }
    }
}

// ---------------------------------------------------------------------------
// One product K_s = M Y_s for the CTA's 128 columns (s = 0 in rhs mode: Y = input)
// ---------------------------------------------------------------------------

struct Pipe {
    unsigned char *op, *yt;
    uint64_t *op_full, *op_empty, *y_full, *y_empty, *acc_full;
    volatile int *abort;
    unsigned long long limit;   // wall-clock bound of one wait (ns)
    uint32_t tmem;
    uint32_t ocnt, ycnt, acnt;  // ring positions (every role advances its own copy identically)
};

__device__ __forceinline__ void raise_abort(const DenseArgs &a, Pipe &p)
{
    *p.abort = 1;
    atomicCAS(a.k.first_error, 0, kStatusTimeout);
}

// The roles of one product over the output chunks [c_lo, c_hi) (256 outputs
// each; all of them except for the halves of a batched product's last wave)
template <int NP>
__device__ void role_tma(const DenseArgs &a, Pipe &p, const CUtensorMap *map, int c_lo, int c_hi)
{
    using S = TcShape<NP>;
    for (int kb = 0; kb < S::NKB; ++kb)
        for (int split = 0; split < kSplits; ++split)
            for (int c = c_lo; c < c_hi; ++c) {
                const uint32_t slot = p.ocnt % kOpRing, ph = (p.ocnt / kOpRing) & 1;
                if (!tc::mbar_wait(&p.op_empty[slot], ph ^ 1, p.abort, p.limit)) {
                    raise_abort(a, p);
                    return;
                }
                const int rows = (S::KD - 256 * c) < 256 ? (S::KD - 256 * c) : 256;
                tc::mbar_arrive_expect_tx(&p.op_full[slot], rows * 128);
                unsigned char *dst = p.op + slot * S::OP_ENTRY;
#pragma unroll 1
                for (int q = 0; q < rows / 128; ++q)
                    tc::tma_load_2d(dst + q * 128 * 128, map, &p.op_full[slot], kb * kKB,
                                    split * S::KD + 256 * c + q * 128);
                ++p.ocnt;
            }
}

template <int NP>
__device__ void role_mma(const DenseArgs &a, Pipe &p, int c_lo, int c_hi)
{
    using S = TcShape<NP>;
    for (int kb = 0; kb < S::NKB; ++kb) {
        const uint32_t ys = p.ycnt & 1, yph = (p.ycnt >> 1) & 1;
        if (!tc::mbar_wait(&p.y_full[ys], yph, p.abort, p.limit)) {
            raise_abort(a, p);
            return;
        }
        tc::tc_fence_after();
        const uint32_t ybase = tc::smem_u32(p.yt + ys * kSplits * kYTile);
        for (int split = 0; split < kSplits; ++split)
            for (int c = c_lo; c < c_hi; ++c) {
                const uint32_t os = p.ocnt % kOpRing, oph = (p.ocnt / kOpRing) & 1;
                if (!tc::mbar_wait(&p.op_full[os], oph, p.abort, p.limit)) {
                    raise_abort(a, p);
                    return;
                }
                tc::tc_fence_after();
                const uint32_t ob = tc::smem_u32(p.op + os * S::OP_ENTRY);
                const int n = (S::KD - 256 * c) < 256 ? (S::KD - 256 * c) : 256;
                const uint32_t idesc = tc::idesc_bf16_f32(128, n);
                const uint32_t d = p.tmem + 256 * c;
#pragma unroll
                for (int k16 = 0; k16 < 4; ++k16) {
                    const uint64_t bdesc = tc::desc_sw128(ob + 32 * k16);
                    // Y terms t with t + split <= 2
                    for (int t = 0; t + split < kSplits; ++t) {
                        const uint64_t adesc = tc::desc_sw128(ybase + t * kYTile + 32 * k16);
                        tc::mma_bf16(d, adesc, bdesc, idesc, (kb | split | k16 | t) != 0);
                    }
                }
                tc::mma_commit(&p.op_empty[os]);
                ++p.ocnt;
            }
        tc::mma_commit(&p.y_empty[ys]);
        ++p.ycnt;
    }
    tc::mma_commit(p.acc_full);
}

// The eight rows of the tile a producer thread forms: their source rows in device
// memory for product s (0: the rhs-mode input; else wt_{s-1} of the column, wt_0 =
// psi), nullptr for an idle column or a row past the rhs-mode input (zero).
template <int NP>
__device__ __forceinline__ void producer_rows(const DenseArgs &a, int s, long long tile_base, int pw, int lane,
                                              const float *s_hf, const int *s_sel, const float *(&src)[8])
{
    constexpr int KD = 2 * NP;
    const size_t vs = (size_t)a.cols * KD;  // distance between the vectors of a column
    const int kk = (lane & 15) * 4;         // this thread's 4 values within a 64-wide k-block
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int row = 16 * pw + 2 * it + (lane >> 4);
        const float *p = nullptr;
        if (a.mode == kDenseRhs) {
            const long long g = tile_base + row;
            if (g < a.rhs_n) p = a.rhs_in + g * KD + kk;
        } else if (s_hf[row] != 0.f) {
            const int v = s == 1 ? (s_sel[row] & 1) : kVK0 + s - 2;  // psi, or wt_{s-1}
            p = a.state + (size_t)(tile_base + row) * KD + kk + v * vs;
        }
        src[it] = p;
    }
}

// This thread's eight values of k-block kb (four consecutive k each)
__device__ __forceinline__ void producer_load(const float *const (&src)[8], int kb, float4 (&y)[8])
{
#pragma unroll
    for (int it = 0; it < 8; ++it) y[it] = src[it] ? ld4(src[it] + kb * kKB) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ... split into three bf16 terms and stored into the swizzled tiles
__device__ __forceinline__ void producer_store(const float4 (&y)[8], int pw, int lane, unsigned char *ytile)
{
    const int chunk = ((lane & 15) * 4) >> 3, half8 = ((lane & 15) * 4) & 7;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int row = 16 * pw + 2 * it + (lane >> 4);
        uint2 t[kSplits];
        split4(y[it], t);
        const int off = row * 128 + ((chunk ^ (row & 7)) << 4) + half8 * 2;
#pragma unroll
        for (int q = 0; q < kSplits; ++q) *reinterpret_cast<uint2 *>(ytile + q * kYTile + off) = t[q];
    }
}

// Producer warps: k-blocks of the product's input for the tile, then the
// epilogue.  The loads of k-block kb + 1 are issued before the wait for a free
// tile and the split of k-block kb, so the device-memory latency overlaps the
// ring's turnover instead of starving the tensor cores.
template <int NP>
__device__ void role_producer(const DenseArgs &a, Pipe &p, int s, long long tile_base, int pw, int lane,
                              const float *s_hf, const int *s_sel, const float *cf, int c_lo, int c_hi)
{
    using S = TcShape<NP>;
    const bool rhs = a.mode == kDenseRhs;
    const float *src[8];
    producer_rows<NP>(a, s, tile_base, pw, lane, s_hf, s_sel, src);
    float4 nxt[8];
    producer_load(src, 0, nxt);
    for (int kb = 0; kb < S::NKB; ++kb) {
        float4 cur[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) cur[it] = nxt[it];
        if (kb + 1 < S::NKB) producer_load(src, kb + 1, nxt);
        const uint32_t ys = p.ycnt & 1, yph = (p.ycnt >> 1) & 1;
        if (!tc::mbar_wait(&p.y_empty[ys], yph ^ 1, p.abort, p.limit)) {
            raise_abort(a, p);
            return;
        }
        unsigned char *ytile = p.yt + ys * kSplits * kYTile;
        producer_store(cur, pw, lane, ytile);
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&p.y_full[ys]);
        ++p.ycnt;
    }

    // epilogue: tensor memory -> K_s
    const uint32_t aph = p.acnt & 1;
    ++p.acnt;
    if (!tc::mbar_wait(p.acc_full, aph, p.abort, p.limit)) {
        raise_abort(a, p);
        return;
    }
    tc::tc_fence_after();
    const int warp = pw + 2;
    const int quarter = warp & 3, hsel = pw >> 2;
    const int row = 32 * quarter + lane;
    float *dst = nullptr;
    if (rhs) {
        const long long g = tile_base + row;
        if (g < a.rhs_n) dst = a.rhs_out + g * S::KD;
    } else {
        const Ctl c{&a, (int)(tile_base + row), NP, S::KD};
        dst = c.vec(wvec(s));  // wt_s
    }
    const uint32_t tbase = p.tmem + ((uint32_t)(32 * quarter) << 16);
    // a chunk-split product (NP = 256: chunk c = the outputs of epilogue half c)
    const bool skip = c_hi - c_lo < S::NCHUNK && (hsel < c_lo || hsel >= c_hi);
    // 64 columns per round: four loads in flight, one wait
    static_assert(S::HALF % 64 == 0, "epilogue rounds of 64 columns");
#pragma unroll 1
    for (int cc = hsel * S::HALF; cc < (skip ? hsel * S::HALF : (hsel + 1) * S::HALF); cc += 64) {
        uint32_t v[4][16];
#pragma unroll
        for (int b = 0; b < 4; ++b) tc::tmem_ld16_async(tbase + cc + 16 * b, v[b]);
        tc::tmem_wait_ld();
        if (dst) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    st4(dst + cc + 16 * b + 4 * i,
                        make_float4(__uint_as_float(v[b][4 * i]), __uint_as_float(v[b][4 * i + 1]),
                                    __uint_as_float(v[b][4 * i + 2]), __uint_as_float(v[b][4 * i + 3])));
        }
    }
    tc::tc_fence_before();
}

template <int NP>
__device__ void stage_product(const DenseArgs &a, Pipe &p, const CUtensorMap *map, int s, long long tile_base,
                              const float *s_hf, const int *s_sel, const float *cf, int c_lo = 0,
                              int c_hi = TcShape<NP>::NCHUNK)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane == 0) role_tma<NP>(a, p, map, c_lo, c_hi);
        // keep the lanes' copies of the ring position in step with lane 0
        p.ocnt = __shfl_sync(0xffffffffu, p.ocnt, 0);
    } else if (warp == 1) {
        if (lane == 0) role_mma<NP>(a, p, c_lo, c_hi);
        p.ocnt = __shfl_sync(0xffffffffu, p.ocnt, 0);
        p.ycnt = __shfl_sync(0xffffffffu, p.ycnt, 0);
    } else {
        role_producer<NP>(a, p, s, tile_base, warp - 2, lane, s_hf, s_sel, cf, c_lo, c_hi);
        // K_s is complete in device memory before any producer reads it
        asm volatile("bar.sync 1, %0;" ::"n"(kProducers) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Per-column control (one warp per column)
// ---------------------------------------------------------------------------

using Arc = ArF32;
using cf32 = cpx<float>;

template <int NP>
struct ColCtl {
    static constexpr int R = NP / 32;
    const DenseArgs &a;
    const KernelArgs &k;
    Group<32> g;
    int lane;
    Ctl c;
    float *scr;          // this warp's scratch: NP complex values, interleaved (re, im)
    const float *cf;

    __device__ float re(int v, int m) const { return c.vec(v)[m]; }
    __device__ float im(int v, int m) const { return c.vec(v)[NP + m]; }
    __device__ CsrView<Arc> op(int i) const { return csr_view<Arc>(k.op[i], k.ints, (const float *)k.vals); }
    // 2^-e as a float and H^q = (h 2^e)^q, q = 0..7, for the Krylov coefficients
    __device__ float down() const { return __int_as_float((127 - k.krylov_shift) << 23); }
    __device__ void powers(double h, float (&hp)[8]) const
    {
        const float H = (float)(h * ldexp(1.0, k.krylov_shift));
        hp[0] = 1.f;
#pragma unroll
        for (int q = 1; q < 8; ++q) hp[q] = hp[q - 1] * H;
    }

    // v[r] = (A_i x)[lane + 32 r] for x = scr, every row of the lane at once.
    // Dense operators: column-major FP32 copy, a column's 32 consecutive rows per
    // load (coalesced), x_k broadcast from shared memory, loads independent of one
    // another.  Sparse operators: the SELL-32 parts with the index and value loads
    // of four entries issued before their x loads.
    __device__ __forceinline__ void opmv(int i, cf32 (&v)[R]) const
    {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = cf32{0.f, 0.f};
        const int off = a.dense_off[i];
        if (off <= -2) {  // diagonal: entry m at dense[-2 - off + m]
            const float2 *D = a.dense + (-2 - off);
            const float2 *x = reinterpret_cast<const float2 *>(scr);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                if (m < k.n) {
                    const float2 dm = D[m], xm = x[m];
                    v[r] = cf32{dm.x * xm.x - dm.y * xm.y, dm.x * xm.y + dm.y * xm.x};
                }
            }
            return;
        }
        if (off >= 0) {
            const float2 *D = a.dense + off + lane;
            const float2 *x = reinterpret_cast<const float2 *>(scr);
#pragma unroll 4
            for (int kk = 0; kk < k.n; ++kk) {
                const float2 xk = x[kk];
                const float2 *col = D + (size_t)kk * NP;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 m = col[32 * r];
                    v[r].re = fmaf(m.x, xk.x, fmaf(-m.y, xk.y, v[r].re));
                    v[r].im = fmaf(m.x, xk.y, fmaf(m.y, xk.x, v[r].im));
                }
            }
            return;
        }
        const CsrView<Arc> A = op(i);
        const cf32 *x = reinterpret_cast<const cf32 *>(scr);
        int2 tabs[2][R];  // slice tables of both parts, loaded together
#pragma unroll
        for (int r = 0; r < R; ++r) {
            tabs[0][r] = make_int2(A.tab_re[2 * r], A.tab_re[2 * r + 1]);  // tables need not be 8-byte aligned
            tabs[1][r] = make_int2(A.tab_im[2 * r], A.tab_im[2 * r + 1]);
        }
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const int *cols = part ? A.col_im : A.col_re;
                const float *vals = part ? A.val_im : A.val_re;
                const int o = tabs[part][r].x + lane, w = tabs[part][r].y;
                int t = 0;
                for (; t + 4 <= w; t += 4) {
                    int ci[4];
                    float cv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        ci[u] = cols[o + (t + u) * 32];
                        cv[u] = vals[o + (t + u) * 32];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const cf32 xv = x[ci[u]];
                        if (part == 0) {
                            ar = fmaf(cv[u], xv.re, ar);
                            ai = fmaf(cv[u], xv.im, ai);
                        } else {
                            ar = fmaf(-cv[u], xv.im, ar);
                            ai = fmaf(cv[u], xv.re, ai);
                        }
                    }
                }
                for (; t < w; ++t) {
                    const float cv = vals[o + t * 32];
                    const cf32 xv = x[cols[o + t * 32]];
                    if (part == 0) {
                        ar = fmaf(cv, xv.re, ar);
                        ai = fmaf(cv, xv.im, ai);
                    } else {
                        ar = fmaf(-cv, xv.im, ar);
                        ai = fmaf(cv, xv.re, ai);
                    }
                }
            }
            v[r] = cf32{ar, ai};
        }
    }

    // scr <- psi + sum_k rho_k(theta) H^k wt_k (the continuous extension) for rows < n
    __device__ __forceinline__ void dense_to_scr(const DenseCol &d, double th) const
    {
        const KCoefs<ArF32> &KC = kcoefs(cf);
        float hp[8];
        powers(d.h, hp);
        const float tf = (float)th;
        float dk[8];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            float p = KC.Q[4][q];
#pragma unroll
            for (int m = 3; m >= 0; --m) p = fmaf(p, tf, KC.Q[m][q]);
            dk[q] = p * tf * hp[q];
        }
        const int pv = d.sel & 1;
#pragma unroll 4
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= k.n) continue;
            float ar = re(pv, m), ai = im(pv, m);
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                ar = fmaf(dk[q], re(wvec(q), m), ar);
                ai = fmaf(dk[q], im(wvec(q), m), ai);
            }
            scr[2 * m] = ar;
            scr[2 * m + 1] = ai;
        }
        __syncwarp();
    }

    // scr <- the vector v (rows < n)
    __device__ void vec_to_scr(int v) const
    {
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= k.n) continue;
            scr[2 * m] = re(v, m);
            scr[2 * m + 1] = im(v, m);
        }
        __syncwarp();
    }

    // Output j from the vector y in scr: Re<y|A_q|y> / <y|y> for every observable
    // (double-float accumulation, FP64 ratio), written by lane 0.
    __device__ __forceinline__ void output(const DenseCol &d, int j) const
    {
        const cf32 *y = reinterpret_cast<const cf32 *>(scr);
        Arc::red nn = Arc::rzero();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m < k.n) nn = Arc::radd(nn, Arc::abs2(y[m]));
        }
        nn = Arc::rsum(g, nn);
        double *out = k.out + ((size_t)d.il * k.n_t + j) * k.n_obs;
        for (int q = 0; q < k.n_obs; ++q) {
            cf32 v[R];
            opmv(1 + k.n_c + q, v);
            Arc::red ev = Arc::rzero();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                if (m < k.n) ev = Arc::radd(ev, Arc::dot_re(y[m], v[r]));
            }
            ev = Arc::rsum(g, ev);
            const double value = Arc::ratio(ev, nn);
            if (lane == 0) out[q] = value;
        }
        __syncwarp();
    }

    // state vector v <- scale M scr (rows < n; padded rows stay zero)
    __device__ __noinline__ void rhs_to(int v, float scale) const
    {
        cf32 y[R];
        opmv(0, y);
        float *dst = c.vec(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m < k.n) {
                dst[m] = scale * y[r].re;
                dst[NP + m] = scale * y[r].im;
            }
        }
    }

    // First theta in (0, 1] with ||y(theta)||^2 = r on the continuous extension
    // (Gram polynomial in FP64, first sign change on 8 points, Newton/bisection).
    __device__ __noinline__ double locate(const DenseCol &d, int &iters) const
    {
        double gram[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) gram[q] = 0.0;
        const KCoefs<ArF32> &KC = kcoefs(cf);
        float hp[8];
        powers(d.h, hp);
        const int pv = d.sel & 1;
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= k.n) continue;
            float ur[6], ui[6];
            ur[0] = re(pv, m);
            ui[0] = im(pv, m);
            float kr[8], ki[8];
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                kr[q] = hp[q] * re(wvec(q), m);
                ki[q] = hp[q] * im(wvec(q), m);
            }
#pragma unroll
            for (int mm = 1; mm <= 5; ++mm) {
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int q = 1; q < 8; ++q) {
                    sr = fmaf(KC.Q[mm - 1][q], kr[q], sr);
                    si = fmaf(KC.Q[mm - 1][q], ki[q], si);
                }
                ur[mm] = sr;
                ui[mm] = si;
            }
            int q = 0;
#pragma unroll
            for (int x = 0; x < 6; ++x)
#pragma unroll
                for (int y = x; y < 6; ++y, ++q)
                    gram[q] += (double)ur[x] * (double)ur[y] + (double)ui[x] * (double)ui[y];
        }
        double P[11];
#pragma unroll
        for (int s = 0; s < 11; ++s) P[s] = 0.0;
        {
            int q = 0;
#pragma unroll
            for (int x = 0; x < 6; ++x)
#pragma unroll
                for (int y = x; y < 6; ++y, ++q) {
                    const double v = g.sum(gram[q]);
                    P[x + y] += (x == y) ? v : 2.0 * v;
                }
        }
        P[0] -= d.r;
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

    // Step (C) with y(tau) in scr: channel n* from the weights ||C_n y||^2 and c_k;
    // psi <- C_n* y / ||C_n* y|| into psi buffer pv and scr.  -1 when every weight is 0.
    __device__ __noinline__ int jump(const DenseCol &d) const
    {
        double wq[kMaxChannels];
        double wsum = 0.0;
        for (int q = 0; q < k.n_c; ++q) {
            cf32 v[R];
            opmv(1 + q, v);
            Arc::red part = Arc::rzero();
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (lane + 32 * r < k.n) part = Arc::radd(part, Arc::abs2(v[r]));
            wq[q] = Arc::rval(Arc::rsum(g, part));
            wsum += wq[q];
        }
        if (!(wsum > 0.0)) return -1;
        const double target = d.c * wsum;
        double cum = 0.0;
        int ch = k.n_c - 1;
        for (int q = 0; q < k.n_c; ++q) {
            cum += wq[q];
            if (cum >= target) {
                ch = q;
                break;
            }
        }
        cf32 v[R];
        opmv(1 + ch, v);
        const double nc = sqrt(wq[ch]);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = Arc::div(v[r], nc);
        __syncwarp();
        float *psi = c.vec(d.sel & 1);
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= k.n) continue;
            scr[2 * m] = v[r].re;
            scr[2 * m + 1] = v[r].im;
            psi[m] = v[r].re;
            psi[NP + m] = v[r].im;
        }
        __syncwarp();
        return ch;
    }

    // Finishes the column's trajectory (status, counters) -- the caller refills.
    __device__ void finish(DenseCol &d, int status) const
    {
        if (lane == 0) {
            double *out = k.out + (size_t)d.il * k.n_t * k.n_obs;
            if (status != 0) {
                for (int j = d.j; j < k.n_t; ++j)
                    for (int q = 0; q < k.n_obs; ++q)
                        out[(size_t)j * k.n_obs + q] = __longlong_as_double(0x7ff8000000000000LL);
                atomicCAS(k.first_error, 0, status);
                atomicAdd(&k.counters[kFailed], 1ULL);
            }
            if (k.max_jumps > 0) k.n_jumps[d.il] = (int)d.n_jump;
            atomicAdd(&k.counters[kAccepted], d.n_acc);
            atomicAdd(&k.counters[kRejected], d.n_rej);
            atomicAdd(&k.counters[kRhs], d.n_rhs);
            atomicAdd(&k.counters[kJumps], d.n_jump);
            atomicAdd(&k.counters[kRootIters], (unsigned long long)d.root_iters);
        }
        d.il = -1;
    }

    // Before an attempt: the end of the time grid, the step limit, the last-step
    // clip.  Returns true when the column integrates on; otherwise the trajectory
    // has been finished.
    __device__ bool prepare(DenseCol &d) const
    {
        const double t_end = k.t[k.n_t - 1];
        if (t_end - d.t <= 4.0 * 2.220446049250313e-16 * fabs(t_end)) {
            if (d.j < k.n_t) {
                vec_to_scr(d.sel & 1);
                for (; d.j < k.n_t; ++d.j) output(d, d.j);
            }
            finish(d, 0);
            return false;
        }
        if (d.attempts >= k.max_steps) {
            finish(d, 4);
            return false;
        }
        d.flags &= ~2;
        if (d.t + 1.01 * d.h >= t_end) {
            d.h = t_end - d.t;
            d.flags |= 2;
        }
        if (d.h < 1e-14 * fmax(1.0, fabs(d.t))) {
            finish(d, 5);
            return false;
        }
        return true;
    }

    // Takes the column's next trajectories until one is ready to integrate or none
    // is left: (A), output 0, K_0 = M psi0 and the starting step.  The assignment
    // is static -- the column at position j of CTA b runs trajectories
    // b + G (j + 128 n), n = 0, 1, ..., for a grid of G CTAs -- so a CTA's work,
    // and with it every result, is reproducible bitwise from run to run.  Position
    // j = 8 u + w for the column u of control warp w spreads a CTA's last,
    // partial round over its control warps.
    __device__ __noinline__ void refill(DenseCol &d) const
    {
        const double t_end = k.t[k.n_t - 1];
        const long long b = blockIdx.x, G = gridDim.x, slot = c.col - b * kTcCols;
        const long long jpos = (slot % 16) * 8 + slot / 16;
        for (;;) {
            const int n = d.round;
            const long long i = b + G * (jpos + (long long)kTcCols * n);
            if (i >= k.ntraj) {
                d.il = -1;
                d.round = n + 1;
                return;
            }
            d = DenseCol{};
            d.round = n + 1;
            d.il = i;
            jump_draws(k.seed, k.traj0 + d.il, 0, d.r, d.c);
            d.t = k.t[0];
            // psi0 into buffer 0 (padded rows zero) and scr
            const cf32 *p0 = static_cast<const cf32 *>(k.psi0);
            float *psi = c.vec(kVPsi0);
            float *k0v = c.vec(kVK0);
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                const cf32 v = m < k.n ? p0[m] : cf32{0.f, 0.f};
                psi[m] = v.re;
                psi[NP + m] = v.im;
                k0v[m] = 0.f;
                k0v[NP + m] = 0.f;
                if (m < k.n) {
                    scr[2 * m] = v.re;
                    scr[2 * m + 1] = v.im;
                }
            }
            __syncwarp();
            output(d, 0);
            d.j = 1;
            rhs_to(wvec(1), 1.f);  // K_0 = M psi0 for the starting step (wt_1 is formed by the products)
            ++d.n_rhs;
            // starting step (Hairer, Norsett & Wanner, Sec. II.4)
            const double span = t_end - d.t;
            double d0 = 0.0, d1 = 0.0;
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                if (m >= k.n) continue;
                const double yr = psi[m], yi = psi[NP + m], fr = k0v[m], fi = k0v[NP + m];
                const double sc = k.atol + k.rtol * sqrt(yr * yr + yi * yi);
                d0 += (yr * yr + yi * yi) / (sc * sc);
                d1 += (fr * fr + fi * fi) / (sc * sc);
            }
            d0 = sqrt(g.sum(d0) / k.n);
            d1 = sqrt(g.sum(d1) / k.n);
            double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
            if (h0 > span) h0 = span;
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                if (m >= k.n) continue;
                scr[2 * m] = (float)((double)psi[m] + h0 * (double)k0v[m]);
                scr[2 * m + 1] = (float)((double)psi[NP + m] + h0 * (double)k0v[NP + m]);
            }
            __syncwarp();
            cf32 f1v[R];
            opmv(0, f1v);
            double d2 = 0.0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cf32 f1 = f1v[r];
                const int m = lane + 32 * r;
                if (m >= k.n) continue;
                const double yr = psi[m], yi = psi[NP + m];
                const double sc = k.atol + k.rtol * sqrt(yr * yr + yi * yi);
                const double dr = (double)f1.re - (double)k0v[m], di = (double)f1.im - (double)k0v[NP + m];
                d2 += (dr * dr + di * di) / (sc * sc);
            }
            __syncwarp();
            ++d.n_rhs;
            d2 = sqrt(g.sum(d2) / k.n) / h0;
            const double dm = d1 > d2 ? d1 : d2;
            const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
            d.h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
            if (d.h > span) d.h = span;
            if (prepare(d)) return;
        }
    }

    // Tail mode: the seven products of one attempt on this warp alone, with the
    // control's own operator copy (FP32 products): wt_s = 2^-e M wt_{s-1}, wt_0 = psi,
    // where the tensor-core products put them.
    __device__ __noinline__ void simt_products(const DenseCol &d) const
    {
        const float dn = down();
        for (int s = 1; s <= 7; ++s) {
            vec_to_scr(s == 1 ? (d.sel & 1) : wvec(s - 1));
            cf32 v[R];
            opmv(0, v);
            float *dst = c.vec(wvec(s));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = lane + 32 * r;
                if (m < k.n) {
                    dst[m] = dn * v[r].re;
                    dst[NP + m] = dn * v[r].im;
                }
            }
            __syncwarp();
        }
    }

    // After the six products of an attempt.
    __device__ void step(DenseCol &d) const
    {
        const double t_end = k.t[k.n_t - 1];
        const KCoefs<ArF32> &KC = kcoefs(cf);
        float hp[8];
        powers(d.h, hp);
        float cb[7];
#pragma unroll
        for (int q = 1; q < 7; ++q) cb[q] = KC.beta[q] * hp[q];
        const float g5 = KC.gam[0] * hp[5], g6 = KC.gam[1] * hp[6], g7 = KC.gam[2] * hp[7];
        const int pv = d.sel & 1;
        float *yn = c.vec(1 - pv);
        d.n_rhs += 7;
        ++d.attempts;
        // the 5th-order solution psi + sum_k beta_k H^k wt_k, its squared norm, and
        // the error estimate sum_k gamma_k H^k wt_k (no cancellation), scaled RMS
        float esum = 0.f;
        Arc::red nr = Arc::rzero();
#pragma unroll 4
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            if (m >= k.n) continue;
            const cf32 y0{re(pv, m), im(pv, m)};
            float yr = y0.re, yi = y0.im;
#pragma unroll
            for (int q = 1; q < 7; ++q) {
                yr = fmaf(cb[q], re(wvec(q), m), yr);
                yi = fmaf(cb[q], im(wvec(q), m), yi);
            }
            yn[m] = yr;
            yn[NP + m] = yi;
            const float ere = fmaf(g5, re(wvec(5), m), fmaf(g6, re(wvec(6), m), g7 * re(wvec(7), m)));
            const float eim = fmaf(g5, im(wvec(5), m), fmaf(g6, im(wvec(6), m), g7 * im(wvec(7), m)));
            const cf32 y1{yr, yi};
            const float ay2 = y0.re * y0.re + y0.im * y0.im, an2 = y1.re * y1.re + y1.im * y1.im;
            const float sc = (float)k.atol + (float)k.rtol * sqrtf(ay2 > an2 ? ay2 : an2);
            esum += (ere * ere + eim * eim) / (sc * sc);
            nr = Arc::radd(nr, Arc::abs2(y1));
        }
        const double err = (double)sqrtf(g.sum(esum) / (float)k.n);
        if (!(err <= 1.0)) {
            if (!isfinite(err)) {
                finish(d, 6);
                refill(d);
                return;
            }
            double fac = Arc::controller(err);
            if (fac < kFacMin) fac = kFacMin;
            d.h *= fac;
            d.flags |= 1;
            ++d.n_rej;
            if (!prepare(d)) refill(d);
            return;
        }
        ++d.n_acc;
        const bool last = (d.flags & 2) != 0;
        const double t_new = last ? t_end : d.t + d.h;
        const double nn = Arc::rval(Arc::rsum(g, nr));
        if (nn < d.r) {
            // (C): the crossing lies in this step
            const double th = locate(d, d.root_iters);
            double tau = d.t + th * d.h;
            if (tau > t_new) tau = t_new;
            for (; d.j < k.n_t && k.t[d.j] <= tau; ++d.j) {
                double thj = (k.t[d.j] - d.t) / d.h;
                if (thj > 1.0) thj = 1.0;
                dense_to_scr(d, thj);
                output(d, d.j);
            }
            dense_to_scr(d, th);
            const int ch = jump(d);
            if (ch < 0) {
                finish(d, 7);
                refill(d);
                return;
            }
            if (lane == 0 && (long long)d.n_jump < k.max_jumps) {
                k.jump_t[(size_t)d.il * k.max_jumps + d.n_jump] = tau;
                k.jump_ch[(size_t)d.il * k.max_jumps + d.n_jump] = ch;
            }
            ++d.n_jump;
            // (D)
            ++d.k;
            jump_draws(k.seed, k.traj0 + d.il, d.k, d.r, d.c);
            d.t = tau;  // the next attempt's products start from the new psi
            d.flags &= ~1;
            if (!prepare(d)) refill(d);
            return;
        }
        for (; d.j < k.n_t && k.t[d.j] <= t_new; ++d.j) {
            double thj = (k.t[d.j] - d.t) / d.h;
            if (thj > 1.0) thj = 1.0;
            dense_to_scr(d, thj);
            output(d, d.j);
        }
        double fac = (err == 0.0) ? kFacMax : Arc::controller(err);
        if (fac > kFacMax) fac = kFacMax;
        if (fac < kFacMin) fac = kFacMin;
        if ((d.flags & 1) && fac > 1.0) fac = 1.0;
        d.flags &= ~1;
        d.t = t_new;
        d.sel ^= 1;  // ynew becomes psi
        d.h *= fac;
        if (!prepare(d)) refill(d);
    }
};

template <int NP>
__global__ void __launch_bounds__(kThreadsTc, 1)
    dense_tc_kernel(const __grid_constant__ DenseArgs a, const __grid_constant__ CUtensorMap opmap)
{
    using S = TcShape<NP>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    float *scr_all = reinterpret_cast<float *>(sm + S::OFF_SCR);
    float *s_hf = reinterpret_cast<float *>(sm + S::OFF_HF);
    int *s_sel = reinterpret_cast<int *>(sm + S::OFF_SEL);
    float *cf = reinterpret_cast<float *>(sm + S::OFF_COEF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + S::OFF_BAR);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + S::OFF_MISC);
    int *s_abort = reinterpret_cast<int *>(sm + S::OFF_MISC + 4);
    int *s_count = reinterpret_cast<int *>(sm + S::OFF_MISC + 8);  // active columns per control warp
    int *s_mode = reinterpret_cast<int *>(sm + S::OFF_MISC + 40);  // next attempt: 0 products, 1 tail, 2 done
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    static_assert(sizeof(KCoefs<ArF32>) == kCoefFloats * sizeof(float), "coefficient table size");
    if (threadIdx.x == 0) {
        krylov_coefs<ArF32>(reinterpret_cast<KCoefs<ArF32> *>(cf));
        for (int i = 0; i < 2 * kOpRing; ++i) tc::mbar_init(&bars[i], 1);  // op full / empty
        for (int i = 0; i < 2; ++i) tc::mbar_init(&bars[2 * kOpRing + i], kProducers);  // y_full
        for (int i = 2; i < 5; ++i) tc::mbar_init(&bars[2 * kOpRing + i], 1);  // y_empty, acc_full
        tc::mbar_init(&bars[2 * kOpRing + 5], 1);                             // final drain
        *s_abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) tc::tma_prefetch_map(&opmap);
    if (warp == 1) {
        tc::tmem_alloc(s_tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();

    Pipe p;
    p.op = sm + S::OFF_OP;
    p.yt = sm + S::OFF_Y;
    p.op_full = bars;               // [kOpRing] full, then [kOpRing] empty
    p.op_empty = bars + kOpRing;
    p.y_full = bars + 2 * kOpRing;
    p.y_empty = bars + 2 * kOpRing + 2;
    p.acc_full = bars + 2 * kOpRing + 4;
    p.abort = s_abort;
    p.tmem = *s_tmem;
    p.ocnt = p.ycnt = p.acnt = 0;
    p.limit = a.wait_limit_ns ? a.wait_limit_ns : tc::kWaitLimitNs;

    if (a.mode == kDenseRhs) {
        // Tiles of 128 vectors; the r = tiles mod CTAs tiles of a partial last
        // wave are split into their two output chunks (NP = 256, where a chunk
        // is one epilogue half), so that wave takes half a tile's time: 157 tiles
        // on 152 CTAs end after 1.5 tile-times instead of 2.
        const long long tiles = (a.rhs_n + kTcCols - 1) / kTcCols, ctas = gridDim.x;
        const long long r = (S::NCHUNK == 2 && S::HALF == 256 && tiles > ctas) ? tiles % ctas : 0;
        const long long full = tiles - r, items = full + 2 * r;
        for (long long i = blockIdx.x; i < items && !*s_abort; i += ctas) {
            if (i < full) {
                stage_product<NP>(a, p, &opmap, 0, i * kTcCols, s_hf, s_sel, cf);
            } else {
                const long long h = i - full;
                const int c = (int)(h & 1);
                stage_product<NP>(a, p, &opmap, 0, (full + h / 2) * kTcCols, s_hf, s_sel, cf, c, c + 1);
            }
        }
    } else {
        const long long tile_base = (long long)blockIdx.x * kTcCols;
        if (warp >= 2) {
            const int pw = warp - 2;
            ColCtl<NP> cc{a, a.k, Group<32>(threadIdx.x, nullptr), lane, Ctl{&a, 0, NP, S::KD},
                          scr_all + pw * S::KD, cf};
            int active = 0;
            for (int r = 16 * pw; r < 16 * pw + 16; ++r) {
                cc.c.col = (int)(tile_base + r);
                DenseCol d{};
                cc.refill(d);
                if (lane == 0) a.col[cc.c.col] = d;
                s_hf[r] = d.il >= 0 ? (float)d.h : 0.f;
                s_sel[r] = d.sel;
                active += d.il >= 0;
            }
            if (lane == 0) s_count[pw] = active;
        }
        __syncthreads();
        for (;;) {
            // one thread decides the mode: with at most one live column per
            // control warp, full 128-column products would mostly multiply idle
            // columns, so the control warps finish their columns alone (the
            // decision depends only on this CTA's columns, so it is reproducible)
            if (threadIdx.x == 0) {
                int active = 0;
                for (int w = 0; w < 8; ++w) active += s_count[w];
                *s_mode = (active == 0 || *s_abort) ? 2 : active <= 8 ? 1 : 0;
            }
            __syncthreads();
            const int mode = *s_mode;
            if (mode == 2) break;
            if (mode == 1) {
                if (warp >= 2) {
                    const int pw = warp - 2;
                    ColCtl<NP> cc{a, a.k, Group<32>(threadIdx.x, nullptr), lane, Ctl{&a, 0, NP, S::KD},
                                  scr_all + pw * S::KD, cf};
                    int act = 0;
                    for (int r = 16 * pw; r < 16 * pw + 16; ++r) {
                        cc.c.col = (int)(tile_base + r);
                        DenseCol d = a.col[cc.c.col];
                        if (d.il >= 0) {
                            cc.simt_products(d);
                            cc.step(d);
                            __syncwarp();
                            if (lane == 0) a.col[cc.c.col] = d;
                        }
                        act += d.il >= 0;
                    }
                    if (lane == 0) s_count[pw] = act;
                }
                __syncthreads();
                continue;
            }
            for (int s = 1; s <= 7; ++s) stage_product<NP>(a, p, &opmap, s, tile_base, s_hf, s_sel, cf);
            if (warp >= 2 && !*s_abort) {
                const int pw = warp - 2;
                ColCtl<NP> cc{a, a.k, Group<32>(threadIdx.x, nullptr), lane, Ctl{&a, 0, NP, S::KD},
                              scr_all + pw * S::KD, cf};
                int act = 0;
                for (int r = 16 * pw; r < 16 * pw + 16; ++r) {
                    cc.c.col = (int)(tile_base + r);
                    DenseCol d = a.col[cc.c.col];
                    if (d.il >= 0) {
                        cc.step(d);
                        __syncwarp();
                        if (lane == 0) a.col[cc.c.col] = d;
                    }
                    s_hf[r] = d.il >= 0 ? (float)d.h : 0.f;
                    s_sel[r] = d.sel;
                    act += d.il >= 0;
                }
                if (lane == 0) s_count[pw] = act;
            }
            __syncthreads();
        }
    }

    // drain: the operator loads this CTA issued have landed (after an abort some
    // may not have been consumed), and every tensor-core operation has completed
    // before the tensor memory is released
    if (warp == 0 && lane == 0) {
        int no_abort = 0;
        for (uint32_t i = p.ocnt > (uint32_t)kOpRing ? p.ocnt - kOpRing : 0; i < p.ocnt; ++i)
            tc::mbar_wait(&p.op_full[i % kOpRing], (i / kOpRing) & 1, &no_abort);
    }
    __syncthreads();
    if (warp == 1) {
        if (lane == 0) {
            tc::mma_commit(&bars[2 * kOpRing + 5]);
            int no_abort = 0;
            tc::mbar_wait(&bars[2 * kOpRing + 5], 0, &no_abort);
        }
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(p.tmem, kTmemCols);
    }
}

}  // namespace

template <int NP>
cudaError_t launch_dense_tc_np(const DenseArgs &a, const CUtensorMap &map, cudaStream_t stream, LaunchInfo *info)
{
    using S = TcShape<NP>;
    auto kern = dense_tc_kernel<NP>;
    // at least 116 KB so that no two CTAs share an SM: each holds all 512
    // tensor-memory columns for its lifetime
    const int smem = S::BYTES > 116 * 1024 ? S::BYTES : 116 * 1024;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid;
    if (a.mode == kDenseRhs) {
        const long long tiles = (a.rhs_n + kTcCols - 1) / kTcCols;
        grid = (int)(tiles < sms ? tiles : sms);
        if (grid < 1) return cudaSuccess;
    } else {
        grid = a.cols / kTcCols;
        if (grid < 1 || grid * kTcCols != a.cols) return cudaErrorInvalidValue;
    }
    kern<<<grid, kThreadsTc, smem, stream>>>(a, map);
    if (info) {
        info->group = kTcCols;
        info->rows = NP;
        info->grid = grid;
        info->block = kThreadsTc;
        info->smem = smem;
    }
    return cudaGetLastError();
}

}  // namespace qtm
