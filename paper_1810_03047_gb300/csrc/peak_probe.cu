// peak_probe.cu -- arithmetic peaks of this GPU, measured: the denominators of the
// roofline fractions of the trajectory kernels, which are bound by arithmetic
// (their state never leaves the SM).  Each probe is a grid of independent
// multiply-add chains (kChains per thread, so the pipe never waits on a
// dependency), sized to fill every SM, for the three arithmetics of the
// trajectory kernel:
//   FP64   fma chains                  -- the complex128 path's pipe
//   FP32   fmaf chains                 -- the complex64 path's pipe
//   DF     double-float multiply-adds  -- the double-float path: the same
//          accumulation the kernel uses (TwoProd with two cross terms into a
//          lazy TwoSum accumulator, 12 FP32 instructions), counted as the two
//          FP64-class flops it stands for.
// The paper has no counterpart; these kernels only measure the machine.
#include "../../include/qtm.h"
#include "qtm_arith.cuh"
#include "qtm_launch.h"

namespace qtm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_fp64(long long iters, double a, double *out)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-9 + c;
    const double b = 1.0 - a;
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;  // keeps the chains alive; never true
}

__global__ void __launch_bounds__(kProbeThreads) probe_fp32(long long iters, float a, float *out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-6f + c;
    const float b = 1.f - a;
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;
}

// x <- a x + b in double-float, the accumulation step of the trajectory kernel
// (dacc_add_prod: TwoProd, two cross terms, TwoSum into the accumulator): 12 FP32
// instructions per step, and the product operand changes every step, as it does
// there, so nothing can be hoisted out of the loop.
__global__ void __launch_bounds__(kProbeThreads) probe_df(long long iters, float a_hi, float a_lo, float b_hi,
                                                          float *out)
{
    df x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = df{1e-3f * (c + 1) + threadIdx.x * 1e-9f, 0.f};
    const df a{a_hi, a_lo};
    for (long long i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            dacc t{b_hi, 0.f};
            dacc_add_prod(t, a, x[c]);
            x[c] = df{t.s, t.c};
        }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].hi + x[c].lo;
    if (s == 12345.678f) out[0] = s;
}

}  // namespace
}  // namespace qtm

extern "C" qtm_status qtm_arith_peak_launch(int32_t kind, int64_t iters, void *scratch_dev, void *cuda_stream,
                                            double *flop)
{
    using namespace qtm;
    if (kind < QTM_PEAK_FP64 || kind > QTM_PEAK_DF64 || iters < 1 || !scratch_dev || !flop) {
        set_last_error("qtm_arith_peak_launch: need a known kind, iters >= 1, scratch and flop");
        return QTM_ERR_ARG;
    }
    int dev = 0, sms = 0, nb = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        set_last_error("qtm_arith_peak_launch: device query failed");
        return QTM_ERR_CUDA;
    }
    const void *fn = kind == QTM_PEAK_FP64   ? (const void *)probe_fp64
                     : kind == QTM_PEAK_FP32 ? (const void *)probe_fp32
                                             : (const void *)probe_df;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kProbeThreads, 0)) != cudaSuccess) {
        set_last_error("qtm_arith_peak_launch: occupancy query failed");
        return QTM_ERR_CUDA;
    }
    if (nb < 1) nb = 1;
    const unsigned grid = (unsigned)(nb * sms);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (kind == QTM_PEAK_FP64)
        probe_fp64<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, static_cast<double *>(scratch_dev));
    else if (kind == QTM_PEAK_FP32)
        probe_fp32<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999f, static_cast<float *>(scratch_dev));
    else
        probe_df<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-12f, 1e-4f, static_cast<float *>(scratch_dev));
    if ((e = cudaGetLastError()) != cudaSuccess) {
        set_last_error("qtm_arith_peak_launch: launch failed");
        return QTM_ERR_CUDA;
    }
    // two flops per multiply-add (a double-float multiply-add counts as one FP64-class multiply-add)
    *flop = 2.0 * (double)grid * kProbeThreads * kChains * (double)iters;
    return QTM_OK;
}
