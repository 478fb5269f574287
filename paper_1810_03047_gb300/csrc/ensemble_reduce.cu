// ensemble_reduce.cu -- the average over trajectories (Sec. 3: every node averages
// its trajectories, the master averages again).  Here one GPU holds every
// trajectory's values, [ntraj][P] with P = n_t * n_obs, and reduces them in FP64
// in a fixed order: S contiguous segments of trajectories are summed
// sequentially (threads run along P, so every load is coalesced), then the S
// partial sums are added in segment order.  The standard error takes a second
// pass over the deviations from the mean.  No floating-point atomics are used,
// so the result is bitwise reproducible for a given trajectory count.
#include <mutex>

#include "../../include/qtm.h"
#include "moments.h"
#include "qtm_launch.h"

namespace qtm {

namespace {
constexpr int kThreads = 128;
constexpr long long kSegLen = 128;   // trajectories per segment
constexpr int kMaxSegments = 4096;

long long segment_length(long long ntraj)
{
    long long seg = kSegLen;
    while ((ntraj + seg - 1) / seg > kMaxSegments) seg *= 2;
    return seg;
}

// Pass 1: per segment, sum x and sum x^2 (the raw sums reported for combining shards).
__global__ void __launch_bounds__(kThreads)
segment_sums(const double *__restrict__ x, long long ntraj, int P, long long seg_len,
             double *__restrict__ psum, double *__restrict__ psq)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const long long s = blockIdx.y;
    if (p >= P) return;
    const long long b0 = s * seg_len;
    const long long b1 = b0 + seg_len < ntraj ? b0 + seg_len : ntraj;
    double sum = 0.0, sq = 0.0;
    for (long long b = b0; b < b1; ++b) {
        const double v = x[b * P + p];
        sum += v;
        sq = fma(v, v, sq);
    }
    psum[s * P + p] = sum;
    psq[s * P + p] = sq;
}

// Segment partials added in segment order; the mean follows.
__global__ void __launch_bounds__(kThreads)
combine_sums(const double *__restrict__ psum, const double *__restrict__ psq, int S, int P,
             long long ntraj, double *sum, double *sumsq, double *mean)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= P) return;
    double s1 = 0.0, s2 = 0.0;
    for (int s = 0; s < S; ++s) {
        s1 += psum[(long long)s * P + p];
        s2 += psq[(long long)s * P + p];
    }
    sum[p] = s1;
    sumsq[p] = s2;
    mean[p] = ntraj > 0 ? s1 / (double)ntraj : 0.0;
}

// Pass 2: per segment, sum (x - mean)^2, so the variance does not suffer the
// cancellation of sum x^2 - (sum x)^2 / n when the spread is small.
__global__ void __launch_bounds__(kThreads)
segment_devs(const double *__restrict__ x, long long ntraj, int P, long long seg_len,
             const double *__restrict__ mean, double *__restrict__ pdev)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const long long s = blockIdx.y;
    if (p >= P) return;
    const long long b0 = s * seg_len;
    const long long b1 = b0 + seg_len < ntraj ? b0 + seg_len : ntraj;
    const double m = mean[p];
    double d2 = 0.0;
    for (long long b = b0; b < b1; ++b) {
        const double d = x[b * P + p] - m;
        d2 = fma(d, d, d2);
    }
    pdev[s * P + p] = d2;
}

// Standard error sqrt(var / n) with the sample variance (n - 1 divisor).
__global__ void __launch_bounds__(kThreads)
combine_devs(const double *__restrict__ pdev, int S, int P, long long ntraj, double *se)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= P) return;
    double d2 = 0.0;
    for (int s = 0; s < S; ++s) d2 += pdev[(long long)s * P + p];
    const double nt = (double)ntraj;
    se[p] = ntraj > 1 ? sqrt(d2 / (nt - 1.0) / nt) : 0.0;
}
// Exact moments (moments.h), pass 1: per segment and output value p, the moment
// words of the segment's values, stored [segment][word][P] so that both passes
// read and write along p.
__global__ void __launch_bounds__(kThreads)
segment_moments(const double *__restrict__ x, long long ntraj, int P, int n_obs, const int *__restrict__ scale_exp,
                long long seg_len, long long *__restrict__ part)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const long long s = blockIdx.y;
    if (p >= P) return;
    const int E = scale_exp[p % n_obs];
    const double sc = pow2(kQuantBits - E), lim = pow2(E);
    const long long b0 = s * seg_len;
    const long long b1 = b0 + seg_len < ntraj ? b0 + seg_len : ntraj;
    MomentAcc acc;
    acc.clear();
    for (long long b = b0; b < b1; ++b) acc.add(x[b * P + p], sc, lim);
    acc.normalize();
    acc.store(part + s * kMomentWords * P + p, P);
}

// Pass 2: the segments' words added per output value (integers: any order gives
// the same totals), normalised, stored [P][kMomentWords].
__global__ void __launch_bounds__(kThreads)
combine_moments(const long long *__restrict__ part, int S, int P, long long *__restrict__ words)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= P) return;
    long long w[kMomentWords] = {};
    for (int s = 0; s < S; ++s) {
        const long long *q = part + (long long)s * kMomentWords * P + p;
#pragma unroll
        for (int k = 0; k < kMomentWords; ++k) w[k] += q[(long long)k * P];
        if ((s & 1023) == 1023) {
            normalize_digits(w + kS1, kS1Digits);
            normalize_digits(w + kS2, kS2Digits);
        }
    }
    normalize_digits(w + kS1, kS1Digits);
    normalize_digits(w + kS2, kS2Digits);
#pragma unroll
    for (int k = 0; k < kMomentWords; ++k) words[(long long)p * kMomentWords + k] = w[k];
}
}  // namespace

cudaError_t launch_ensemble_moments(const double *out, long long ntraj, int P, int n_obs, const int *scale_exp,
                                    long long *partial, long long *words, cudaStream_t stream)
{
    if (P <= 0) return cudaSuccess;
    const int S = reduce_segments(ntraj);
    const long long seg = segment_length(ntraj);
    const dim3 grid_seg((P + kThreads - 1) / kThreads, S);
    const unsigned grid_p = (P + kThreads - 1) / kThreads;
    segment_moments<<<grid_seg, kThreads, 0, stream>>>(out, ntraj, P, n_obs, scale_exp, seg, partial);
    combine_moments<<<grid_p, kThreads, 0, stream>>>(partial, S, P, words);
    return cudaGetLastError();
}

int reduce_segments(long long ntraj)
{
    const long long seg = segment_length(ntraj);
    const long long S = (ntraj + seg - 1) / seg;
    return (int)(S < 1 ? 1 : S);
}

cudaError_t launch_ensemble_reduce(const double *out, long long ntraj, int P, double *partial,
                                   double *sum, double *sumsq, double *mean, double *se,
                                   cudaStream_t stream)
{
    if (P <= 0) return cudaSuccess;
    const int S = reduce_segments(ntraj);
    const long long seg = segment_length(ntraj);
    double *psum = partial, *psq = partial + (size_t)S * P;
    const dim3 grid_seg((P + kThreads - 1) / kThreads, S);
    const unsigned grid_p = (P + kThreads - 1) / kThreads;
    segment_sums<<<grid_seg, kThreads, 0, stream>>>(out, ntraj, P, seg, psum, psq);
    combine_sums<<<grid_p, kThreads, 0, stream>>>(psum, psq, S, P, ntraj, sum, sumsq, mean);
    segment_devs<<<grid_seg, kThreads, 0, stream>>>(out, ntraj, P, seg, mean, psum);
    combine_devs<<<grid_p, kThreads, 0, stream>>>(psum, S, P, ntraj, se);
    return cudaGetLastError();
}

}  // namespace qtm

// ---------------------------------------------------------------------------
// Allocation-free variant: the same four kernels, with the partial sums in a
// fixed array of the library's device image instead of context memory.
// ---------------------------------------------------------------------------

namespace {

static __device__ __align__(256) double g_static_scratch[QTM_STATIC_SCRATCH_DOUBLES];

// The array's device address, cached per CUDA context: host code cannot use the
// symbol itself as a device pointer, and the address belongs to the context the
// module was loaded into, so a cache keyed on the device ordinal alone would go
// stale when that device's context is destroyed and created again (a device
// reset).  The current context is read through the driver's cuCtxGetCurrent.
constexpr int kMaxContexts = 64;
std::mutex g_static_scratch_mutex;
struct ScratchEntry {
    void *ctx;
    double *addr;
};
ScratchEntry g_static_scratch_addr[kMaxContexts] = {};
int g_static_scratch_entries = 0;

typedef int (*CtxGetCurrentFn)(void **);

cudaError_t current_context(void **ctx)
{
    static CtxGetCurrentFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !f) return cudaErrorNotSupported;
        fn = reinterpret_cast<CtxGetCurrentFn>(f);
    }
    *ctx = nullptr;
    return fn(ctx) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of g_static_scratch in the current context, looked up the first
// time a context is seen (cudaGetSymbolAddress also binds the device's primary
// context to this thread when none is current yet).
cudaError_t static_scratch(double **out)
{
    void *ctx = nullptr;
    cudaError_t e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_static_scratch_mutex);
    if (ctx)
        for (int i = 0; i < g_static_scratch_entries; ++i)
            if (g_static_scratch_addr[i].ctx == ctx) {
                *out = g_static_scratch_addr[i].addr;
                return cudaSuccess;
            }
    void *p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_static_scratch)) != cudaSuccess) return e;
    if (!ctx && (e = current_context(&ctx)) != cudaSuccess) return e;
    if (ctx && g_static_scratch_entries < kMaxContexts)
        g_static_scratch_addr[g_static_scratch_entries++] = ScratchEntry{ctx, static_cast<double *>(p)};
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" qtm_status qtm_ensemble_reduce_static(const double *values_dev, int64_t ntraj, int32_t n_values,
                                                 double *sum_dev, double *sumsq_dev, double *mean_dev,
                                                 double *stderr_dev, void *cuda_stream)
{
    using namespace qtm;
    if (ntraj < 0) {
        set_last_error("qtm_ensemble_reduce_static: ntraj must be >= 0");
        return QTM_ERR_ARG;
    }
    if (n_values < 1 || n_values > QTM_STATIC_MAX_VALUES) {
        set_last_error("qtm_ensemble_reduce_static: n_values must be in 1..QTM_STATIC_MAX_VALUES (262144); "
                       "the fixed scratch array cannot hold the partial sums of more");
        return QTM_ERR_ARG;
    }
    if ((ntraj > 0 && !values_dev) || !sum_dev || !sumsq_dev || !mean_dev || !stderr_dev) {
        set_last_error("qtm_ensemble_reduce_static: NULL buffer");
        return QTM_ERR_ARG;
    }
    double *scratch = nullptr;
    cudaError_t e = static_scratch(&scratch);
    if (e != cudaSuccess) {
        set_last_error("qtm_ensemble_reduce_static: cudaGetSymbolAddress of the scratch array failed");
        return QTM_ERR_CUDA;
    }
    // Segments: as in the context path, but never more than the scratch holds
    // (pass 1 keeps two partials per segment and value).
    const long long P = n_values;
    long long max_seg_count = QTM_STATIC_SCRATCH_DOUBLES / (2 * P);
    if (max_seg_count > kMaxSegments) max_seg_count = kMaxSegments;
    long long seg = kSegLen;
    while ((ntraj + seg - 1) / seg > max_seg_count) seg *= 2;
    long long S = (ntraj + seg - 1) / seg;
    if (S < 1) S = 1;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    double *psum = scratch, *psq = scratch + S * P;
    const dim3 grid_seg((unsigned)((P + kThreads - 1) / kThreads), (unsigned)S);
    const unsigned grid_p = (unsigned)((P + kThreads - 1) / kThreads);
    segment_sums<<<grid_seg, kThreads, 0, stream>>>(values_dev, ntraj, (int)P, seg, psum, psq);
    combine_sums<<<grid_p, kThreads, 0, stream>>>(psum, psq, (int)S, (int)P, ntraj, sum_dev, sumsq_dev,
                                                  mean_dev);
    segment_devs<<<grid_seg, kThreads, 0, stream>>>(values_dev, ntraj, (int)P, seg, mean_dev, psum);
    combine_devs<<<grid_p, kThreads, 0, stream>>>(psum, (int)S, (int)P, ntraj, stderr_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        set_last_error("qtm_ensemble_reduce_static: kernel launch failed");
        return QTM_ERR_CUDA;
    }
    return QTM_OK;
}
