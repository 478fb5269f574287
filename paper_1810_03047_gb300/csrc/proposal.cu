// proposal.cu -- training kernels of the jump-time proposal MLP (6 -> 64 -> 64 -> 1,
// SiLU, FP32).  One training step = one tile kernel (forward and backward pass of
// 64 samples per CTA, per-CTA partial gradients), one reduction kernel (partials
// added in CTA order, so the gradient is bitwise reproducible) and one Adam update.
#include "proposal.cuh"

namespace qtm {

namespace {

constexpr int kTile = 64;     // samples per CTA
constexpr int kThreads = 256;
constexpr int kLd = kMlpHidden + 1;  // padded row length of the per-sample arrays

struct TileSmem {
    float p[kMlpParams];
    float x[kTile][kMlpIn];
    float t[kTile];
    float dy[kTile];
    float z1[kTile][kLd];
    float h1[kTile][kLd];
    float z2[kTile][kLd];
    float d2[kTile][kLd];
    float d1[kTile][kLd];
};

__global__ void __launch_bounds__(kThreads)
mlp_tile(const float *__restrict__ params, const float *__restrict__ X, const float *__restrict__ T, long long n,
         float *__restrict__ gpart, float *__restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(raw);
    const int tid = threadIdx.x;
    const long long s0 = (long long)blockIdx.x * kTile;
    const float inv_n = 1.0f / (float)n;
    for (int i = tid; i < kMlpParams; i += kThreads) S.p[i] = params[i];
    for (int i = tid; i < kTile * kMlpIn; i += kThreads) {
        const long long s = s0 + i / kMlpIn;
        S.x[i / kMlpIn][i % kMlpIn] = s < n ? X[s * kMlpIn + i % kMlpIn] : 0.0f;
    }
    for (int i = tid; i < kTile; i += kThreads) S.t[i] = s0 + i < n ? T[s0 + i] : 0.0f;
    __syncthreads();
    const float *W1 = S.p + kOffW1, *B1 = S.p + kOffB1, *W2 = S.p + kOffW2, *B2 = S.p + kOffB2;
    const float *W3 = S.p + kOffW3, b3 = S.p[kOffB3];

    // forward: z1 = W1 x + b1, h1 = silu(z1), z2 = W2 h1 + b2, y = w3 . silu(z2) + b3
    for (int i = tid; i < kTile * kMlpHidden; i += kThreads) {
        const int s = i / kMlpHidden, j = i % kMlpHidden;
        float z = B1[j];
#pragma unroll
        for (int q = 0; q < kMlpIn; ++q) z = fmaf(W1[j * kMlpIn + q], S.x[s][q], z);
        S.z1[s][j] = z;
        S.h1[s][j] = silu(z);
    }
    __syncthreads();
    for (int i = tid; i < kTile * kMlpHidden; i += kThreads) {
        const int s = i / kMlpHidden, k = i % kMlpHidden;
        float z = B2[k];
        for (int j = 0; j < kMlpHidden; ++j) z = fmaf(W2[k * kMlpHidden + j], S.h1[s][j], z);
        S.z2[s][k] = z;
    }
    __syncthreads();
    float lsum = 0.0f;
    if (tid < kTile) {
        float y = b3;
        for (int k = 0; k < kMlpHidden; ++k) y = fmaf(W3[k], silu(S.z2[tid][k]), y);
        const bool valid = s0 + tid < n;
        const float e = valid ? y - S.t[tid] : 0.0f;
        S.dy[tid] = 2.0f * e * inv_n;
        lsum = e * e * inv_n;
    }
    __syncthreads();
    // backward
    for (int i = tid; i < kTile * kMlpHidden; i += kThreads) {
        const int s = i / kMlpHidden, k = i % kMlpHidden;
        S.d2[s][k] = S.dy[s] * W3[k] * silu_grad(S.z2[s][k]);
    }
    __syncthreads();
    float *g = gpart + (size_t)blockIdx.x * kMlpParams;
    for (int i = tid; i < kMlpHidden * kMlpHidden; i += kThreads) {  // dW2[k][j]
        const int k = i / kMlpHidden, j = i % kMlpHidden;
        float a = 0.0f;
        for (int s = 0; s < kTile; ++s) a = fmaf(S.d2[s][k], S.h1[s][j], a);
        g[kOffW2 + i] = a;
    }
    for (int i = tid; i < kTile * kMlpHidden; i += kThreads) {  // d1 = silu'(z1) * W2^T d2
        const int s = i / kMlpHidden, j = i % kMlpHidden;
        float a = 0.0f;
        for (int k = 0; k < kMlpHidden; ++k) a = fmaf(S.d2[s][k], W2[k * kMlpHidden + j], a);
        S.d1[s][j] = a * silu_grad(S.z1[s][j]);
    }
    if (tid < kMlpHidden) {  // dw3, db2
        float a = 0.0f, b = 0.0f;
        for (int s = 0; s < kTile; ++s) {
            a = fmaf(S.dy[s], silu(S.z2[s][tid]), a);
            b += S.d2[s][tid];
        }
        g[kOffW3 + tid] = a;
        g[kOffB2 + tid] = b;
    }
    if (tid == kMlpHidden) {  // db3
        float a = 0.0f;
        for (int s = 0; s < kTile; ++s) a += S.dy[s];
        g[kOffB3] = a;
    }
    __syncthreads();
    for (int i = tid; i < kMlpHidden * kMlpIn; i += kThreads) {  // dW1[j][q]
        const int j = i / kMlpIn, q = i % kMlpIn;
        float a = 0.0f;
        for (int s = 0; s < kTile; ++s) a = fmaf(S.d1[s][j], S.x[s][q], a);
        g[kOffW1 + i] = a;
    }
    if (tid < kMlpHidden) {  // db1
        float a = 0.0f;
        for (int s = 0; s < kTile; ++s) a += S.d1[s][tid];
        g[kOffB1 + tid] = a;
    }
    // per-CTA loss: sum over the tile's threads in a fixed order
    if (tid < kTile) S.dy[tid] = lsum;
    __syncthreads();
    if (tid == 0) {
        float a = 0.0f;
        for (int s = 0; s < kTile; ++s) a += S.dy[s];
        lpart[blockIdx.x] = a;
    }
}

__global__ void mlp_reduce(const float *__restrict__ gpart, const float *__restrict__ lpart, int tiles,
                           float *__restrict__ grad, float *__restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMlpParams) {
        float a = 0.0f;
        for (int b = 0; b < tiles; ++b) a += gpart[(size_t)b * kMlpParams + p];
        grad[p] = a;
    }
    if (p == 0) {
        float a = 0.0f;
        for (int b = 0; b < tiles; ++b) a += lpart[b];
        *loss = a;
    }
}

// Adam (Kingma & Ba): beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
__global__ void mlp_adam(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                         const float *__restrict__ grad, float lr, int step)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpParams) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gp = grad[p];
    const float mp = b1 * m[p] + (1.0f - b1) * gp;
    const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.0f - powf(b1, (float)step));
    const float vh = vp / (1.0f - powf(b2, (float)step));
    params[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__global__ void mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ X, long long n,
                                   float *__restrict__ Y)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h1[kMlpHidden];
    for (int j = 0; j < kMlpHidden; ++j) {
        float z = P[kOffB1 + j];
        for (int q = 0; q < kMlpIn; ++q) z = fmaf(P[kOffW1 + j * kMlpIn + q], X[s * kMlpIn + q], z);
        h1[j] = silu(z);
    }
    float y = P[kOffB3];
    for (int k = 0; k < kMlpHidden; ++k) {
        float z = P[kOffB2 + k];
        for (int j = 0; j < kMlpHidden; ++j) z = fmaf(P[kOffW2 + k * kMlpHidden + j], h1[j], z);
        y = fmaf(P[kOffW3 + k], silu(z), y);
    }
    Y[s] = y;
}

}  // namespace

int mlp_tile_count(long long n) { return (int)((n + kTile - 1) / kTile); }

cudaError_t mlp_loss_grad(const float *params, const float *X, const float *T, long long n, float *gpart,
                          float *lpart, float *grad, float *loss, cudaStream_t stream)
{
    const int tiles = mlp_tile_count(n);
    if (tiles < 1) return cudaErrorInvalidValue;
    const size_t smem = sizeof(TileSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp_tile<<<tiles, kThreads, smem, stream>>>(params, X, T, n, gpart, lpart);
    mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(gpart, lpart, tiles, grad, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam_step(float *params, float *m, float *v, const float *grad, float lr, int step,
                          cudaStream_t stream)
{
    mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, m, v, grad, lr, step);
    return cudaGetLastError();
}

cudaError_t mlp_forward(const float *params, const float *X, long long n, float *Y, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(params, X, n, Y);
    return cudaGetLastError();
}

}  // namespace qtm
