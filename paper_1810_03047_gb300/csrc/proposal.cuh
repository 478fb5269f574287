// proposal.cuh -- the learned jump-time proposal: a small MLP that predicts the
// time left until a trajectory's norm falls to its threshold r (the crossing of
// Algorithm 1, step (B)) from cheap features of the current state.
//
// Features (raw):  f0 = Gamma = <sum_n C_n^dag C_n> = -2 Re<psi|M psi>/<psi|psi>,
// the instantaneous decay rate of the norm (Eq. eqn:probabil:collapse per unit
// time); f1 = dGamma/dt; f2 = <psi|psi>; f3 = log r; f4, f5 = the latest output
// values of the first two observables.  The network sees x = (f - mu) / sd.
// Output: a correction y to the constant-rate estimate, so the proposed time to
// the crossing is  dt = log(<psi|psi> / r) / Gamma * exp(y).
// Architecture: 6 -> 64 -> 64 -> 1, SiLU activations, FP32 weights.
#pragma once

#include <cuda_runtime.h>

namespace qtm {

constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 64;
// parameter block (floats)
constexpr int kOffW1 = 0;                                  // W1[j][i], 64 x 6
constexpr int kOffB1 = kOffW1 + kMlpHidden * kMlpIn;       // 64
constexpr int kOffW2 = kOffB1 + kMlpHidden;                // W2[k][j], 64 x 64
constexpr int kOffB2 = kOffW2 + kMlpHidden * kMlpHidden;   // 64
constexpr int kOffW3 = kOffB2 + kMlpHidden;                // 64
constexpr int kOffB3 = kOffW3 + kMlpHidden;                // 1
constexpr int kMlpParams = kOffB3 + 1;                     // trainable: 4673
constexpr int kOffMu = kMlpParams;                         // feature means, 6
constexpr int kOffSd = kOffMu + kMlpIn;                    // feature scales, 6
constexpr int kMlpBlock = kOffSd + kMlpIn;                 // 4685 floats in all

// One training record per sampled step: 6 raw features, the step's time and
// (filled in at the next jump) the time left to that jump; NaN when the
// trajectory ended before a jump.
constexpr int kRecFloats = 8;

#ifdef __CUDACC__
__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
#endif

// Launchers of the training kernels (proposal.cu).  X: n x 6 standardised
// features, T: n targets (log of the ratio of the true time left to the
// constant-rate estimate).  Loss = mean over the batch of (y - T)^2.
int mlp_tile_count(long long n);
cudaError_t mlp_loss_grad(const float *params, const float *X, const float *T, long long n, float *gpart,
                          float *lpart, float *grad, float *loss, cudaStream_t stream);
cudaError_t mlp_adam_step(float *params, float *m, float *v, const float *grad, float lr, int step,
                          cudaStream_t stream);
// Inference on the host-visible batch path (tests): Y[i] = network output for X[i].
cudaError_t mlp_forward(const float *params, const float *X, long long n, float *Y, cudaStream_t stream);

}  // namespace qtm
