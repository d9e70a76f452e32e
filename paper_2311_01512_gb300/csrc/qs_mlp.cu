// The cost-model network on the GPU: a two-hidden-layer perceptron
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3
// (F = 64 features, H = 64 hidden units, FP32) trained with a mean-squared
// loss and Adam.  Forward, backward and update are this file's kernels; the
// backward pass is deterministic: per-sample deltas first, then one thread per
// parameter sums its gradient over the batch in a fixed order.
//
// Flat parameter layout: W1 [H x F] row-major, b1 [H], W2 [H x H], b2 [H],
// W3 [H], b3 [1].
#include "qs_device.cuh"

namespace qsk {

namespace {
constexpr int F = kCostFeatures;
constexpr int H = kCostHidden;
constexpr int OW1 = 0, OB1 = H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
}  // namespace

// One thread per sample: x -> z1, h1, z2, h2 (stored when not null) -> y.
// Samples are rows idx[b] of X (idx null: row b).
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X,
                                                     const int* __restrict__ idx, int B, float* __restrict__ y,
                                                     float* __restrict__ z1s, float* __restrict__ z2s) {
  __shared__ float w[OB3 + 1];
  for (int e = threadIdx.x; e <= OB3; e += blockDim.x) w[e] = params[e];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int row = idx ? idx[b] : b;
  float x[F], h1[H];
#pragma unroll
  for (int f = 0; f < F; ++f) x[f] = X[(size_t)row * F + f];
#pragma unroll 4
  for (int i = 0; i < H; ++i) {
    float z = w[OB1 + i];
#pragma unroll
    for (int f = 0; f < F; ++f) z = fmaf(w[OW1 + i * F + f], x[f], z);
    if (z1s) z1s[(size_t)b * H + i] = z;
    h1[i] = fmaxf(z, 0.0f);
  }
  float out = w[OB3];
#pragma unroll 4
  for (int i = 0; i < H; ++i) {
    float z = w[OB2 + i];
#pragma unroll
    for (int j = 0; j < H; ++j) z = fmaf(w[OW2 + i * H + j], h1[j], z);
    if (z2s) z2s[(size_t)b * H + i] = z;
    out = fmaf(w[OW3 + i], fmaxf(z, 0.0f), out);
  }
  y[b] = out;
}

// Per-sample deltas of the mean-squared loss: dy = 2 (y - t) / B,
// dz2 = dy W3 . [z2 > 0], dz1 = (W2^T dz2) . [z1 > 0].
__global__ void __launch_bounds__(128) k_mlp_delta(const float* __restrict__ params, const float* __restrict__ t,
                                                   const int* __restrict__ idx, int B, const float* __restrict__ y,
                                                   const float* __restrict__ z1s, const float* __restrict__ z2s,
                                                   float* __restrict__ dy, float* __restrict__ dz1,
                                                   float* __restrict__ dz2) {
  __shared__ float w[OB3 + 1];
  for (int e = threadIdx.x; e <= OB3; e += blockDim.x) w[e] = params[e];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int row = idx ? idx[b] : b;
  const float d = 2.0f * (y[b] - t[row]) / (float)B;
  dy[b] = d;
  float g2[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    g2[i] = z2s[(size_t)b * H + i] > 0.0f ? d * w[OW3 + i] : 0.0f;
    dz2[(size_t)b * H + i] = g2[i];
  }
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < H; ++i) s = fmaf(w[OW2 + i * H + j], g2[i], s);
    dz1[(size_t)b * H + j] = z1s[(size_t)b * H + j] > 0.0f ? s : 0.0f;
  }
}

// One thread per parameter: its gradient summed over the batch in order b = 0..B-1.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* __restrict__ X, const int* __restrict__ idx, int B,
                                                   const float* __restrict__ z1s, const float* __restrict__ z2s,
                                                   const float* __restrict__ dy, const float* __restrict__ dz1,
                                                   const float* __restrict__ dz2, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > OB3) return;
  float s = 0.0f;
  if (p < OB1) {                       // W1[i][f]: dz1[b][i] x[b][f]
    const int i = p / F, f = p % F;
    for (int b = 0; b < B; ++b) s = fmaf(dz1[(size_t)b * H + i], X[(size_t)(idx ? idx[b] : b) * F + f], s);
  } else if (p < OW2) {                // b1[i]
    const int i = p - OB1;
    for (int b = 0; b < B; ++b) s += dz1[(size_t)b * H + i];
  } else if (p < OB2) {                // W2[i][j]: dz2[b][i] h1[b][j]
    const int i = (p - OW2) / H, j = (p - OW2) % H;
    for (int b = 0; b < B; ++b) s = fmaf(dz2[(size_t)b * H + i], fmaxf(z1s[(size_t)b * H + j], 0.0f), s);
  } else if (p < OW3) {                // b2[i]
    const int i = p - OB2;
    for (int b = 0; b < B; ++b) s += dz2[(size_t)b * H + i];
  } else if (p < OB3) {                // W3[i]: dy[b] h2[b][i]
    const int i = p - OW3;
    for (int b = 0; b < B; ++b) s = fmaf(dy[b], fmaxf(z2s[(size_t)b * H + i], 0.0f), s);
  } else {                             // b3
    for (int b = 0; b < B; ++b) s += dy[b];
  }
  grad[p] = s;
}

// Adam (Kingma and Ba, 2015), bias-corrected, one thread per parameter.
__global__ void __launch_bounds__(256) k_mlp_adam(float* __restrict__ params, const float* __restrict__ grad,
                                                  float* __restrict__ m, float* __restrict__ v, int step, float lr,
                                                  float beta1, float beta2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > OB3) return;
  const float g = grad[p];
  const float mm = beta1 * m[p] + (1.0f - beta1) * g;
  const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mhat = mm / (1.0f - powf(beta1, (float)step));
  const float vhat = vv / (1.0f - powf(beta2, (float)step));
  params[p] -= lr * mhat / (sqrtf(vhat) + eps);
}

cudaError_t launch_mlp_forward(const float* params, const float* X, const int* idx, int B, float* y, float* z1,
                               float* z2, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_mlp_forward<<<(B + 127) / 128, 128, 0, st>>>(params, X, idx, B, y, z1, z2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float* params, const float* X, const float* t, const int* idx, int B,
                                const float* y, const float* z1, const float* z2, float* dy, float* dz1, float* dz2,
                                float* grad, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_mlp_delta<<<(B + 127) / 128, 128, 0, st>>>(params, t, idx, B, y, z1, z2, dy, dz1, dz2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mlp_wgrad<<<(kCostParams + 255) / 256, 256, 0, st>>>(X, idx, B, z1, z2, dy, dz1, dz2, grad);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                            cudaStream_t st) {
  k_mlp_adam<<<(kCostParams + 255) / 256, 256, 0, st>>>(params, grad, m, v, step, lr, 0.9f, 0.999f, 1e-8f);
  return cudaGetLastError();
}

}  // namespace qsk
