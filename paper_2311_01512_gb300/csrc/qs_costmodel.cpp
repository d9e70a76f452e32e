// Learned cost model for fusion planning (C ABI, include/qs.h).
//
// A small perceptron (qs_mlp.cu) predicts log(milliseconds) of one kernel
// launch from a fixed feature encoding of the launch: kernel kind, width,
// which qubits it touches, controls, state size and precision.  It is trained
// on timings the simulator itself measures, with the GPU kernels of
// qs_mlp.cu; the planner (qs_circuit_plan_cost) only reads its predictions,
// so the model never changes a result, only the grouping of gates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"
#include "qs_handle.h"
#include "qs_internal.h"

using qsk::kCostFeatures;
using qsk::kCostHidden;
using qsk::kCostParams;

struct qs_costmodel {
  float* d_params = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_grad = nullptr;
  int step = 0;
};

namespace {

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

// Work buffers of one forward/backward pass over B samples.
struct Pass {
  float *X = nullptr, *t = nullptr, *y = nullptr, *z1 = nullptr, *z2 = nullptr, *dy = nullptr, *dz1 = nullptr,
        *dz2 = nullptr;
  int* idx = nullptr;
  int cap = 0;
  ~Pass() {
    for (void* p : {(void*)X, (void*)t, (void*)y, (void*)z1, (void*)z2, (void*)dy, (void*)dz1, (void*)dz2, (void*)idx})
      if (p) cudaFree(p);
  }
  bool alloc(int n, int batch) {
    const size_t H = kCostHidden, F = kCostFeatures;
    cap = batch;
    return cudaMalloc(&X, sizeof(float) * F * n) == cudaSuccess && cudaMalloc(&t, sizeof(float) * n) == cudaSuccess &&
           cudaMalloc(&y, sizeof(float) * batch) == cudaSuccess &&
           cudaMalloc(&z1, sizeof(float) * H * batch) == cudaSuccess &&
           cudaMalloc(&z2, sizeof(float) * H * batch) == cudaSuccess &&
           cudaMalloc(&dy, sizeof(float) * batch) == cudaSuccess &&
           cudaMalloc(&dz1, sizeof(float) * H * batch) == cudaSuccess &&
           cudaMalloc(&dz2, sizeof(float) * H * batch) == cudaSuccess &&
           cudaMalloc(&idx, sizeof(int) * std::max(n, batch)) == cudaSuccess;
  }
};

}  // namespace

extern "C" {

qs_status qs_costmodel_create(unsigned long long seed, qs_costmodel** out) {
  if (!out) return QS_ERR_ARG;
  *out = nullptr;
  qs_costmodel* m = new (std::nothrow) qs_costmodel();
  if (!m) return QS_ERR_OOM;
  const size_t bytes = sizeof(float) * kCostParams;
  if (cudaMalloc(&m->d_params, bytes) != cudaSuccess || cudaMalloc(&m->d_m, bytes) != cudaSuccess ||
      cudaMalloc(&m->d_v, bytes) != cudaSuccess || cudaMalloc(&m->d_grad, bytes) != cudaSuccess) {
    cudaGetLastError();
    qs_costmodel_destroy(m);
    return QS_ERR_OOM;
  }
  // He-uniform initial weights, zero biases (splitmix64 stream from the seed)
  std::vector<float> p(kCostParams, 0.0f);
  uint64_t s = seed;
  const int F = kCostFeatures, H = kCostHidden;
  auto fill = [&](int off, int count, int fan_in) {
    const double lim = std::sqrt(6.0 / fan_in);
    for (int i = 0; i < count; ++i) p[off + i] = (float)((2.0 * uniform01(s) - 1.0) * lim);
  };
  fill(0, H * F, F);
  fill(H * F + H, H * H, H);
  fill(H * F + H + H * H + H, H, H);
  if (cudaMemcpy(m->d_params, p.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->d_m, 0, bytes) != cudaSuccess || cudaMemset(m->d_v, 0, bytes) != cudaSuccess) {
    qs_costmodel_destroy(m);
    return QS_ERR_CUDA;
  }
  *out = m;
  return QS_OK;
}

qs_status qs_costmodel_destroy(qs_costmodel* m) {
  if (!m) return QS_ERR_ARG;
  for (float* p : {m->d_params, m->d_m, m->d_v, m->d_grad})
    if (p) cudaFree(p);
  delete m;
  return QS_OK;
}

qs_status qs_costmodel_get_params(const qs_costmodel* m, float* host, int n) {
  if (!m || !host || n != kCostParams) return QS_ERR_ARG;
  return cudaMemcpy(host, m->d_params, sizeof(float) * n, cudaMemcpyDeviceToHost) == cudaSuccess ? QS_OK
                                                                                                  : QS_ERR_CUDA;
}

qs_status qs_costmodel_set_params(qs_costmodel* m, const float* host, int n) {
  if (!m || !host || n != kCostParams) return QS_ERR_ARG;
  m->step = 0;
  const size_t bytes = sizeof(float) * n;
  if (cudaMemcpy(m->d_params, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->d_m, 0, bytes) != cudaSuccess || cudaMemset(m->d_v, 0, bytes) != cudaSuccess)
    return QS_ERR_CUDA;
  return QS_OK;
}

qs_status qs_costmodel_encode(int kind, int width, unsigned long long qmask, int nctrl, int weight,
                              const qs_state* s, float* out) {
  if (!out || !s || kind < 0 || kind > QS_COST_PHASE || width < 0 || width > 6) return QS_ERR_ARG;
  std::memset(out, 0, sizeof(float) * kCostFeatures);
  out[kind] = 1.0f;
  if (width >= 1) out[6 + width - 1] = 1.0f;
  out[12] = (float)nctrl / 6.0f;
  for (int q = 0; q < 34; ++q)
    if (qmask >> q & 1ull) out[13 + q] = 1.0f;
  out[47] = (float)s->ns / 34.0f;
  out[48] = s->prec == QS_C128 ? 1.0f : 0.0f;
  out[49] = s->is_density ? 1.0f : 0.0f;
  // complex128 off the FP64 pipe (double-float or block fixed point)
  out[50] = (s->prec == QS_C128 && s->arith != QS_ARITH_F64) ? 1.0f : 0.0f;
  // dense launches that run on the tensor-core kernels (complex64: 2..6 targets;
  // complex128 with double-float or block fixed point: 2..5)
  const bool tc_prec = s->prec == QS_C64 || s->arith != QS_ARITH_F64;
  const int tc_max = s->prec == QS_C64 ? 6 : 5;
  out[51] = (tc_prec && s->tensor_cores && (kind == QS_COST_FUSED_DENSE || kind == QS_COST_DENSE) && width >= 2 &&
             width <= tc_max)
                ? 1.0f
                : 0.0f;
  out[52] = (float)weight / 34.0f;
  return QS_OK;
}

qs_status qs_costmodel_predict(qs_costmodel* m, const float* X, int n, float* out) {
  if (!m || !X || !out || n < 0) return QS_ERR_ARG;
  if (n == 0) return QS_OK;
  float *dX = nullptr, *dy = nullptr;
  qs_status st = QS_OK;
  if (cudaMalloc(&dX, sizeof(float) * kCostFeatures * n) != cudaSuccess ||
      cudaMalloc(&dy, sizeof(float) * n) != cudaSuccess) {
    st = QS_ERR_OOM;
  } else if (cudaMemcpy(dX, X, sizeof(float) * kCostFeatures * n, cudaMemcpyHostToDevice) != cudaSuccess ||
             qsk::launch_mlp_forward(m->d_params, dX, nullptr, n, dy, nullptr, nullptr, nullptr) != cudaSuccess ||
             cudaMemcpy(out, dy, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    st = QS_ERR_CUDA;
  }
  if (dX) cudaFree(dX);
  if (dy) cudaFree(dy);
  cudaGetLastError();
  return st;
}

qs_status qs_costmodel_gradient(qs_costmodel* m, const float* X, const float* t, int n, float* grad, float* loss) {
  if (!m || !X || !t || !grad || n < 1) return QS_ERR_ARG;
  Pass ps;
  if (!ps.alloc(n, n)) {
    cudaGetLastError();
    return QS_ERR_OOM;
  }
  if (cudaMemcpy(ps.X, X, sizeof(float) * kCostFeatures * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ps.t, t, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      qsk::launch_mlp_forward(m->d_params, ps.X, nullptr, n, ps.y, ps.z1, ps.z2, nullptr) != cudaSuccess ||
      qsk::launch_mlp_backward(m->d_params, ps.X, ps.t, nullptr, n, ps.y, ps.z1, ps.z2, ps.dy, ps.dz1, ps.dz2,
                               m->d_grad, nullptr) != cudaSuccess ||
      cudaMemcpy(grad, m->d_grad, sizeof(float) * kCostParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return QS_ERR_CUDA;
  if (loss) {
    std::vector<float> y(n);
    if (cudaMemcpy(y.data(), ps.y, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return QS_ERR_CUDA;
    double acc = 0.0;
    for (int b = 0; b < n; ++b) acc += ((double)y[b] - t[b]) * ((double)y[b] - t[b]);
    *loss = (float)(acc / n);
  }
  return QS_OK;
}

qs_status qs_costmodel_train(qs_costmodel* m, const float* X, const float* t, int n, int epochs, int batch,
                             float lr, unsigned long long seed, float* final_loss) {
  if (!m || !X || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f)) return QS_ERR_ARG;
  batch = std::min(batch, n);
  Pass ps;
  if (!ps.alloc(n, batch)) {
    cudaGetLastError();
    return QS_ERR_OOM;
  }
  if (cudaMemcpy(ps.X, X, sizeof(float) * kCostFeatures * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ps.t, t, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return QS_ERR_CUDA;
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  uint64_t s = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(s) % (uint64_t)(i + 1)]);
    if (cudaMemcpy(ps.idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) return QS_ERR_CUDA;
    for (int b0 = 0; b0 + batch <= n; b0 += batch) {
      const int* idx = ps.idx + b0;
      m->step += 1;
      if (qsk::launch_mlp_forward(m->d_params, ps.X, idx, batch, ps.y, ps.z1, ps.z2, nullptr) != cudaSuccess ||
          qsk::launch_mlp_backward(m->d_params, ps.X, ps.t, idx, batch, ps.y, ps.z1, ps.z2, ps.dy, ps.dz1, ps.dz2,
                                   m->d_grad, nullptr) != cudaSuccess ||
          qsk::launch_mlp_adam(m->d_params, m->d_grad, m->d_m, m->d_v, m->step, lr, nullptr) != cudaSuccess)
        return QS_ERR_CUDA;
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return QS_ERR_CUDA;
  if (final_loss) {
    std::vector<float> y(n);
    if (qs_costmodel_predict(m, X, n, y.data()) != QS_OK) return QS_ERR_CUDA;
    double acc = 0.0;
    for (int b = 0; b < n; ++b) acc += ((double)y[b] - t[b]) * ((double)y[b] - t[b]);
    *final_loss = (float)(acc / n);
  }
  return QS_OK;
}

}  // extern "C"
