// Batched engine (C ABI, include/qs.h): many independent statevectors with
// their own circuits, run by one persistent kernel launch (qs_batch_kernels.cu)
// that is captured once in a CUDA graph and replayed.
//
// Scheduling: states are ordered by estimated work (amplitudes x operations),
// largest first, and CTAs take them from a shared counter, so the long states
// start early and the short ones fill the gaps (longest-processing-time
// order).  The launch shape (threads per CTA, CTAs per SM, and with it the
// largest state kept in shared memory) is chosen by timing every candidate on
// the batch itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"
#include "qs_handle.h"
#include "qs_internal.h"

struct qs_batch {
  qs_prec prec = QS_C64;
  cudaStream_t stream = nullptr;
  std::vector<int> nq;
  std::vector<size_t> offset;  // amplitudes
  size_t pool_amps = 0;
  void* pool = nullptr;
  std::vector<std::vector<qsk::BatchOp>> progs;
  qsk::BatchState* d_states = nullptr;
  int* d_order = nullptr;
  qsk::BatchOp* d_ops = nullptr;
  int* d_counter = nullptr;
  int threads = 256, ctas = 0, smem_qubits = -1;
  cudaStream_t capture_stream = nullptr;  // own stream for recording (the caller's may be the legacy stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool compiled = false;
  long total_ops = 0;
  float best_ms = 0.f;
};

namespace {

void free_device(qs_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : {(void*)b->d_states, (void*)b->d_order, (void*)b->d_ops, (void*)b->d_counter})
    if (p) cudaFree(p);
  b->exec = nullptr;
  b->graph = nullptr;
  b->d_states = nullptr;
  b->d_order = nullptr;
  b->d_ops = nullptr;
  b->d_counter = nullptr;
  b->compiled = false;
}

qs_status check_state(const qs_batch* b, int s) {
  if (!b || s < 0 || s >= (int)b->nq.size()) return QS_ERR_ARG;
  return QS_OK;
}

qs_status add(qs_batch* b, int s, qsk::BatchOp&& op) {
  b->progs[s].push_back(op);
  b->compiled = false;
  return QS_OK;
}

int smem_qubits_for(qs_prec prec, int ctas_per_sm) {
  const size_t per_cta = std::min<size_t>(200 * 1024 / ctas_per_sm, 200 * 1024);
  const size_t amp = prec == QS_C128 ? 16 : 8;
  int q = 0;
  while (((size_t)1 << (q + 1)) * amp <= per_cta) ++q;
  return q;
}

}  // namespace

extern "C" {

qs_status qs_batch_create(int num_states, const int* num_qubits, qs_prec prec, void* cuda_stream, qs_batch** out) {
  if (!out || num_states < 1 || !num_qubits || (prec != QS_C64 && prec != QS_C128)) return QS_ERR_ARG;
  *out = nullptr;
  qs_batch* b = new (std::nothrow) qs_batch();
  if (!b) return QS_ERR_OOM;
  b->prec = prec;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->nq.assign(num_qubits, num_qubits + num_states);
  b->progs.resize(num_states);
  size_t off = 0;
  for (int q : b->nq) {
    if (q < 1 || q > 24) {
      delete b;
      return QS_ERR_ARG;
    }
    b->offset.push_back(off);
    off += (size_t)1 << q;
    off = (off + 31) & ~(size_t)31;    // 256-byte aligned starts for complex64 and complex128
  }
  b->pool_amps = off;
  *out = b;
  return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* b) {
  if (!b) return QS_ERR_ARG;
  free_device(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return QS_OK;
}

qs_status qs_batch_pool_amps(const qs_batch* b, size_t* num_amps) {
  if (!b || !num_amps) return QS_ERR_ARG;
  *num_amps = b->pool_amps;
  return QS_OK;
}

qs_status qs_batch_state_offset(const qs_batch* b, int state, size_t* offset_amps) {
  if (check_state(b, state) != QS_OK || !offset_amps) return QS_ERR_ARG;
  *offset_amps = b->offset[state];
  return QS_OK;
}

qs_status qs_batch_bind_pool(qs_batch* b, void* d_pool) {
  if (!b || !d_pool) return QS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_pool) % 256 != 0) return QS_ERR_ALIGN;
  b->pool = d_pool;
  b->compiled = false;
  return QS_OK;
}

qs_status qs_batch_add_unitary(qs_batch* b, int state, const int* ctrls, int nctrl, const int* targs, int ntarg,
                               const double* mat) {
  if (check_state(b, state) != QS_OK || !mat || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > 2 || nctrl > 5) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(b->nq[state], targs, ntarg, ctrls, nctrl);
  if (st != QS_OK) return st;
  qsk::BatchOp op{};
  op.kind = 0;
  op.n = ntarg;
  std::vector<int> ins;
  for (int q = 0; q < ntarg; ++q) {
    op.t[q] = targs[q];
    ins.push_back(targs[q]);
  }
  for (int q = 0; q < nctrl; ++q) {
    op.ctrl |= 1u << ctrls[q];
    ins.push_back(ctrls[q]);
  }
  std::sort(ins.begin(), ins.end());
  op.nins = (int)ins.size();
  for (int i = 0; i < op.nins; ++i) op.ins[i] = (int8_t)ins[i];
  std::memcpy(op.m, mat, sizeof(double) * 2 * (1u << (2 * ntarg)));
  return add(b, state, std::move(op));
}

qs_status qs_batch_add_diagonal(qs_batch* b, int state, const int* targs, int ntarg, const double* diag) {
  if (check_state(b, state) != QS_OK || !diag || ntarg < 1) return QS_ERR_ARG;
  if (ntarg > 3) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = qsapi::check_qubits(b->nq[state], targs, ntarg, nullptr, 0);
  if (st != QS_OK) return st;
  qsk::BatchOp op{};
  op.kind = 1;
  op.n = ntarg;
  for (int q = 0; q < ntarg; ++q) op.t[q] = targs[q];
  std::memcpy(op.m, diag, sizeof(double) * 2 * (1u << ntarg));
  return add(b, state, std::move(op));
}

qs_status qs_batch_add_pauli_gadget(qs_batch* b, int state, const int* targs, const int* paulis, int n,
                                    double theta) {
  if (check_state(b, state) != QS_OK || n < 0 || (n > 0 && (!targs || !paulis))) return QS_ERR_ARG;
  qs_status st = qsapi::check_qubits(b->nq[state], targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  qsk::BatchOp op{};
  op.kind = 2;
  int ny = 0;
  for (int q = 0; q < n; ++q) {
    if (paulis[q] < 0 || paulis[q] > 3) return QS_ERR_ARG;
    if (paulis[q] == 1 || paulis[q] == 2) op.xy |= 1u << targs[q];
    if (paulis[q] == 2 || paulis[q] == 3) op.yz |= 1u << targs[q];
    if (paulis[q] == 2) ++ny;
  }
  op.eta = ny & 3;
  op.h = op.xy ? 31 - __builtin_clz(op.xy) : 0;
  const double phi = -0.5 * theta;
  op.c = std::cos(phi);
  op.s = std::sin(phi);
  return add(b, state, std::move(op));
}

qs_status qs_batch_compile(qs_batch* b, int autotune) {
  if (!b || !b->pool) return QS_ERR_ARG;
  free_device(b);
  const int S = (int)b->nq.size();
  std::vector<qsk::BatchState> states(S);
  std::vector<qsk::BatchOp> ops;
  for (int s = 0; s < S; ++s) {
    states[s].offset = b->offset[s];
    states[s].nq = b->nq[s];
    states[s].first_op = (int)ops.size();
    states[s].nops = (int)b->progs[s].size();
    ops.insert(ops.end(), b->progs[s].begin(), b->progs[s].end());
  }
  b->total_ops = (long)ops.size();
  std::vector<int> order(S);
  for (int s = 0; s < S; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return ((double)(1ull << b->nq[x]) * (1 + b->progs[x].size())) >
           ((double)(1ull << b->nq[y]) * (1 + b->progs[y].size()));
  });
  if (cudaMalloc(&b->d_states, sizeof(qsk::BatchState) * S) != cudaSuccess ||
      cudaMalloc(&b->d_order, sizeof(int) * S) != cudaSuccess ||
      cudaMalloc(&b->d_ops, sizeof(qsk::BatchOp) * std::max<size_t>(1, ops.size())) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_device(b);
    return QS_ERR_OOM;
  }
  if (cudaMemcpy(b->d_states, states.data(), sizeof(qsk::BatchState) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!ops.empty() &&
       cudaMemcpy(b->d_ops, ops.data(), sizeof(qsk::BatchOp) * ops.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    free_device(b);
    return QS_ERR_CUDA;
  }
  // launch-shape candidates: (threads, CTAs per SM)
  const int sms = qsk::num_sms();
  if (qsk::batch_set_max_smem(200 * 1024) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  std::vector<std::pair<int, int>> cands;
  if (autotune)
    cands = {{128, 4}, {256, 2}, {256, 4}, {512, 1}, {512, 2}, {1024, 1}};
  else
    cands = {{256, 2}};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (const auto& c : cands) {
    const int sq = smem_qubits_for(b->prec, c.second);
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream) != cudaSuccess) return QS_ERR_CUDA;
    cudaEventRecord(e0, b->stream);
    if (qsk::launch_batch(b->prec, b->pool, b->d_states, b->d_order, S, b->d_ops, b->d_counter, c.first,
                          sms * c.second, sq, b->stream) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return QS_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      b->threads = c.first;
      b->ctas = sms * c.second;
      b->smem_qubits = sq;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (b->ctas == 0) return QS_ERR_CUDA;
  b->best_ms = best;
  // record on the batch's own stream: reset the work counter, one persistent launch
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return QS_ERR_CUDA;
  if (!b->capture_stream && cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return QS_ERR_CUDA;
  if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->capture_stream);
  if (e == cudaSuccess)
    e = qsk::launch_batch(b->prec, b->pool, b->d_states, b->d_order, S, b->d_ops, b->d_counter, b->threads, b->ctas,
                          b->smem_qubits, b->capture_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return QS_ERR_CUDA;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    return QS_ERR_CUDA;
  }
  b->compiled = true;
  return QS_OK;
}

qs_status qs_batch_run(qs_batch* b) {
  if (!b || !b->compiled) return QS_ERR_ARG;
  return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

qs_status qs_batch_info(const qs_batch* b, int* threads, int* ctas, int* smem_qubits, long* total_ops) {
  if (!b) return QS_ERR_ARG;
  if (threads) *threads = b->threads;
  if (ctas) *ctas = b->ctas;
  if (smem_qubits) *smem_qubits = b->smem_qubits;
  if (total_ops) *total_ops = b->total_ops;
  return QS_OK;
}

}  // extern "C"
