// C ABI (include/qs.h): state handles, argument validation, and the host-side
// lowering of each operation to kernel parameters.  All arithmetic on
// amplitudes runs in the CUDA kernels; this file only computes index masks,
// sorted positions, cos/sin of gadget angles and channel coefficients.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"
#include "qs_df.cuh"
#include "qs_superop1.h"
#include "qs_fx.cuh"
#include "qs_alloc.h"
#include "qs_internal.h"

using qsk::kMaxQ;

#include "qs_handle.h"

using qsapi::kRingSlots;
using qsapi::kSlotBytes;

namespace qsapi {

size_t amp_bytes(qs_prec p) { return p == QS_C128 ? 16 : 8; }

qs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? QS_OK : QS_ERR_CUDA; }

// Injected allocation failures (qs_test_fail_allocations): the next
// g_alloc_skip allocations succeed, the g_alloc_fail after them fail.
std::atomic<int> g_alloc_skip{0}, g_alloc_fail{0};

bool injected_failure() {
  if (g_alloc_fail.load() <= 0) return false;
  if (g_alloc_skip.load() > 0) {
    --g_alloc_skip;
    return false;
  }
  --g_alloc_fail;
  return true;
}

void release(qs_state* s) {
  if (!s) return;
  if (s->d_partials) cudaFree(s->d_partials);
  if (s->d_ring) cudaFree(s->d_ring);
  if (s->h_result) cudaFreeHost(s->h_result);
  if (s->h_ring) cudaFreeHost(s->h_ring);
  for (auto& ev : s->ring_ev)
    if (ev) cudaEventDestroy(ev);
  delete s;
}

qs_status create(int nq, int ns, int is_density, qs_prec prec, void* d_amps, void* stream, qs_state** out) {
  if (!out || !d_amps) return QS_ERR_ARG;
  *out = nullptr;
  if (prec != QS_C64 && prec != QS_C128) return QS_ERR_ARG;
  if (nq < 1 || ns > QS_MAX_STORAGE_QUBITS) return QS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_amps) % 256 != 0) return QS_ERR_ALIGN;
  qs_state* s = new (std::nothrow) qs_state();
  if (!s) return QS_ERR_OOM;
  s->amps = d_amps;
  s->nq = nq;
  s->ns = ns;
  s->is_density = is_density;
  s->prec = prec;
  s->stream = static_cast<cudaStream_t>(stream);
  const size_t scratch = sizeof(double2) * (qsk::kPartials + 2);
  if (qsalloc::device(reinterpret_cast<void**>(&s->d_partials), scratch) != cudaSuccess ||
      qsalloc::device(reinterpret_cast<void**>(&s->d_ring), kRingSlots * kSlotBytes) != cudaSuccess ||
      qsalloc::pinned(reinterpret_cast<void**>(&s->h_result), sizeof(double2) * 2) != cudaSuccess ||
      qsalloc::pinned(reinterpret_cast<void**>(&s->h_ring), kRingSlots * kSlotBytes) != cudaSuccess) {
    cudaGetLastError();
    release(s);
    return QS_ERR_OOM;
  }
  s->d_result = s->d_partials + qsk::kPartials;
  s->d_err = reinterpret_cast<int*>(s->d_partials + qsk::kPartials + 1);
  if (cudaMemset(s->d_err, 0, sizeof(int)) != cudaSuccess) {
    release(s);
    return QS_ERR_CUDA;
  }
  for (auto& ev : s->ring_ev) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      release(s);
      return QS_ERR_CUDA;
    }
  }
  *out = s;
  return QS_OK;
}

// ---- recorded programs ------------------------------------------------------
}  // namespace qsapi

// A recorded program: the CUDA graph captured from the state's stream between
// qs_record_begin and qs_record_end, and the device memory its kernels read
// (matrices, Kraus operators, superoperators), which lives as long as the
// program.
struct qs_program {
  qs_state* state = nullptr;
  std::vector<void*> chunks;      // device arena, never moved (the graph holds its addresses)
  size_t used = 0, cap = 0;       // in the last chunk
  cudaStream_t side = nullptr;    // uploads during recording (outside the capture)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace qsapi {

void* rec_alloc(qs_program* p, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (p->chunks.empty() || p->used + bytes > p->cap) {
    const size_t cap = std::max<size_t>(bytes, size_t(4) << 20);
    void* c = nullptr;
    if (qsalloc::device(&c, cap) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    p->chunks.push_back(c);
    p->used = 0;
    p->cap = cap;
  }
  void* d = static_cast<unsigned char*>(p->chunks.back()) + p->used;
  p->used += bytes;
  return d;
}

qs_status rec_put(qs_program* p, const void* host, size_t bytes, const void** dev, int* slot) {
  *slot = -1;
  void* d = rec_alloc(p, bytes);
  if (!d) return QS_ERR_OOM;
  if (cudaMemcpyAsync(d, host, bytes, cudaMemcpyHostToDevice, p->side) != cudaSuccess ||
      cudaStreamSynchronize(p->side) != cudaSuccess)
    return QS_ERR_CUDA;
  *dev = d;
  return QS_OK;
}

void program_free(qs_program* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (void* c : p->chunks) cudaFree(c);
  if (p->side) cudaStreamDestroy(p->side);
  delete p;
}

// Stage `bytes` of host data through the next ring slot and return its device
// copy.  The slot is reused only after the event recorded by its previous user
// has completed.  The caller records the slot's event after queuing the
// kernels that read it (ring_done).
qs_status ring_put(qs_state* s, const void* host, size_t bytes, const void** dev, int* slot) {
  if (bytes > kSlotBytes) return QS_ERR_ARG;
  if (s->rec) return rec_put(s->rec, host, bytes, dev, slot);
  const int k = s->ring_next;
  s->ring_next = (k + 1) % kRingSlots;
  if (cudaEventSynchronize(s->ring_ev[k]) != cudaSuccess) return QS_ERR_CUDA;
  unsigned char* h = s->h_ring + (size_t)k * kSlotBytes;
  unsigned char* d = s->d_ring + (size_t)k * kSlotBytes;
  std::memcpy(h, host, bytes);
  if (cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) return QS_ERR_CUDA;
  *dev = d;
  *slot = k;
  return QS_OK;
}

// A device-side ring slot with no host data (written by a kernel).
qs_status ring_take(qs_state* s, size_t bytes, void** dev, int* slot) {
  if (bytes > kSlotBytes) return QS_ERR_ARG;
  if (s->rec) {
    *slot = -1;
    *dev = rec_alloc(s->rec, bytes);
    return *dev ? QS_OK : QS_ERR_OOM;
  }
  const int k = s->ring_next;
  s->ring_next = (k + 1) % kRingSlots;
  if (cudaEventSynchronize(s->ring_ev[k]) != cudaSuccess) return QS_ERR_CUDA;
  *dev = s->d_ring + (size_t)k * kSlotBytes;
  *slot = k;
  return QS_OK;
}

qs_status ring_done(qs_state* s, int slot) {
  if (slot < 0) return QS_OK;      // arena data of a recorded program: nothing to release
  return cuda_status(cudaEventRecord(s->ring_ev[slot], s->stream));
}

// Validate qubits: each in [0, nq), no repeats within a list, targets and
// controls disjoint (Sec. "Many-control one-target gate": t not in c).
qs_status check_qubits(int nq, const int* targs, int ntarg, const int* ctrls, int nctrl) {
  if (ntarg < 0 || nctrl < 0) return QS_ERR_ARG;
  if ((ntarg > 0 && !targs) || (nctrl > 0 && !ctrls)) return QS_ERR_ARG;
  uint64_t tm = 0, cm = 0;
  for (int i = 0; i < ntarg; ++i) {
    if (targs[i] < 0 || targs[i] >= nq) return QS_ERR_QUBIT_RANGE;
    if (tm >> targs[i] & 1) return QS_ERR_DUP_QUBIT;
    tm |= 1ull << targs[i];
  }
  for (int i = 0; i < nctrl; ++i) {
    if (ctrls[i] < 0 || ctrls[i] >= nq) return QS_ERR_QUBIT_RANGE;
    if (cm >> ctrls[i] & 1) return QS_ERR_DUP_QUBIT;
    cm |= 1ull << ctrls[i];
  }
  if (tm & cm) return QS_ERR_TARGET_IS_CTRL;
  return QS_OK;
}

qs_status check_prob(double p) { return (p >= 0.0 && p <= 1.0) ? QS_OK : QS_ERR_ARG; }

// Block fixed-point constants (qs_fx.cuh): the largest biased exponent of a
// row group, and one constant's 60-bit parts in that group.
int fx_em(std::initializer_list<double> v) {
  int e = 0;
  for (double x : v) e = std::max(e, qsfx::expo_of(x));
  return e;
}
qsk::FxPart fx_part(double v, int em) {
  const qsfx::Part q = qsfx::fixed_const(v, em);
  return qsk::FxPart{q.h, q.l};
}
bool is_fx(const qs_state* s) { return s->prec == QS_C128 && s->arith == QS_ARITH_FX; }

// One dense or one-target gate pass on storage positions (already shifted).
qs_status gate_pass(qs_state* s, const std::vector<int>& ctrls, const std::vector<int>& targs, const double* host_mat,
                    const void* dev_mat, int conj, bool force_dense) {
  const int n = (int)targs.size();
  uint64_t cmask = 0;
  for (int c : ctrls) cmask |= 1ull << c;
  const bool df = s->prec == QS_C128 && s->arith == QS_ARITH_DF;
  if (n == 1 && is_fx(s) && !force_dense) {
    // rows (out0.re, out0.im, out1.re, out1.im) over (a.re, a.im, b.re, b.im)
    double m[8];
    for (int e = 0; e < 8; ++e) m[e] = (conj && (e & 1)) ? -host_mat[e] : host_mat[e];
    const double rows[4][4] = {{m[0], -m[1], m[2], -m[3]}, {m[1], m[0], m[3], m[2]},
                               {m[4], -m[5], m[6], -m[7]}, {m[5], m[4], m[7], m[6]}};
    qsk::Gate1FxParams p{};
    p.em[0] = fx_em({m[0], m[1], m[2], m[3]});
    p.em[1] = fx_em({m[4], m[5], m[6], m[7]});
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) p.m[r][c] = fx_part(rows[r][c], p.em[r >> 1]);
    std::vector<int> ins(ctrls);
    ins.push_back(targs[0]);
    std::sort(ins.begin(), ins.end());
    p.nins = (int)ins.size();
    for (int i = 0; i < p.nins; ++i) p.ins[i] = (int8_t)ins[i];
    p.t = targs[0];
    p.ctrl_mask = cmask;
    p.npairs = 1ull << (s->ns - p.nins);
    return cuda_status(qsk::launch_gate1_fx(s->amps, p, s->stream));
  }
  if (n == 2 && is_fx(s) && host_mat && !force_dense) {
    // u_jk = mat[4 j + k] (conjugated when conj); rows (out_j.re, out_j.im)
    // over (a_k.re, a_k.im), k = 0..3
    qsk::Gate2FxParams p{};
    for (int j = 0; j < 4; ++j) {
      double ur[4], ui[4];
      for (int k = 0; k < 4; ++k) {
        ur[k] = host_mat[2 * (4 * j + k)];
        ui[k] = conj ? -host_mat[2 * (4 * j + k) + 1] : host_mat[2 * (4 * j + k) + 1];
      }
      p.em[j] = fx_em({ur[0], ui[0], ur[1], ui[1], ur[2], ui[2], ur[3], ui[3]});
      for (int k = 0; k < 4; ++k) {
        p.m[2 * j][2 * k] = fx_part(ur[k], p.em[j]);
        p.m[2 * j][2 * k + 1] = fx_part(-ui[k], p.em[j]);
        p.m[2 * j + 1][2 * k] = fx_part(ui[k], p.em[j]);
        p.m[2 * j + 1][2 * k + 1] = fx_part(ur[k], p.em[j]);
      }
    }
    std::vector<int> ins(ctrls);
    ins.push_back(targs[0]);
    ins.push_back(targs[1]);
    std::sort(ins.begin(), ins.end());
    p.nins = (int)ins.size();
    for (int i = 0; i < p.nins; ++i) p.ins[i] = (int8_t)ins[i];
    p.t0 = targs[0];
    p.t1 = targs[1];
    p.lo = std::min(targs[0], targs[1]);
    p.hi = std::max(targs[0], targs[1]);
    p.ctrl_mask = cmask;
    p.nquads = 1ull << (s->ns - p.nins);
    return cuda_status(qsk::launch_gate2_fx(s->amps, p, s->stream));
  }
  if (n == 1 && df && !force_dense) {
    qsk::Gate1DfParams p{};
    for (int e = 0; e < 8; ++e) {
      const double v = (conj && (e & 1)) ? -host_mat[e] : host_mat[e];
      const qsdf::df sv = qsdf::split_const(v);
      p.mh[e] = sv.h;
      p.ml[e] = sv.l;
      p.m[e] = v;
    }
    std::vector<int> ins(ctrls);
    ins.push_back(targs[0]);
    std::sort(ins.begin(), ins.end());
    p.nins = (int)ins.size();
    for (int i = 0; i < p.nins; ++i) p.ins[i] = (int8_t)ins[i];
    p.t = targs[0];
    p.ctrl_mask = cmask;
    p.npairs = 1ull << (s->ns - p.nins);
    p.f64_mod = 16;
    p.f64_count = s->f64_share;
    return cuda_status(qsk::launch_gate1_df(s->amps, p, s->stream));
  }
  if (n == 1 && !force_dense) {
    qsk::Gate1Params p{};
    for (int e = 0; e < 4; ++e) {
      p.m[2 * e] = host_mat[2 * e];
      p.m[2 * e + 1] = conj ? -host_mat[2 * e + 1] : host_mat[2 * e + 1];
    }
    std::vector<int> ins(ctrls);
    ins.push_back(targs[0]);
    std::sort(ins.begin(), ins.end());
    p.nins = (int)ins.size();
    for (int i = 0; i < p.nins; ++i) p.ins[i] = (int8_t)ins[i];
    p.t = targs[0];
    p.ctrl_mask = cmask;
    p.npairs = 1ull << (s->ns - p.nins);
    return cuda_status(qsk::launch_gate1(s->prec, s->amps, p, s->stream));
  }
  uint64_t fixed = cmask;
  for (int t : targs) fixed |= 1ull << t;
  const int nfree = s->ns - n - (int)ctrls.size();
  // two targets run on the three-target tensor-core kernels with an identity
  // on the lowest free qubit
  const bool tc_n = n <= 5 && (n >= 3 || (n == 2 && nfree >= 1));
  const bool tc64 = s->prec == QS_C64 && s->tensor_cores && (tc_n || n == 6);   // 6: bf16x3 slices
  // complex128: seven integer slices (49 bits) with double-float arithmetic,
  // eight (56 bits) with block fixed point
  const bool tc128 = s->prec == QS_C128 && (s->arith == QS_ARITH_DF || s->arith == QS_ARITH_FX) &&
                     s->tensor_cores && tc_n;
  if (tc64 || tc128) {
    std::vector<int> kt(targs);
    if (n == 2) {
      int f = 0;
      while (fixed >> f & 1) ++f;
      kt.push_back(f);
      fixed |= 1ull << f;
    }
    const int nk = (int)kt.size();
    // tensor-core tile: 128 groups, P = kernel targets u the 7 lowest free qubits
    const int g = std::min(7, s->ns - nk - (int)ctrls.size());
    std::vector<int> P(kt);
    for (int q = 0, added = 0; q < s->ns && added < g; ++q)
      if (!(fixed >> q & 1)) {
        P.push_back(q);
        ++added;
      }
    std::sort(P.begin(), P.end());
    qsk::TcParams p{};
    p.mat = static_cast<const double*>(dev_mat);
    p.err = s->d_err;
    p.ctrl_mask = cmask;
    p.n = nk;
    p.nmat = n;
    p.conj = conj;
    p.tile_bits = (int)P.size();
    for (int b = 0; b < p.tile_bits; ++b) p.P[b] = (int8_t)P[b];
    for (int q = 0; q < nk; ++q) {
      p.tslot[q] = (int8_t)(std::find(P.begin(), P.end(), kt[q]) - P.begin());
      p.tslot_mask |= 1u << p.tslot[q];
      p.tpos[q] = (int8_t)kt[q];
    }
    std::vector<int> hi(P);
    hi.insert(hi.end(), ctrls.begin(), ctrls.end());
    std::sort(hi.begin(), hi.end());
    p.nhi = (int)hi.size();
    for (int i = 0; i < p.nhi; ++i) p.hi_ins[i] = (int8_t)hi[i];
    p.ntiles = 1ull << (s->ns - p.nhi);
    return cuda_status(tc64 ? qsk::launch_dense_tc(s->amps, p, s->stream)
                            : qsk::launch_dense_ozaki(s->amps, p, s->arith == QS_ARITH_FX ? 8 : 7, s->stream));
  }
  // Dense tile: P = targets u the lowest free qubits, |P| = min(kTileBits, free + n).
  const int g = std::min(qsk::kTileBits - n, nfree) < 0 ? 0 : std::min(qsk::kTileBits - n, nfree);
  std::vector<int> P(targs);
  for (int q = 0, added = 0; q < s->ns && added < g; ++q)
    if (!(fixed >> q & 1)) {
      P.push_back(q);
      ++added;
    }
  std::sort(P.begin(), P.end());
  qsk::DenseParams p{};
  p.mat = static_cast<const double*>(dev_mat);
  p.ctrl_mask = cmask;
  p.n = n;
  p.conj = conj;
  p.tile_bits = (int)P.size();
  for (int b = 0; b < p.tile_bits; ++b) p.P[b] = (int8_t)P[b];
  for (int q = 0; q < n; ++q)
    p.tslot[q] = (int8_t)(std::find(P.begin(), P.end(), targs[q]) - P.begin());
  std::vector<int> hi(P);
  hi.insert(hi.end(), ctrls.begin(), ctrls.end());
  std::sort(hi.begin(), hi.end());
  p.nhi = (int)hi.size();
  for (int i = 0; i < p.nhi; ++i) p.hi_ins[i] = (int8_t)hi[i];
  p.ntiles = 1ull << (s->ns - p.nhi);
  if (df) return cuda_status(qsk::launch_dense_df(s->amps, p, s->stream));
  return cuda_status(qsk::launch_dense(s->prec, s->amps, p, s->stream));
}

qs_status gadget_pass(qs_state* s, const std::vector<int>& targs, const int* paulis, double theta) {
  qsk::GadgetParams p{};
  int num_y = 0;
  for (size_t q = 0; q < targs.size(); ++q) {
    const int c = paulis[q];
    if (c == 1 || c == 2) p.xy |= 1ull << targs[q];
    if (c == 2 || c == 3) p.yz |= 1ull << targs[q];
    if (c == 2) ++num_y;
  }
  const double phi = -0.5 * theta;
  p.c = std::cos(phi);
  p.s = std::sin(phi);
  p.eta = num_y & 3;
  if (p.xy) {
    p.h = 63 - __builtin_clzll(p.xy);
    p.nwork = 1ull << (s->ns - 1);
  } else {
    p.h = 0;
    p.nwork = 1ull << s->ns;
  }
  if (is_fx(s)) {
    qsk::GadgetFxParams q{};
    q.xy = p.xy;
    q.yz = p.yz;
    q.nwork = p.nwork;
    q.em = fx_em({p.c, p.s});
    q.c = fx_part(p.c, q.em);
    q.s = fx_part(p.s, q.em);
    q.ns = fx_part(-p.s, q.em);
    q.eta = p.eta;
    q.h = p.h;
    return cuda_status(qsk::launch_gadget_fx(s->amps, q, s->stream));
  }
  if (s->prec == QS_C128 && s->arith == QS_ARITH_DF) {
    qsk::GadgetDfParams q{};
    q.xy = p.xy;
    q.yz = p.yz;
    q.nwork = p.nwork;
    const qsdf::df c = qsdf::split_const(p.c), sn = qsdf::split_const(p.s);
    q.ch = c.h;
    q.cl = c.l;
    q.sh = sn.h;
    q.sl = sn.l;
    q.eta = p.eta;
    q.h = p.h;
    return cuda_status(qsk::launch_gadget_df(s->amps, q, s->stream));
  }
  return cuda_status(qsk::launch_gadget(s->prec, s->amps, p, s->stream));
}

qs_status reduce_to_host(qs_state* s, double* out) {
  if (cudaMemcpyAsync(s->h_result, s->d_result, sizeof(double2), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return QS_ERR_CUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return QS_ERR_CUDA;
  out[0] = s->h_result[0].x;
  out[1] = s->h_result[0].y;
  return QS_OK;
}

}  // namespace qsapi

using namespace qsapi;

cudaError_t qsalloc::device(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t qsalloc::pinned(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}


extern "C" {

qs_status qs_test_fail_allocations(int skip, int count) {
  if (skip < 0 || count < 0) return QS_ERR_ARG;
  g_alloc_fail.store(0);
  g_alloc_skip.store(skip);
  g_alloc_fail.store(count);
  return QS_OK;
}

qs_status qs_test_set_error_word(qs_state* s) {
  if (!s || s->rec) return QS_ERR_ARG;
  const int one = 1;
  if (cudaMemcpyAsync(s->d_err, &one, sizeof(int), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return QS_ERR_CUDA;
  return QS_OK;
}

qs_status qs_test_bounded_wait(qs_state* s, unsigned polls) {
  if (!s || s->rec || polls > (1u << 20)) return QS_ERR_ARG;
  return cuda_status(qsk::launch_test_wait_timeout(s->d_err, polls, s->stream));
}

const char* qs_status_str(qs_status status) {
  switch (status) {
    case QS_OK: return "ok";
    case QS_ERR_ARG: return "invalid argument";
    case QS_ERR_QUBIT_RANGE: return "qubit index out of range";
    case QS_ERR_DUP_QUBIT: return "repeated qubit";
    case QS_ERR_TARGET_IS_CTRL: return "qubit is both target and control";
    case QS_ERR_TOO_MANY_TARGETS: return "too many targets";
    case QS_ERR_NOT_DENSMATR: return "operation needs a density matrix";
    case QS_ERR_OOM: return "library scratch allocation failed";
    case QS_ERR_CUDA: return "CUDA runtime error";
    case QS_ERR_TIMEOUT: return "bounded device wait ran out";
    case QS_ERR_ALIGN: return "device pointer not 256-byte aligned";
  }
  return "unknown status";
}

qs_status qs_create_statevector(int num_qubits, qs_prec prec, void* d_amps, void* cuda_stream, qs_state** out) {
  return create(num_qubits, num_qubits, 0, prec, d_amps, cuda_stream, out);
}

qs_status qs_create_densmatr(int num_qubits, qs_prec prec, void* d_amps, void* cuda_stream, qs_state** out) {
  if (num_qubits < 1 || 2 * num_qubits > QS_MAX_STORAGE_QUBITS) {
    if (out) *out = nullptr;
    return QS_ERR_ARG;
  }
  return create(num_qubits, 2 * num_qubits, 1, prec, d_amps, cuda_stream, out);
}

qs_status qs_destroy(qs_state* state) {
  if (!state || state->rec) return QS_ERR_ARG;
  const cudaError_t e = cudaStreamSynchronize(state->stream);
  release(state);
  return cuda_status(e);
}

qs_status qs_get_info(const qs_state* s, int* num_qubits, int* storage_qubits, int* is_density, int* prec) {
  if (!s) return QS_ERR_ARG;
  if (num_qubits) *num_qubits = s->nq;
  if (storage_qubits) *storage_qubits = s->ns;
  if (is_density) *is_density = s->is_density;
  if (prec) *prec = (int)s->prec;
  return QS_OK;
}

qs_status qs_set_arithmetic(qs_state* s, qs_arith arith, int f64_share_16ths) {
  if (!s || (arith != QS_ARITH_DF && arith != QS_ARITH_F64 && arith != QS_ARITH_FX)) return QS_ERR_ARG;
  if (f64_share_16ths < 0 || f64_share_16ths > 16) return QS_ERR_ARG;
  s->arith = arith;
  s->f64_share = f64_share_16ths;
  return QS_OK;
}

qs_status qs_set_tensor_cores(qs_state* s, int enable) {
  if (!s) return QS_ERR_ARG;
  s->tensor_cores = enable ? 1 : 0;
  return QS_OK;
}

qs_status qs_device_ptr(const qs_state* s, void** d_amps) {
  if (!s || !d_amps) return QS_ERR_ARG;
  *d_amps = s->amps;
  return QS_OK;
}

// Uploads of at least this many bytes from page-locked memory use the SM copy.
constexpr size_t kSmCopyMinBytes = size_t(1) << 20;

qs_status qs_set_amps(qs_state* s, const void* host_amps, size_t first, size_t count) {
  if (s && s->rec) return QS_ERR_ARG;   // not while recording
  if (!s || (!host_amps && count)) return QS_ERR_ARG;
  const size_t total = size_t(1) << s->ns;
  if (first > total || count > total - first) return QS_ERR_ARG;
  const size_t b = amp_bytes(s->prec);
  char* dst = static_cast<char*>(s->amps) + first * b;
  const size_t bytes = count * b;
  // Page-locked host memory (pinned allocations, registered ranges) is read by
  // the SMs through its mapped device pointer (qsk::launch_copy16); pageable
  // memory, small copies and unaligned ranges go through the copy engine.
  if (bytes >= kSmCopyMinBytes && bytes % 16 == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, host_amps) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
        attr.devicePointer && reinterpret_cast<uintptr_t>(attr.devicePointer) % 16 == 0)
      return cuda_status(qsk::launch_copy16(dst, attr.devicePointer, bytes, s->stream));
    cudaGetLastError();   // a failed query leaves no sticky error; clear it
  }
  return cuda_status(cudaMemcpyAsync(dst, host_amps, bytes, cudaMemcpyHostToDevice, s->stream));
}

qs_status qs_get_amps(const qs_state* s, void* host_amps, size_t first, size_t count) {
  if (s && s->rec) return QS_ERR_ARG;   // not while recording
  if (!s || (!host_amps && count)) return QS_ERR_ARG;
  const size_t total = size_t(1) << s->ns;
  if (first > total || count > total - first) return QS_ERR_ARG;
  const size_t b = amp_bytes(s->prec);
  if (cudaMemcpyAsync(host_amps, static_cast<const char*>(s->amps) + first * b, count * b, cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess)
    return QS_ERR_CUDA;
  return cuda_status(cudaStreamSynchronize(s->stream));
}

qs_status qs_init_zero(qs_state* s) {
  if (!s) return QS_ERR_ARG;
  return cuda_status(qsk::launch_init_zero(s->prec, s->amps, s->ns, s->stream));
}

qs_status qs_init_pure_densmatr(qs_state* rho, const qs_state* psi, double weight, int accumulate) {
  if (!rho || !psi) return QS_ERR_ARG;
  if (!rho->is_density) return QS_ERR_NOT_DENSMATR;
  if (psi->is_density || psi->nq != rho->nq || psi->prec != rho->prec) return QS_ERR_ARG;
  return cuda_status(qsk::launch_dm_from_pure(rho->prec, rho->amps, psi->amps, rho->nq, weight, accumulate ? 1 : 0,
                                              rho->stream, rho->arith != QS_ARITH_DF));
}

qs_status qs_apply_ctrl_multi_target(qs_state* s, const int* ctrls, int nctrl, const int* targs, int ntarg,
                                     const double* mat) {
  if (!s || !mat) return QS_ERR_ARG;
  if (ntarg < 1) return QS_ERR_ARG;
  if (ntarg > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = check_qubits(s->nq, targs, ntarg, ctrls, nctrl);
  if (st != QS_OK) return st;
  std::vector<int> c(ctrls, ctrls + nctrl), t(targs, targs + ntarg);
  if (s->is_density && nctrl == 0 && ntarg == 1 && is_fx(s)) {
    // U on t and U^* on t + N in one two-target pass of conj(U) (x) U
    double sup[32];
    qsh::superop1(mat, 1, sup);
    return gate_pass(s, {}, {t[0], t[0] + s->nq}, sup, nullptr, 0);
  }
  const size_t mat_bytes = sizeof(double) * 2 * (size_t(1) << (2 * ntarg));
  const void* dmat = nullptr;
  int slot = -1;
  if (ntarg > 1) {
    st = ring_put(s, mat, mat_bytes, &dmat, &slot);
    if (st != QS_OK) return st;
  }
  // Density matrix, uncontrolled two-target unitary on the tensor-core path:
  // U on t and U^* on t + N in one 4-target pass of conj(U) (x) U, the
  // superoperator of the one-operator Kraus map {U} (Sec. "Kraus map"), which
  // reads and writes the Choi vector once instead of twice.
  const bool tc = s->tensor_cores && (s->prec == QS_C64 || s->arith == QS_ARITH_DF || s->arith == QS_ARITH_FX);
  if (s->is_density && nctrl == 0 && ntarg == 2 && tc) {
    void* dsup = nullptr;
    int slot_s = -1;
    st = ring_take(s, sizeof(double) * 2 * 256, &dsup, &slot_s);
    if (st == QS_OK)
      st = cuda_status(qsk::launch_superop(static_cast<const double*>(dmat), 1, 2, static_cast<double*>(dsup),
                                           s->stream));
    if (st == QS_OK) {
      std::vector<int> t4(t);
      for (int q = 0; q < 2; ++q) t4.push_back(t[q] + s->nq);
      st = gate_pass(s, {}, t4, nullptr, dsup, 0);
    }
    const qs_status a = slot_s >= 0 ? ring_done(s, slot_s) : QS_OK;
    const qs_status b = ring_done(s, slot);
    if (st == QS_OK) st = a != QS_OK ? a : b;
    return st;
  }
  st = gate_pass(s, c, t, mat, dmat, 0);
  if (st == QS_OK && s->is_density) {
    // U^* on the same qubits shifted by N (Eq. (unitary on a vectorised density matrix))
    for (int& q : c) q += s->nq;
    for (int& q : t) q += s->nq;
    st = gate_pass(s, c, t, mat, dmat, 1);
  }
  if (slot >= 0) {
    const qs_status st2 = ring_done(s, slot);
    if (st == QS_OK) st = st2;
  }
  return st;
}

qs_status qs_apply_dense_block(qs_state* s, const int* targs, int ntarg, const double* mat) {
  if (!s || !mat) return QS_ERR_ARG;
  if (ntarg < 1) return QS_ERR_ARG;
  if (ntarg > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = check_qubits(s->nq, targs, ntarg, nullptr, 0);
  if (st != QS_OK) return st;
  std::vector<int> t(targs, targs + ntarg);
  const size_t mat_bytes = sizeof(double) * 2 * (size_t(1) << (2 * ntarg));
  const void* dmat = nullptr;
  int slot = -1;
  st = ring_put(s, mat, mat_bytes, &dmat, &slot);
  if (st != QS_OK) return st;
  st = gate_pass(s, {}, t, nullptr, dmat, 0, true);
  if (st == QS_OK && s->is_density) {
    for (int& q : t) q += s->nq;
    st = gate_pass(s, {}, t, nullptr, dmat, 1, true);
  }
  const qs_status st2 = ring_done(s, slot);
  return st != QS_OK ? st : st2;
}

qs_status qs_apply_swap(qs_state* s, int t1, int t2) {
  if (!s) return QS_ERR_ARG;
  const int tt[2] = {t1, t2};
  qs_status st = check_qubits(s->nq, tt, 2, nullptr, 0);
  if (st != QS_OK) return st;
  if (t1 > t2) std::swap(t1, t2);
  st = cuda_status(qsk::launch_swap(s->prec, s->amps, s->ns, t1, t2, s->stream));
  // density matrix: SWAP is real, so SWAP^* on (t1 + N, t2 + N) is SWAP again
  if (st == QS_OK && s->is_density)
    st = cuda_status(qsk::launch_swap(s->prec, s->amps, s->ns, t1 + s->nq, t2 + s->nq, s->stream));
  return st;
}

qs_status qs_apply_diagonal(qs_state* s, const int* targs, int ntarg, const double* diag) {
  if (!s || !diag) return QS_ERR_ARG;
  if (ntarg < 1) return QS_ERR_ARG;
  if (ntarg > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = check_qubits(s->nq, targs, ntarg, nullptr, 0);
  if (st != QS_OK) return st;
  qsk::DiagParams p{};
  p.n = ntarg;
  p.namps = 1ull << s->ns;
  for (int j = 0; j < (1 << ntarg); ++j) {
    p.d[2 * j] = diag[2 * j];
    p.d[2 * j + 1] = diag[2 * j + 1];
  }
  for (int q = 0; q < ntarg; ++q) p.tpos[q] = (int8_t)targs[q];
  const bool df = s->prec == QS_C128 && s->arith == QS_ARITH_DF;
  auto launch = [&]() {
    if (is_fx(s)) {
      qsk::DiagFxParams q{};
      q.n = p.n;
      q.namps = p.namps;
      for (int k = 0; k < p.n; ++k) q.tpos[k] = p.tpos[k];
      for (int j = 0; j < (1 << p.n); ++j) {
        const double re = p.d[2 * j], im = p.d[2 * j + 1];
        qsk::DiagFxEntry& e = q.e[j];
        e.em = fx_em({re, im});
        e.re = fx_part(re, e.em);
        e.im = fx_part(im, e.em);
        e.nim = fx_part(-im, e.em);
      }
      return qsk::launch_diag_fx(s->amps, q, s->stream);
    }
    return df ? qsk::launch_diag_df(s->amps, p, s->stream) : qsk::launch_diag(s->prec, s->amps, p, s->stream);
  };
  st = cuda_status(launch());
  if (st == QS_OK && s->is_density) {
    for (int j = 0; j < (1 << ntarg); ++j) p.d[2 * j + 1] = -diag[2 * j + 1];
    for (int q = 0; q < ntarg; ++q) p.tpos[q] = (int8_t)(targs[q] + s->nq);
    st = cuda_status(launch());
  }
  return st;
}

qs_status qs_apply_pauli_gadget(qs_state* s, const int* targs, const int* paulis, int n, double theta) {
  if (!s || n < 0 || (n > 0 && (!targs || !paulis))) return QS_ERR_ARG;
  qs_status st = check_qubits(s->nq, targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  int num_y = 0;
  for (int q = 0; q < n; ++q) {
    if (paulis[q] < 0 || paulis[q] > 3) return QS_ERR_ARG;
    if (paulis[q] == 2) ++num_y;
  }
  std::vector<int> t(targs, targs + n);
  st = gadget_pass(s, t, paulis, theta);
  if (st == QS_OK && s->is_density) {
    // U(theta)^* = U((-1)^(#Y + 1) theta) (Algorithm "specific unitaries on density matrices")
    for (int& q : t) q += s->nq;
    const double theta2 = (num_y % 2 == 0) ? -theta : theta;
    st = gadget_pass(s, t, paulis, theta2);
  }
  return st;
}

qs_status qs_apply_kraus(qs_state* s, const int* targs, int n, const double* kraus, int num_ops) {
  if (!s || !kraus || num_ops < 1) return QS_ERR_ARG;
  if (!s->is_density) return QS_ERR_NOT_DENSMATR;
  if (n < 1) return QS_ERR_ARG;
  if (2 * n > QS_MAX_DENSE_TARGETS) return QS_ERR_TOO_MANY_TARGETS;
  qs_status st = check_qubits(s->nq, targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  const size_t kbytes = sizeof(double) * 2 * (size_t(1) << (2 * n)) * (size_t)num_ops;
  if (kbytes > kSlotBytes) return QS_ERR_ARG;
  if (n == 1 && is_fx(s)) {
    // S on (t, t + N), one two-target pass with its constants made on the host
    double sup[32];
    qsh::superop1(kraus, num_ops, sup);
    return gate_pass(s, {}, {targs[0], targs[0] + s->nq}, sup, nullptr, 0);
  }
  const void* dk = nullptr;
  void* dsup = nullptr;
  int slot_k = -1, slot_s = -1;
  st = ring_put(s, kraus, kbytes, &dk, &slot_k);
  if (st != QS_OK) return st;
  st = ring_take(s, sizeof(double) * 2 * ((size_t)1 << (4 * n)), &dsup, &slot_s);
  if (st == QS_OK)
    st = cuda_status(qsk::launch_superop(static_cast<const double*>(dk), num_ops, n, static_cast<double*>(dsup),
                                         s->stream));
  if (st == QS_OK) {
    // S on t u (t + N): matrix bit q on t[q], bit n + q on t[q] + N (Sec. "Kraus map")
    std::vector<int> t(targs, targs + n);
    for (int q = 0; q < n; ++q) t.push_back(targs[q] + s->nq);
    st = gate_pass(s, {}, t, nullptr, dsup, 0);
  }
  const qs_status a = ring_done(s, slot_k);
  const qs_status b = slot_s >= 0 ? ring_done(s, slot_s) : QS_OK;
  if (st == QS_OK) st = a != QS_OK ? a : b;
  return st;
}

namespace {

qs_status group_channel(qs_state* s, int op, int t1, int t2, const double* f) {
  if (!s) return QS_ERR_ARG;
  if (!s->is_density) return QS_ERR_NOT_DENSMATR;
  const bool two = (op == qsk::G_DEPHASE2 || op == qsk::G_DEPOL2);
  int tt[2] = {t1, t2};
  qs_status st = check_qubits(s->nq, tt, two ? 2 : 1, nullptr, 0);
  if (st != QS_OK) return st;
  qsk::GroupParams p{};
  std::vector<int> pos;
  if (two)
    pos = {t1, t2, t1 + s->nq, t2 + s->nq};
  else
    pos = {t1, t1 + s->nq};
  p.nbits = (int)pos.size();
  for (int b = 0; b < p.nbits; ++b) p.mpos[b] = (int8_t)pos[b];
  std::sort(pos.begin(), pos.end());
  for (int b = 0; b < p.nbits; ++b) p.ins[b] = (int8_t)pos[b];
  p.ngroups = 1ull << (s->ns - p.nbits);
  for (int k = 0; k < 4; ++k) p.f[k] = f[k];
  // complex128 with double-float arithmetic: channels that mix or scale by
  // non-trivial coefficients use the double-float kernel (the FP64 one is
  // bound by the FP64 pipe, not by memory); dephasing stays on FP64
  if (s->prec == QS_C128 && s->arith == QS_ARITH_DF && op != qsk::G_DEPHASE1 && op != qsk::G_DEPHASE2)
    return cuda_status(qsk::launch_group_df(s->amps, op, p, s->stream));
  // block fixed point: coefficient slots as stated at k_group_fx (coefficients
  // that one output combines share an exponent)
  if (is_fx(s) && op != qsk::G_DEPHASE1 && op != qsk::G_DEPHASE2) {
    qsk::GroupFxParams q{};
    q.ngroups = p.ngroups;
    q.nbits = p.nbits;
    for (int b = 0; b < 4; ++b) {
      q.ins[b] = p.ins[b];
      q.mpos[b] = p.mpos[b];
    }
    double c[4] = {p.f[0], p.f[1], p.f[2], p.f[3]};
    int em[4];
    if (op == qsk::G_DAMP) {
      c[0] = 1.0;
      c[1] = p.f[1];
      c[2] = p.f[2];
      c[3] = p.f[0];
      em[0] = em[1] = fx_em({c[0], c[1]});
      em[2] = fx_em({c[2]});
      em[3] = fx_em({c[3]});
    } else {
      em[0] = em[1] = fx_em({c[0], c[1]});
      em[2] = em[3] = op == qsk::G_PAULI1 ? fx_em({c[2], c[3]}) : fx_em({c[2]});
    }
    for (int k = 0; k < 4; ++k) {
      q.em[k] = em[k];
      q.cf[k] = fx_part(c[k], em[k]);
    }
    return cuda_status(qsk::launch_group_fx(s->amps, op, q, s->stream));
  }
  return cuda_status(qsk::launch_group(s->prec, s->amps, op, p, s->stream));
}

}  // namespace

qs_status qs_apply_dephasing(qs_state* s, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - 2.0 * p, 0.0, 0.0, 0.0};
  return group_channel(s, qsk::G_DEPHASE1, t, t, f);
}

qs_status qs_apply_two_qubit_dephasing(qs_state* s, int t1, int t2, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - 4.0 * p / 3.0, 0.0, 0.0, 0.0};
  return group_channel(s, qsk::G_DEPHASE2, t1, t2, f);
}

qs_status qs_apply_depolarising(qs_state* s, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - 2.0 * p / 3.0, 2.0 * p / 3.0, 1.0 - 4.0 * p / 3.0, 0.0};
  return group_channel(s, qsk::G_DEPOL1, t, t, f);
}

qs_status qs_apply_two_qubit_depolarising(qs_state* s, int t1, int t2, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - 4.0 * p / 5.0, 4.0 * p / 15.0, 1.0 - 16.0 * p / 15.0, 0.0};
  return group_channel(s, qsk::G_DEPOL2, t1, t2, f);
}

qs_status qs_apply_damping(qs_state* s, int t, double p) {
  if (check_prob(p) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - p, p, std::sqrt(1.0 - p), 0.0};
  return group_channel(s, qsk::G_DAMP, t, t, f);
}

qs_status qs_apply_pauli_channel(qs_state* s, int t, double px, double py, double pz) {
  if (check_prob(px) != QS_OK || check_prob(py) != QS_OK || check_prob(pz) != QS_OK) return QS_ERR_ARG;
  const double f[4] = {1.0 - px - py, px + py, 1.0 - px - py - 2.0 * pz, px - py};
  return group_channel(s, qsk::G_PAULI1, t, t, f);
}

qs_status qs_partial_trace(const qs_state* in, const int* targs, int n, void* d_out_amps, qs_state** out) {
  if (in && in->rec) return QS_ERR_ARG;   // not while recording
  if (!in || !out || !d_out_amps) return QS_ERR_ARG;
  *out = nullptr;
  if (!in->is_density) return QS_ERR_NOT_DENSMATR;
  if (n < 1 || n >= in->nq) return QS_ERR_ARG;
  qs_status st = check_qubits(in->nq, targs, n, nullptr, 0);
  if (st != QS_OK) return st;
  if (reinterpret_cast<uintptr_t>(d_out_amps) % 256 != 0) return QS_ERR_ALIGN;
  const int m = in->nq - n;
  qs_state* o = nullptr;
  st = qs_create_densmatr(m, in->prec, d_out_amps, in->stream, &o);
  if (st != QS_OK) return st;
  qsk::PtraceParams p{};
  p.n = n;
  std::vector<int> pos;
  for (int q = 0; q < n; ++q) {
    pos.push_back(targs[q]);
    pos.push_back(targs[q] + in->nq);
    p.pair_mask[q] = (1ull << targs[q]) | (1ull << (targs[q] + in->nq));
  }
  std::sort(pos.begin(), pos.end());
  p.nins = (int)pos.size();
  for (int i = 0; i < p.nins; ++i) p.ins[i] = (int8_t)pos[i];
  p.nout = 1ull << (2 * m);
  st = cuda_status(qsk::launch_ptrace(in->prec, in->amps, d_out_amps, p, in->stream));
  if (st != QS_OK) {
    release(o);
    return st;
  }
  *out = o;
  return QS_OK;
}

qs_status qs_expec_pauli_sum(const qs_state* cs, const int* paulis, const double* coeffs, int num_terms,
                             double* out) {
  if (cs && cs->rec) return QS_ERR_ARG;   // not while recording
  qs_state* s = const_cast<qs_state*>(cs);
  if (!s || !paulis || !coeffs || !out || num_terms < 1) return QS_ERR_ARG;
  std::vector<qsk::PauliTerm> terms((size_t)num_terms);
  for (int n = 0; n < num_terms; ++n) {
    qsk::PauliTerm t{};
    int num_y = 0;
    for (int q = 0; q < s->nq; ++q) {
      const int c = paulis[(size_t)n * s->nq + q];
      if (c < 0 || c > 3) return QS_ERR_ARG;
      if (c == 1 || c == 2) t.xy |= 1ull << q;
      if (c == 2 || c == 3) t.yz |= 1ull << q;
      if (c == 2) ++num_y;
    }
    t.h = coeffs[n];
    t.eta = num_y & 3;
    terms[(size_t)n] = t;
  }
  // statevectors: terms sharing their flip mask become neighbours, so the kernel
  // loads each partner amplitude once per mask (the sum's order changes only)
  if (!s->is_density)
    std::stable_sort(terms.begin(), terms.end(),
                     [](const qsk::PauliTerm& x, const qsk::PauliTerm& y) { return x.xy < y.xy; });
  // statevector: the leading run of diagonal terms (xy = 0 sorts first) goes to
  // the Walsh-Hadamard kernel when it is long enough to pay for the transform
  int ndiag = 0;
  if (!s->is_density)
    while (ndiag < num_terms && terms[(size_t)ndiag].xy == 0) ++ndiag;
  if (s->nq < 5 || ndiag < 8) ndiag = 0;
  for (int first = 0; first < num_terms;) {
    const int lim = first < ndiag ? ndiag : num_terms;
    const int cnt = std::min(qsk::kTermChunk, lim - first);
    const void* dterms = nullptr;
    int slot = -1;
    qs_status st = ring_put(s, terms.data() + first, sizeof(qsk::PauliTerm) * (size_t)cnt, &dterms, &slot);
    if (st != QS_OK) return st;
    const auto* dt = static_cast<const qsk::PauliTerm*>(dterms);
    cudaError_t e;
    if (s->is_density)
      e = qsk::launch_expec_dm(s->prec, s->amps, s->nq, dt, cnt, s->d_partials, s->stream);
    else if (first < ndiag)
      e = qsk::launch_expec_sv_diag(s->prec, s->amps, s->nq, dt, cnt, s->d_partials, s->stream,
                                       s->arith != QS_ARITH_DF);
    else
      e = qsk::launch_expec_sv(s->prec, s->amps, s->nq, dt, cnt, s->d_partials, s->stream, s->arith != QS_ARITH_DF,
                               qsk::make_tile_order(terms.data() + first, cnt));
    if (e == cudaSuccess) e = qsk::launch_reduce_final(s->d_partials, s->d_result, first > 0, s->stream);
    first += cnt;
    st = ring_done(s, slot);
    if (e != cudaSuccess) return QS_ERR_CUDA;
    if (st != QS_OK) return st;
  }
  return reduce_to_host(s, out);
}

qs_status qs_calc_norm_or_trace(const qs_state* cs, double* out) {
  if (cs && cs->rec) return QS_ERR_ARG;   // not while recording
  qs_state* s = const_cast<qs_state*>(cs);
  if (!s || !out) return QS_ERR_ARG;
  cudaError_t e = s->is_density ? qsk::launch_trace(s->prec, s->amps, s->nq, s->d_partials, s->stream)
                                : qsk::launch_norm(s->prec, s->amps, s->ns, s->d_partials, s->stream,
                                                   s->arith != QS_ARITH_DF);
  if (e == cudaSuccess)
    e = qsk::launch_reduce_final(s->d_partials, s->d_result, 0, s->stream,
                                 s->is_density ? qsk::kReduceBlocks : qsk::kNormBlocks);
  if (e != cudaSuccess) return QS_ERR_CUDA;
  return reduce_to_host(s, out);
}

qs_status qs_synchronize(const qs_state* s) {
  if (s && s->rec) return QS_ERR_ARG;   // not while recording
  if (!s) return QS_ERR_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return QS_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return QS_ERR_CUDA;
  if (err) {
    cudaMemset(s->d_err, 0, sizeof(int));
    return QS_ERR_TIMEOUT;
  }
  return QS_OK;
}

qs_status qs_record_begin(qs_state* s) {
  if (!s || s->rec || !s->stream) return QS_ERR_ARG;
  qs_program* p = new (std::nothrow) qs_program();
  if (!p) return QS_ERR_OOM;
  p->state = s;
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    program_free(p);
    return QS_ERR_CUDA;
  }
  if (!rec_alloc(p, 256)) {
    program_free(p);
    return QS_ERR_OOM;
  }
  // relaxed: the uploads on the side stream and arena allocations may run
  // during the capture
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    program_free(p);
    return QS_ERR_CUDA;
  }
  s->rec = p;
  return QS_OK;
}

qs_status qs_record_end(qs_state* s, qs_program** out) {
  if (!s || !s->rec || !out) return QS_ERR_ARG;
  *out = nullptr;
  qs_program* p = s->rec;
  s->rec = nullptr;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  if (e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    program_free(p);
    return QS_ERR_CUDA;
  }
  p->graph = g;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    program_free(p);
    return QS_ERR_CUDA;
  }
  *out = p;
  return QS_OK;
}

qs_status qs_program_run(qs_program* p) {
  if (!p || !p->exec || p->state->rec) return QS_ERR_ARG;
  return cuda_status(cudaGraphLaunch(p->exec, p->state->stream));
}

qs_status qs_program_destroy(qs_program* p) {
  if (!p) return QS_ERR_ARG;
  const cudaError_t e = cudaStreamSynchronize(p->state->stream);
  program_free(p);
  return cuda_status(e);
}

}  // extern "C"
