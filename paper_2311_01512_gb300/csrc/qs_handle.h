// The state handle and the host-side helpers shared by the C-ABI files
// (qs_api.cpp: single operations; qs_circuit.cpp: planned circuits).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "qs.h"

namespace qsapi {

constexpr int kRingSlots = 16;
constexpr size_t kSlotBytes = 64 * 1024;  // one 64 x 64 complex128 matrix

}  // namespace qsapi

struct qs_state {
  void* amps = nullptr;
  int nq = 0;          // N
  int ns = 0;          // storage qubits
  int is_density = 0;
  qs_prec prec = QS_C128;
  qs_arith arith = QS_ARITH_FX;
  int f64_share = 0;     // sixteenths of one-target-gate chunks run in native FP64
  int tensor_cores = 1;  // complex64 dense gates with 3..5 targets on tcgen05
  int* d_err = nullptr;  // device error word (bounded waits that ran out)
  cudaStream_t stream = nullptr;
  // reduction scratch (device) and its pinned host mirror
  double2* d_partials = nullptr;
  double2* d_result = nullptr;
  double2* h_result = nullptr;
  // staging ring for matrices and term lists: pinned host slot -> device slot
  unsigned char* h_ring = nullptr;
  unsigned char* d_ring = nullptr;
  cudaEvent_t ring_ev[qsapi::kRingSlots] = {};
  int ring_next = 0;
  // between qs_record_begin and qs_record_end: the program being recorded
  // (operation data goes to its device arena instead of the ring)
  qs_program* rec = nullptr;
};

namespace qsapi {

qs_status cuda_status(cudaError_t e);
qs_status check_qubits(int nq, const int* targs, int ntarg, const int* ctrls, int nctrl);
qs_status ring_put(qs_state* s, const void* host, size_t bytes, const void** dev, int* slot);
// device scratch for `bytes` written by a kernel (ring slot, or arena while recording)
qs_status ring_take(qs_state* s, size_t bytes, void** dev, int* slot);
qs_status ring_done(qs_state* s, int slot);
// One dense-gate pass on storage positions (already shifted for the conjugate
// pass of a density matrix).  host_mat is needed only for one-target gates
// unless force_dense; dev_mat (complex128, row-major) for more targets.
qs_status gate_pass(qs_state* s, const std::vector<int>& ctrls, const std::vector<int>& targs, const double* host_mat,
                    const void* dev_mat, int conj, bool force_dense = false);
qs_status gadget_pass(qs_state* s, const std::vector<int>& targs, const int* paulis, double theta);

}  // namespace qsapi
