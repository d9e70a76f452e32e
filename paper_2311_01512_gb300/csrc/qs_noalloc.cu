// Pauli-sum expectation value without any allocation by the library.
//
// Who needs this: callers that must not allocate GPU memory.  cudaMalloc and
// cudaFree synchronise the whole device, so a latency-sensitive loop cannot
// afford them; some host programs hand every byte of device memory to their
// own pool or budget and forbid third-party allocations; and a caller that
// only holds a raw device pointer to amplitudes may not want to create a
// handle, which allocates a scratch area and a pinned staging ring.
//
// This entry point takes a raw device pointer and uses a fixed scratch array
// that lives in the library's own device image (g_noalloc_scratch below).
// Every GPU that loads the library keeps that array until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "qs_device.cuh"

namespace {

constexpr int kMaxDevices = 64;

// Layout of the scratch array: the term list, then one partial sum per block
// of the reduction, then the final sum.
constexpr size_t kTermsBytes = sizeof(qsk::PauliTerm) * QS_NOALLOC_MAX_TERMS;
constexpr size_t kPartialsOffset = kTermsBytes;
constexpr size_t kResultOffset = kPartialsOffset + sizeof(double2) * qsk::kReduceBlocks;
constexpr size_t kScratchBytes = kResultOffset + sizeof(double2);

static_assert(kTermsBytes % 256 == 0, "partials must stay 16-byte aligned");

// The shared scratch.  Nothing in it has to start at zero: each call writes the
// term list, stage one writes every partial, stage two overwrites the result.
// Calls that overlap on the GPU (from two streams, or two threads) share this
// array and race; serialise them.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name only stands in for the symbol, so the address is looked up once
// per device with that device current, on the first call made on it.
qs_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QS_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return QS_OK;
}

}  // namespace

extern "C" qs_status qs_expec_pauli_sum_noalloc(const void* d_amps, int num_qubits, int is_density, qs_prec prec,
                                                const int* paulis, const double* coeffs, int num_terms,
                                                void* cuda_stream, double* out) {
  if (!d_amps || !paulis || !coeffs || !out) return QS_ERR_ARG;
  if (prec != QS_C64 && prec != QS_C128) return QS_ERR_ARG;
  if (num_terms < 1 || num_terms > QS_NOALLOC_MAX_TERMS) return QS_ERR_ARG;
  const int ns = is_density ? 2 * num_qubits : num_qubits;
  if (num_qubits < 1 || ns > QS_MAX_STORAGE_QUBITS) return QS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(d_amps) % 256 != 0) return QS_ERR_ALIGN;

  // Term list on the stack: masks of the X/Y (flipped) and Y/Z (sign) qubits.
  qsk::PauliTerm terms[QS_NOALLOC_MAX_TERMS];
  for (int n = 0; n < num_terms; ++n) {
    qsk::PauliTerm t{};
    int num_y = 0;
    for (int q = 0; q < num_qubits; ++q) {
      const int c = paulis[(size_t)n * num_qubits + q];
      if (c < 0 || c > 3) return QS_ERR_ARG;
      if (c == 1 || c == 2) t.xy |= 1ull << q;
      if (c == 2 || c == 3) t.yz |= 1ull << q;
      if (c == 2) ++num_y;
    }
    t.h = coeffs[n];
    t.eta = num_y & 3;
    terms[n] = t;
  }
  // Terms with equal flip masks next to each other: the kernel shares one
  // partner load per run of equal masks.
  std::stable_sort(terms, terms + num_terms,
                   [](const qsk::PauliTerm& x, const qsk::PauliTerm& y) { return x.xy < y.xy; });

  unsigned char* scratch = nullptr;
  qs_status st = scratch_for_current_device(&scratch);
  if (st != QS_OK) return st;
  auto* d_terms = reinterpret_cast<qsk::PauliTerm*>(scratch);
  auto* d_partials = reinterpret_cast<double2*>(scratch + kPartialsOffset);
  auto* d_result = reinterpret_cast<double2*>(scratch + kResultOffset);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

  // The host term list is pageable stack memory: the copy has read it by the
  // time cudaMemcpyAsync returns.
  if (cudaMemcpyAsync(d_terms, terms, sizeof(qsk::PauliTerm) * (size_t)num_terms, cudaMemcpyHostToDevice, stream) !=
      cudaSuccess)
    return QS_ERR_CUDA;
  cudaError_t e = is_density ? qsk::launch_expec_dm(prec, d_amps, num_qubits, d_terms, num_terms, d_partials, stream)
                             : qsk::launch_expec_sv(prec, d_amps, num_qubits, d_terms, num_terms, d_partials, stream, true,
                                                    qsk::make_tile_order(terms, num_terms));
  if (e == cudaSuccess) e = qsk::launch_reduce_final(d_partials, d_result, 0, stream);
  double2 result;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&result, d_result, sizeof(double2), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return QS_ERR_CUDA;
  out[0] = result.x;
  out[1] = result.y;
  return QS_OK;
}
