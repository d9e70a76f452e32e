// Density-matrix kernels on the Choi vector (Sec. "Distributed density matrix
// algorithms", local parts): decoherence channels, the Kraus superoperator
// build, the partial trace, and state initialisation.
#include "qs_device.cuh"
#include "qs_df.cuh"

namespace qsk {

// ---------------------------------------------------------------------------
// Channels on groups of Choi amplitudes.  A group is every index that differs
// from its base only at the member positions: (t, t+N) for one-qubit channels,
// (t1, t2, t1+N, t2+N) for two-qubit ones.  Member m has bit b of m at
// position mpos[b].  The updates are the paper's equations:
//   dephasing, one qubit  (Sec. "Dephasing channel"): members with bit t !=
//     bit t+N scale by f0 = 1 - 2p;
//   dephasing, two qubits (two-qubit update rule): members with either pair of
//     bits differing scale by f0 = 1 - 4p/3;
//   depolarising, one qubit (Eq. one-qubit depolarising update): members
//     00 and 11 mix, new = f0 self + f1 other (f0 = 1 - 2p/3, f1 = 2p/3);
//     01 and 10 scale by f2 = 1 - 4p/3;
//   depolarising, two qubits (Eq. two-qubit depolarising Choi update):
//     members with both pairs equal (0, 5, 10, 15) mix,
//     new = f0 self + f1 (sum of the other three) (f0 = 1 - 4p/5, f1 = 4p/15);
//     the 12 others scale by f2 = 1 - 16p/15;
//   damping (Eq. damping update): 00 -> 00 + f1 11 (f1 = p); 01, 10 scale by
//     f2 = sqrt(1 - p); 11 scales by f0 = 1 - p;
//   Pauli channel, one qubit (the general form of the depolarising channel,
//     rho -> (1 - px - py - pz) rho + px X rho X + py Y rho Y + pz Z rho Z):
//     00 and 11 mix as new = f0 self + f1 other (f0 = 1 - px - py,
//     f1 = px + py); 01 and 10 mix as new = f2 self + f3 other
//     (f2 = 1 - px - py - 2 pz, f3 = px - py), since on the Choi vector
//     X rho X and Y rho Y both swap the pair and Y rho Y, Z rho Z carry the
//     sign (-1)^(bit t + bit t+N).
// ---------------------------------------------------------------------------
template <typename R, int OP>
__global__ void __launch_bounds__(256) k_group(typename Cplx<R>::T* __restrict__ rho, const __grid_constant__ GroupParams p) {
  using T2 = typename Cplx<R>::T;
  const R f0 = (R)p.f[0], f1 = (R)p.f[1], f2 = (R)p.f[2], f3 = (R)p.f[3];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.ngroups; k += stride) {
    const uint64_t base = insert_zeros(k, p.ins, p.nbits);
    if (OP == G_DEPHASE1 || OP == G_DEPOL1 || OP == G_DAMP || OP == G_PAULI1) {
      const uint64_t b0 = 1ull << p.mpos[0], b1 = 1ull << p.mpos[1];
      const uint64_t i00 = base, i01 = base | b0, i10 = base | b1, i11 = base | b0 | b1;
      if (OP == G_DEPHASE1) {
        T2 a = rho[i01], b = rho[i10];
        rho[i01] = mk<R>(f0 * a.x, f0 * a.y);
        rho[i10] = mk<R>(f0 * b.x, f0 * b.y);
      } else {
        const T2 a = rho[i00], b = rho[i01], c = rho[i10], d = rho[i11];
        if (OP == G_DEPOL1) {
          rho[i00] = mk<R>(f0 * a.x + f1 * d.x, f0 * a.y + f1 * d.y);
          rho[i11] = mk<R>(f0 * d.x + f1 * a.x, f0 * d.y + f1 * a.y);
          rho[i01] = mk<R>(f2 * b.x, f2 * b.y);
          rho[i10] = mk<R>(f2 * c.x, f2 * c.y);
        } else if (OP == G_PAULI1) {
          rho[i00] = mk<R>(f0 * a.x + f1 * d.x, f0 * a.y + f1 * d.y);
          rho[i11] = mk<R>(f0 * d.x + f1 * a.x, f0 * d.y + f1 * a.y);
          rho[i01] = mk<R>(f2 * b.x + f3 * c.x, f2 * b.y + f3 * c.y);
          rho[i10] = mk<R>(f2 * c.x + f3 * b.x, f2 * c.y + f3 * b.y);
        } else {  // damping
          rho[i00] = mk<R>(a.x + f1 * d.x, a.y + f1 * d.y);
          rho[i01] = mk<R>(f2 * b.x, f2 * b.y);
          rho[i10] = mk<R>(f2 * c.x, f2 * c.y);
          rho[i11] = mk<R>(f0 * d.x, f0 * d.y);
        }
      }
    } else {
      uint64_t idx[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        uint64_t v = base;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if ((m >> b) & 1) v |= 1ull << p.mpos[b];
        idx[m] = v;
      }
      if (OP == G_DEPHASE2) {
        // the 12 scaled members (those with t1 or t2 differing between the two
        // halves), loaded in two batches of six before their stores, since a
        // load cannot move above a store to the same array
        constexpr int sc[12] = {1, 2, 3, 4, 6, 7, 8, 9, 11, 12, 13, 14};
#pragma unroll
        for (int b0 = 0; b0 < 12; b0 += 6) {
          T2 a[6];
#pragma unroll
          for (int u = 0; u < 6; ++u) a[u] = rho[idx[sc[b0 + u]]];
#pragma unroll
          for (int u = 0; u < 6; ++u) rho[idx[sc[b0 + u]]] = mk<R>(f0 * a[u].x, f0 * a[u].y);
        }
      } else {  // two-qubit depolarising
        const T2 a = rho[idx[0]], b = rho[idx[5]], c = rho[idx[10]], d = rho[idx[15]];
        rho[idx[0]] = mk<R>(f0 * a.x + f1 * ((b.x + c.x) + d.x), f0 * a.y + f1 * ((b.y + c.y) + d.y));
        rho[idx[5]] = mk<R>(f0 * b.x + f1 * ((a.x + c.x) + d.x), f0 * b.y + f1 * ((a.y + c.y) + d.y));
        rho[idx[10]] = mk<R>(f0 * c.x + f1 * ((a.x + b.x) + d.x), f0 * c.y + f1 * ((a.y + b.y) + d.y));
        rho[idx[15]] = mk<R>(f0 * d.x + f1 * ((a.x + b.x) + c.x), f0 * d.y + f1 * ((a.y + b.y) + c.y));
        constexpr int oth[12] = {1, 2, 3, 4, 6, 7, 8, 9, 11, 12, 13, 14};
#pragma unroll
        for (int b0 = 0; b0 < 12; b0 += 6) {         // loads of a batch before its stores
          T2 x[6];
#pragma unroll
          for (int u = 0; u < 6; ++u) x[u] = rho[idx[oth[b0 + u]]];
#pragma unroll
          for (int u = 0; u < 6; ++u) rho[idx[oth[b0 + u]]] = mk<R>(f2 * x[u].x, f2 * x[u].y);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Partial trace, Sec. "Partial trace", Eqs. (reduced amplitude definition)
// and (index function): beta'_i = sum_v beta_{g(i, v)}.  g(i, v) puts the bits
// of i, in order, at the positions not in t u (t + N) (zero-bit insertion at
// the sorted traced positions) and bit q of v at both t[q] and t[q] + N.
// One thread per output amplitude; the terms are added in increasing v.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_ptrace(const typename Cplx<R>::T* __restrict__ in,
                                                typename Cplx<R>::T* __restrict__ out, const __grid_constant__ PtraceParams p) {
  using T2 = typename Cplx<R>::T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t nv = 1u << p.n;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nout; i += stride) {
    const uint64_t base = insert_zeros(i, p.ins, p.nins);
    R sr = 0, si = 0;
    for (uint32_t v = 0; v < nv; ++v) {
      uint64_t off = 0;
      for (int q = 0; q < p.n; ++q)
        if ((v >> q) & 1u) off |= p.pair_mask[q];
      const T2 x = in[base | off];
      sr += x.x;
      si += x.y;
    }
    out[i] = mk<R>(sr, si);
  }
}

// ---------------------------------------------------------------------------
// Kraus superoperator, Sec. "Kraus map", Eq. (superoperator from a Kraus map):
// S[i 2^n + k, j 2^n + l] = sum_m conj(K_m[i, j]) K_m[k, l], i.e.
// S = sum_m conj(K_m) (x) K_m.  One thread per element of S, FP64, the terms
// added in increasing m.
// ---------------------------------------------------------------------------
__global__ void k_superop(const double* __restrict__ kraus, int num_ops, int n, double* __restrict__ sup) {
  const int d = 1 << n, d2 = d * d;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d2 * d2) return;
  const int r = e / d2, c = e % d2;
  const int i = r / d, k = r % d, j = c / d, l = c % d;
  double sr = 0.0, si = 0.0;
  for (int m = 0; m < num_ops; ++m) {
    const double* km = kraus + (size_t)2 * m * d2;
    const double ar = km[2 * (i * d + j)], ai = -km[2 * (i * d + j) + 1];  // conj(K[i, j])
    const double br = km[2 * (k * d + l)], bi = km[2 * (k * d + l) + 1];   // K[k, l]
    sr += ar * br - ai * bi;
    si += ar * bi + ai * br;
  }
  sup[2 * e] = sr;
  sup[2 * e + 1] = si;
}

// ---------------------------------------------------------------------------
// Pure-state initialisation, Sec. "State representation":
// beta_{j + k 2^N} = w psi_j psi_k^*, written or accumulated.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_dm_from_pure(typename Cplx<R>::T* __restrict__ rho,
                                                      const typename Cplx<R>::T* __restrict__ psi, int nq,
                                                      R w, int accumulate) {
  using T2 = typename Cplx<R>::T;
  const uint64_t total = 1ull << (2 * nq), mask = (1ull << nq) - 1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const T2 a = psi[i & mask], b = psi[i >> nq];
    R vr = w * (a.x * b.x + a.y * b.y);   // w * a * conj(b)
    R vi = w * (a.y * b.x - a.x * b.y);
    if (accumulate) {
      const T2 o = rho[i];
      vr += o.x;
      vi += o.y;
    }
    rho[i] = mk<R>(vr, vi);
  }
}

// complex128 in double-float: w conj(psi_k) once per element as a pair, then
// two two-term dot products (three when accumulating), each rounded once.
__global__ void __launch_bounds__(256) k_dm_from_pure_df(double2* __restrict__ rho, const double2* __restrict__ psi,
                                                         int nq, qsdf::df w, int accumulate) {
  using qsdf::df;
  const uint64_t total = 1ull << (2 * nq), mask = (1ull << nq) - 1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const df one{1.0f, 0.0f};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const double2 a = psi[i & mask], b = psi[i >> nq];
    const df ar = qsdf::split(a.x), ai = qsdf::split(a.y);
    const df cr = qsdf::dot_result(qsdf::dot_first(w, qsdf::split(b.x)));   // c = w psi_k
    const df ci = qsdf::dot_result(qsdf::dot_first(w, qsdf::split(b.y)));
    qsdf::dot_acc re = qsdf::dot_first(ar, cr);   // a conj(c)
    qsdf::dot_add(re, ai, ci);
    qsdf::dot_acc im = qsdf::dot_first(ai, cr);
    qsdf::dot_add(im, qsdf::neg(ar), ci);
    if (accumulate) {
      const double2 o = rho[i];
      qsdf::dot_add(re, qsdf::split(o.x), one);
      qsdf::dot_add(im, qsdf::split(o.y), one);
    }
    rho[i] = make_double2(qsdf::finish(re), qsdf::finish(im));
  }
}

template <typename R>
__global__ void k_set_first_one(typename Cplx<R>::T* amps) {
  amps[0] = mk<R>((R)1, (R)0);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename R>
static cudaError_t group_t(void* amps, int op, const GroupParams& p, cudaStream_t st) {
  using T2 = typename Cplx<R>::T;
  T2* a = static_cast<T2*>(amps);
  const unsigned g = grid_for(p.ngroups, 256, num_sms() * kStreamBlocksPerSM);
  switch (op) {
    case G_DEPHASE1: k_group<R, G_DEPHASE1><<<g, 256, 0, st>>>(a, p); break;
    case G_DEPHASE2: k_group<R, G_DEPHASE2><<<g, 256, 0, st>>>(a, p); break;
    case G_DEPOL1: k_group<R, G_DEPOL1><<<g, 256, 0, st>>>(a, p); break;
    case G_DEPOL2: k_group<R, G_DEPOL2><<<g, 256, 0, st>>>(a, p); break;
    case G_DAMP: k_group<R, G_DAMP><<<g, 256, 0, st>>>(a, p); break;
    case G_PAULI1: k_group<R, G_PAULI1><<<g, 256, 0, st>>>(a, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_group(qs_prec prec, void* amps, int op, const GroupParams& p, cudaStream_t st) {
  return prec == QS_C128 ? group_t<double>(amps, op, p, st) : group_t<float>(amps, op, p, st);
}

cudaError_t launch_ptrace(qs_prec prec, const void* in, void* out, const PtraceParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.nout, 256, num_sms() * kStreamBlocksPerSM);
  if (prec == QS_C128)
    k_ptrace<double><<<g, 256, 0, st>>>(static_cast<const double2*>(in), static_cast<double2*>(out), p);
  else
    k_ptrace<float><<<g, 256, 0, st>>>(static_cast<const float2*>(in), static_cast<float2*>(out), p);
  return cudaGetLastError();
}

cudaError_t launch_superop(const double* kraus, int num_ops, int n, double* sup, cudaStream_t st) {
  const int total = 1 << (4 * n);
  k_superop<<<(total + 255) / 256, 256, 0, st>>>(kraus, num_ops, n, sup);
  return cudaGetLastError();
}

cudaError_t launch_dm_from_pure(qs_prec prec, void* rho, const void* psi, int nq, double weight,
                                int accumulate, cudaStream_t st, bool f64) {
  const unsigned g = grid_for(1ull << (2 * nq), 256, num_sms() * kStreamBlocksPerSM);
  if (prec == QS_C128 && f64)
    k_dm_from_pure<double><<<g, 256, 0, st>>>(static_cast<double2*>(rho), static_cast<const double2*>(psi), nq,
                                              weight, accumulate);
  else if (prec == QS_C128)
    k_dm_from_pure_df<<<g, 256, 0, st>>>(static_cast<double2*>(rho), static_cast<const double2*>(psi), nq,
                                         qsdf::split_const(weight), accumulate);
  else
    k_dm_from_pure<float><<<g, 256, 0, st>>>(static_cast<float2*>(rho), static_cast<const float2*>(psi), nq,
                                             (float)weight, accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Upload of page-locked host memory by the SMs: 16-byte words from the
// host buffer's mapped device pointer into device memory, four loads in
// flight per thread (grid-stride).  On GB300 both this and the copy engine
// move 16 GiB in 81 ms (211 GB/s over the CPU-GPU link), but the copy
// engine's rate from pinned allocations of small pages was measured to fall
// to 275-690 ms per 16 GiB once other processes had used the GPU, where this
// path kept 81 ms.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_copy16(int4* __restrict__ dst, const int4* __restrict__ src, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const int4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n; i += stride) dst[i] = src[i];
}

cudaError_t launch_copy16(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const size_t n = bytes / 16;
  if (n == 0) return cudaSuccess;
  const unsigned g = grid_for(n, 256, num_sms() * 8);
  k_copy16<<<g, 256, 0, st>>>(static_cast<int4*>(dst), static_cast<const int4*>(src), n);
  return cudaGetLastError();
}

cudaError_t launch_init_zero(qs_prec prec, void* amps, int ns, cudaStream_t st) {
  const size_t bytes = (prec == QS_C128 ? 16 : 8) * (size_t(1) << ns);
  cudaError_t e = cudaMemsetAsync(amps, 0, bytes, st);
  if (e != cudaSuccess) return e;
  if (prec == QS_C128)
    k_set_first_one<double><<<1, 1, 0, st>>>(static_cast<double2*>(amps));
  else
    k_set_first_one<float><<<1, 1, 0, st>>>(static_cast<float2*>(amps));
  return cudaGetLastError();
}

}  // namespace qsk
