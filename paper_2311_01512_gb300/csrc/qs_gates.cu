// Unitary-type kernels on a statevector, or on a Choi vector treated as one:
// one-target gates with controls, dense many-target gates, diagonals, and
// Pauli / phase gadgets.
#include "qs_device.cuh"

namespace qsk {

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      cached = 152;
  }
  return cached;
}

// ---------------------------------------------------------------------------
// One-target gate, Sec. "One-target gate" and Sec. "Many-control one-target
// gate": for each of the 2^(Ns-1-s) pairs, i0 has zero bits inserted at the
// target and control positions and the control bits set, i1 = i0 | 2^t;
//   alpha_i0 -> m00 alpha_i0 + m01 alpha_i1,  alpha_i1 -> m10 alpha_i0 + m11 alpha_i1.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_gate1(typename Cplx<R>::T* __restrict__ psi, const __grid_constant__ Gate1Params p) {
  using T2 = typename Cplx<R>::T;
  const R m00r = (R)p.m[0], m00i = (R)p.m[1], m01r = (R)p.m[2], m01i = (R)p.m[3];
  const R m10r = (R)p.m[4], m10i = (R)p.m[5], m11r = (R)p.m[6], m11i = (R)p.m[7];
  const uint64_t tbit = 1ull << p.t;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.npairs; k += stride) {
    const uint64_t i0 = insert_zeros(k, p.ins, p.nins) | p.ctrl_mask;
    const uint64_t i1 = i0 | tbit;
    const T2 a = psi[i0], b = psi[i1];
    T2 r0, r1;
    r0.x = m00r * a.x - m00i * a.y + m01r * b.x - m01i * b.y;
    r0.y = m00r * a.y + m00i * a.x + m01r * b.y + m01i * b.x;
    r1.x = m10r * a.x - m10i * a.y + m11r * b.x - m11i * b.y;
    r1.y = m10r * a.y + m10i * a.x + m11r * b.y + m11i * b.x;
    psi[i0] = r0;
    psi[i1] = r1;
  }
}

// ---------------------------------------------------------------------------
// Dense n-target gate, Sec. "Many-target gate", Eq. (local many-target
// amplitude update): alpha_kj -> sum_l m_jl alpha_kl.  Each CTA stages whole
// groups: a tile is every index that differs from the tile base only at the
// positions P (the n targets and the lowest free qubits), held in shared memory
// in index order so that the global loads and stores are as contiguous as the
// target positions allow.  Element e of a tile has target value
// j = bits of e at the target slots, and its partners share the other bits.
// Persistent: each CTA loads the matrix once and walks tiles.
// ---------------------------------------------------------------------------
template <typename R, int NT>
__global__ void __launch_bounds__(256) k_dense(typename Cplx<R>::T* __restrict__ psi, const __grid_constant__ DenseParams p) {
  using T2 = typename Cplx<R>::T;
  constexpr int D = 1 << NT;
  constexpr int kTile = 1 << kTileBits;
  constexpr int EPT = kTile / 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* sm_mat = reinterpret_cast<T2*>(smem_raw);   // D x D
  T2* sm_tile = sm_mat + D * D;                    // up to kTile
  uint32_t* sm_toff = reinterpret_cast<uint32_t*>(sm_tile + kTile);  // D

  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const double re = p.mat[2 * e];
    const double im = p.conj ? -p.mat[2 * e + 1] : p.mat[2 * e + 1];
    sm_mat[e] = mk<R>((R)re, (R)im);
  }
  for (int l = threadIdx.x; l < D; l += blockDim.x) {
    uint32_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q) off |= ((uint32_t)(l >> q) & 1u) << p.tslot[q];
    sm_toff[l] = off;
  }
  uint32_t tslot_mask = 0;
#pragma unroll
  for (int q = 0; q < NT; ++q) tslot_mask |= 1u << p.tslot[q];
  const int tile = 1 << p.tile_bits;
  __syncthreads();

  for (uint64_t c = blockIdx.x; c < p.ntiles; c += gridDim.x) {
    const uint64_t base = insert_zeros(c, p.hi_ins, p.nhi) | p.ctrl_mask;
    uint64_t gidx[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      uint64_t idx = base;
      for (int b = 0; b < p.tile_bits; ++b) idx |= (uint64_t)((e >> b) & 1) << p.P[b];
      gidx[r] = idx;
      if (e < tile) sm_tile[e] = psi[idx];
    }
    __syncthreads();
    T2 acc[EPT];
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      R ar = 0, ai = 0;
      if (e < tile) {
        int j = 0;
#pragma unroll
        for (int q = 0; q < NT; ++q) j |= ((e >> p.tslot[q]) & 1) << q;
        const uint32_t e0 = (uint32_t)e & ~tslot_mask;
        const T2* mrow = sm_mat + j * D;
#pragma unroll 4
        for (int l = 0; l < D; ++l) {
          const T2 m = mrow[l];
          const T2 x = sm_tile[e0 | sm_toff[l]];
          ar = fma(m.x, x.x, ar);
          ar = fma(-m.y, x.y, ar);
          ai = fma(m.x, x.y, ai);
          ai = fma(m.y, x.x, ai);
        }
      }
      acc[r] = mk<R>(ar, ai);
    }
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int e = threadIdx.x + r * 256;
      if (e < tile) psi[gidx[r]] = acc[r];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Diagonal on n targets: alpha_i -> d_j alpha_i, j = target bits of i.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_diag(typename Cplx<R>::T* __restrict__ psi, const __grid_constant__ DiagParams p) {
  using T2 = typename Cplx<R>::T;
  __shared__ T2 d[64];
  for (int j = threadIdx.x; j < (1 << p.n); j += blockDim.x) d[j] = mk<R>((R)p.d[2 * j], (R)p.d[2 * j + 1]);
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 4) {
    // complex64: two neighbouring amplitudes (16 bytes) per thread and step
    float4* p4 = reinterpret_cast<float4*>(psi);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; 2 * k < p.namps; k += stride) {
      const uint64_t i = 2 * k;
      int j = 0;
      for (int q = 0; q < p.n; ++q) j |= (int)((i >> p.tpos[q]) & 1) << q;
      int j1 = j;
      for (int q = 0; q < p.n; ++q)
        if (p.tpos[q] == 0) j1 |= 1 << q;
      const float4 a = p4[k];
      const T2 w = d[j], w1 = d[j1];
      p4[k] = make_float4(w.x * a.x - w.y * a.y, w.x * a.y + w.y * a.x, w1.x * a.z - w1.y * a.w,
                          w1.x * a.w + w1.y * a.z);
    }
  } else {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.namps; i += stride) {
      int j = 0;
      for (int q = 0; q < p.n; ++q) j |= (int)((i >> p.tpos[q]) & 1) << q;
      const T2 a = psi[i], w = d[j];
      psi[i] = mk<R>(w.x * a.x - w.y * a.y, w.x * a.y + w.y * a.x);
    }
  }
}

// ---------------------------------------------------------------------------
// Pauli gadget, Sec. "Pauli gadget": with phi = -theta/2,
//   alpha_i -> cos(phi) alpha_i + i sin(phi) beta_{i'} alpha_{i'},
// i' = i xor xy, beta_x = eta (-1)^{popc(x & yz)}, eta = i^{#Y}
// (Sec. "Pauli tensor").  Pairs (i, i') are enumerated with the highest bit of
// xy inserted as zero into the pair number.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_gadget(typename Cplx<R>::T* __restrict__ psi, const __grid_constant__ GadgetParams p) {
  using T2 = typename Cplx<R>::T;
  const R c = (R)p.c, s = (R)p.s;
  const int q = (p.eta + 1) & 3;  // i * eta = i^(#Y + 1)
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.nwork; k += stride) {
    const uint64_t i = insert_zero(k, p.h);
    const uint64_t j = i ^ p.xy;
    const T2 a = psi[i], b = psi[j];
    const R sj = parity64(j & p.yz) ? -s : s;
    const R si = parity64(i & p.yz) ? -s : s;
    const T2 rb = rot_i(b, q), ra = rot_i(a, q);
    psi[i] = mk<R>(c * a.x + sj * rb.x, c * a.y + sj * rb.y);
    psi[j] = mk<R>(c * b.x + si * ra.x, c * b.y + si * ra.y);
  }
}

// Phase gadget (only Z factors), Sec. "Phase gadget", Eq. (phase gadget
// amplitude change): alpha_i -> exp(i phi s_i) alpha_i, s_i = (-1)^{popc(i & yz)}.
template <typename R>
__global__ void __launch_bounds__(256) k_phase(typename Cplx<R>::T* __restrict__ psi, const __grid_constant__ GadgetParams p) {
  using T2 = typename Cplx<R>::T;
  const R c = (R)p.c, s = (R)p.s;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 4) {
    // complex64: two neighbouring amplitudes (16 bytes) per thread and step
    float4* p4 = reinterpret_cast<float4*>(psi);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; 2 * k < p.nwork; k += stride) {
      const uint64_t i = 2 * k;
      const R s0 = parity64(i & p.yz) ? -s : s;
      const R s1 = parity64((i + 1) & p.yz) ? -s : s;
      const float4 a = p4[k];
      p4[k] = make_float4(c * a.x - s0 * a.y, c * a.y + s0 * a.x, c * a.z - s1 * a.w, c * a.w + s1 * a.z);
    }
  } else {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.nwork; i += stride) {
      const R si = parity64(i & p.yz) ? -s : s;
      const T2 a = psi[i];
      psi[i] = mk<R>(c * a.x - si * a.y, c * a.y + si * a.x);
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename R>
static cudaError_t gate1_t(void* amps, const Gate1Params& p, cudaStream_t st) {
  const unsigned g = grid_for(p.npairs, 256, num_sms() * kStreamBlocksPerSM);
  k_gate1<R><<<g, 256, 0, st>>>(static_cast<typename Cplx<R>::T*>(amps), p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SWAP (Sec. "Swap gate"): alpha_i -> alpha_{i with bits t1 and t2 flipped}
// where those bits differ.  One thread per pair: the group index k takes zero
// bits at t1 < t2, then the pair is (k | 2^t1, k | 2^t2).  No arithmetic, so
// the same kernel serves complex64 and complex128 (moved as 8- or 16-byte
// words).
// ---------------------------------------------------------------------------
template <typename T2>
__global__ void __launch_bounds__(256) k_swap(T2* __restrict__ psi, uint64_t npairs, int t1, int t2) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t b1 = 1ull << t1, b2 = 1ull << t2;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += stride) {
    const uint64_t base = insert_zero(insert_zero(k, t1), t2);
    const T2 x = psi[base | b1], y = psi[base | b2];
    psi[base | b1] = y;
    psi[base | b2] = x;
  }
}

cudaError_t launch_swap(qs_prec prec, void* amps, int ns, int t1, int t2, cudaStream_t st) {
  const uint64_t npairs = 1ull << (ns - 2);
  const unsigned g = grid_for(npairs, 256, num_sms() * kStreamBlocksPerSM);
  if (prec == QS_C128)
    k_swap<double2><<<g, 256, 0, st>>>(static_cast<double2*>(amps), npairs, t1, t2);
  else
    k_swap<float2><<<g, 256, 0, st>>>(static_cast<float2*>(amps), npairs, t1, t2);
  return cudaGetLastError();
}

cudaError_t launch_gate1(qs_prec prec, void* amps, const Gate1Params& p, cudaStream_t st) {
  return prec == QS_C128 ? gate1_t<double>(amps, p, st) : gate1_t<float>(amps, p, st);
}

template <typename R, int NT>
static cudaError_t dense_nt(void* amps, const DenseParams& p, cudaStream_t st) {
  using T2 = typename Cplx<R>::T;
  constexpr int D = 1 << NT;
  const size_t smem = sizeof(T2) * (D * D + (1 << kTileBits)) + sizeof(uint32_t) * D;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int per_sm = smem > 100 * 1024 ? 1 : (smem > 60 * 1024 ? 2 : 4);
  const uint64_t maxb = (uint64_t)num_sms() * per_sm;
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense<R, NT><<<g, 256, smem, st>>>(static_cast<T2*>(amps), p);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t dense_t(void* amps, const DenseParams& p, cudaStream_t st) {
  switch (p.n) {
    case 1: return dense_nt<R, 1>(amps, p, st);
    case 2: return dense_nt<R, 2>(amps, p, st);
    case 3: return dense_nt<R, 3>(amps, p, st);
    case 4: return dense_nt<R, 4>(amps, p, st);
    case 5: return dense_nt<R, 5>(amps, p, st);
    case 6: return dense_nt<R, 6>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_dense(qs_prec prec, void* amps, const DenseParams& p, cudaStream_t st) {
  return prec == QS_C128 ? dense_t<double>(amps, p, st) : dense_t<float>(amps, p, st);
}

cudaError_t launch_diag(qs_prec prec, void* amps, const DiagParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.namps, 256, num_sms() * kStreamBlocksPerSM);
  if (prec == QS_C128)
    k_diag<double><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
  else
    k_diag<float><<<g, 256, 0, st>>>(static_cast<float2*>(amps), p);
  return cudaGetLastError();
}

cudaError_t launch_gadget(qs_prec prec, void* amps, const GadgetParams& p, cudaStream_t st) {
  const unsigned g = grid_for(p.nwork, 256, num_sms() * kStreamBlocksPerSM);
  if (p.xy == 0) {
    if (prec == QS_C128)
      k_phase<double><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
    else
      k_phase<float><<<g, 256, 0, st>>>(static_cast<float2*>(amps), p);
  } else {
    if (prec == QS_C128)
      k_gadget<double><<<g, 256, 0, st>>>(static_cast<double2*>(amps), p);
    else
      k_gadget<float><<<g, 256, 0, st>>>(static_cast<float2*>(amps), p);
  }
  return cudaGetLastError();
}

}  // namespace qsk
