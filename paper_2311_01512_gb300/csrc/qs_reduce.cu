// Reductions: norm, trace, and Pauli-sum expectation values.  Stage one runs
// a fixed grid (kNormBlocks for the norm, kReduceBlocks for the others), each
// block writing one complex128 partial sum; stage two adds the partials in a
// fixed order, so results do not depend on scheduling.
#include "qs_device.cuh"
#include "qs_df.cuh"

namespace qsk {

__device__ __forceinline__ qsdf::df to_df(double x) { return qsdf::split(x); }
__device__ __forceinline__ qsdf::df to_df(float x) { return qsdf::df{x, 0.0f}; }

// sum_i |alpha_i|^2 (Sec. "Local statevector algorithms": the state model).
// Each thread sums its squares exactly in double-float (TwoProd squares,
// TwoSum accumulation; no FP64 instruction in the loop) and rounds once; the
// block and stage-two sums are FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_norm(const typename Cplx<R>::T* __restrict__ psi, uint64_t n,
                                              double2* __restrict__ partials) {
  qsdf::dot_acc acc{0.0f, 0.0f};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    // complex64: two amplitudes per 16-byte load (twice the bytes in flight)
    const float4* p4 = reinterpret_cast<const float4*>(psi);
    for (uint64_t i = first; i < n / 2; i += stride) {
      const float4 a = p4[i];
      qsdf::dot_add(acc, qsdf::df{a.x, 0.0f}, qsdf::df{a.x, 0.0f});
      qsdf::dot_add(acc, qsdf::df{a.y, 0.0f}, qsdf::df{a.y, 0.0f});
      qsdf::dot_add(acc, qsdf::df{a.z, 0.0f}, qsdf::df{a.z, 0.0f});
      qsdf::dot_add(acc, qsdf::df{a.w, 0.0f}, qsdf::df{a.w, 0.0f});
    }
    if ((n & 1) && first == 0) {
      const auto a = psi[n - 1];
      qsdf::dot_add(acc, qsdf::df{a.x, 0.0f}, qsdf::df{a.x, 0.0f});
      qsdf::dot_add(acc, qsdf::df{a.y, 0.0f}, qsdf::df{a.y, 0.0f});
    }
  } else {
    for (uint64_t i = first; i < n; i += stride) {
      const auto a = psi[i];
      const qsdf::df ar = to_df(a.x), ai = to_df(a.y);
      qsdf::dot_add(acc, ar, ar);
      qsdf::dot_add(acc, ai, ai);
    }
  }
  const double2 s = block_sum(make_double2(qsdf::finish(acc), 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The same sum in native FP64 (complex128 with FP64 or block fixed-point
// arithmetic): one FMA per square, a per-thread FP64 sum.
__global__ void __launch_bounds__(256) k_norm_f64(const double2* __restrict__ psi, uint64_t n,
                                                  double2* __restrict__ partials) {
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double2 a = psi[i];
    acc = fma(a.x, a.x, acc);
    acc = fma(a.y, a.y, acc);
  }
  const double2 s = block_sum(make_double2(acc, 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Tr rho = sum_j beta_{j (2^N + 1)} (Sec. "Pauli string expectation value").
template <typename R>
__global__ void __launch_bounds__(256) k_trace(const typename Cplx<R>::T* __restrict__ rho, int nq,
                                               double2* __restrict__ partials) {
  double sr = 0.0, si = 0.0;
  const uint64_t dim = 1ull << nq;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < dim; j += stride) {
    const auto a = rho[j * (dim + 1)];
    sr += (double)a.x;
    si += (double)a.y;
  }
  const double2 s = block_sum(make_double2(sr, si));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Tr(H rho) = sum_i H_i beta_i (Sec. "Pauli string expectation value",
// Eq. (density expectation sum)).  For the term h P, H_i is non-zero only
// where the row index l = i >> N equals the column index k = i mod 2^N with
// the X/Y bits flipped, and there pauliTensorElem = eta (-1)^{popc(k & yz)}:
// Y contributes i (-1)^{k_q}, Z contributes (-1)^{k_q}, X contributes 1.  The
// sum runs over those 2^N entries per term.
template <typename R>
__global__ void __launch_bounds__(256) k_expec_dm(const typename Cplx<R>::T* __restrict__ rho, int nq,
                                                  const PauliTerm* __restrict__ terms, int nterms,
                                                  double2* __restrict__ partials) {
  double sr = 0.0, si = 0.0;
  const uint64_t dim = 1ull << nq;
  const uint64_t total = dim * (uint64_t)nterms;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += stride) {
    const int n = (int)(w >> nq);
    const uint64_t k = w & (dim - 1);
    const PauliTerm t = terms[n];
    const auto b = rho[k | ((k ^ t.xy) << nq)];
    double2 v = make_double2((double)b.x, (double)b.y);
    v = rot_i(v, t.eta);
    const double h = parity64(k & t.yz) ? -t.h : t.h;
    sr += h * v.x;
    si += h * v.y;
  }
  const double2 s = block_sum(make_double2(sr, si));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// <psi|H|psi> = sum_n h_n sum_i conj(alpha_i) (P_n psi)_i with
// (P psi)_i = beta_{i'} alpha_{i'}, i' = i xor xy (Sec. "Pauli tensor",
// Eq. (Pauli tensor amplitude update)), in one pass over the amplitudes with
// every term evaluated at each amplitude read:
//  * terms with xy = 0 (I/Z strings) are diagonal: h_n (-1)^{popc(i & yz_n)}
//    |alpha_i|^2 from the amplitude alone;
//  * terms that share xy (consecutive after the host's sort) share the
//    partner load alpha_{i xor xy} and the product q = conj(alpha_i) alpha_{i'};
//  * each Pauli string is Hermitian and h is real, so the contributions of i
//    and i xor xy are complex conjugates: only indices with the highest bit
//    of xy clear are visited, each counting 2 Re(i^eta q) h (-1)^{popc(i' & yz)}.
// Arithmetic is double-float (qs_df.cuh): q and |alpha_i|^2 as error-free
// FP32 dot products, every contribution added to one per-thread accumulator
// with TwoSum, so the loop needs no FP64 instruction; each thread rounds its
// sum to double once.  The imaginary part of the result is exactly zero.
// A term as the kernel reads it from shared memory: h already split.
struct TermDf {
  uint64_t xy, yz;
  float hh, hl;
  int eta, pad;
};
// A run of terms sharing xy.
struct GroupDf {
  uint64_t xy, hb;       // flip mask, its highest bit (0 for the diagonal run)
  int first, count;
};

// Virtual tile positions handed out in increasing order: ctr[0] is the next
// position, ctr[1] counts finished blocks; the last block to finish resets
// both, so the slot reads as zero in the final reduction.  Thread 0 fetches
// one position ahead (s_v double-buffered), the block reads it after the
// barrier that ends a tile.
struct TileCounter {
  unsigned long long* ctr;
  __device__ void first(uint64_t* s_v) const {
    if (threadIdx.x == 0) s_v[0] = atomicAdd(ctr, 1ull);
    __syncthreads();
  }
  __device__ void prefetch(uint64_t* s_v, int it) const {
    if (threadIdx.x == 0) s_v[(it + 1) & 1] = atomicAdd(ctr, 1ull);
  }
  __device__ void finish() const {
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(ctr + 1, 1ull) == gridDim.x - 1) {
        atomicExch(ctr, 0ull);
        atomicExch(ctr + 1, 0ull);
      }
    }
  }
};

// Work mapping: a block takes tiles of 256 E consecutive amplitudes (thread t
// holds amplitudes t, t + 256, ... of the tile) and runs every group over the
// tile.  Tiles are handed out in increasing virtual order by a counter
// (TileCounter), so the blocks stay on neighbouring virtual tiles: a coset of
// the order is processed while it is in L2, however unevenly the blocks run.  A group whose highest flip bit lies above the tile either visits the
// whole tile or none of it, so the test is made once per tile and group; the
// E partner loads of a visited tile are in flight together.
template <typename R, int E>
__global__ void __launch_bounds__(256) k_expec_sv(const typename Cplx<R>::T* __restrict__ psi, int nq,
                                                  const PauliTerm* __restrict__ terms, int nterms,
                                                  double2* __restrict__ partials, const __grid_constant__ TileOrder ord,
                                                  TileCounter tc) {
  using qsdf::df;
  using T2 = typename Cplx<R>::T;
  extern __shared__ unsigned char sm_raw[];
  TermDf* ts = reinterpret_cast<TermDf*>(sm_raw);
  GroupDf* gs = reinterpret_cast<GroupDf*>(ts + nterms);
  __shared__ int ngroups;
  for (int n = threadIdx.x; n < nterms; n += blockDim.x) {
    const PauliTerm t = terms[n];
    const df h = qsdf::split(t.h);
    ts[n] = TermDf{t.xy, t.yz, h.h, h.l, t.eta, 0};
  }
  __syncthreads();
  if (threadIdx.x == 0) {                 // runs of equal xy, in order
    int ng = 0;
    for (int n = 0; n < nterms; ++n) {
      if (n == 0 || ts[n].xy != ts[n - 1].xy) {
        const uint64_t xy = ts[n].xy;
        gs[ng] = GroupDf{xy, xy ? 1ull << (63 - __clzll((long long)xy)) : 0ull, n, 0};
        ++ng;
      }
      ++gs[ng - 1].count;
    }
    ngroups = ng;
  }
  __syncthreads();
  const int ng = ngroups;
  qsdf::dot_acc acc{0.0f, 0.0f};
  constexpr uint64_t kTile = 256ull * E;
  const uint64_t dim = 1ull << nq;
  const uint64_t ntiles = dim > kTile ? dim / kTile : 1;
  __shared__ uint64_t s_v[2];
  tc.first(s_v);
  for (int it = 0;; ++it) {
    const uint64_t vt = s_v[it & 1];
    if (vt >= ntiles) break;
    tc.prefetch(s_v, it);
    const uint64_t base = ordered_tile(vt, ord) * kTile;
    uint64_t iu[E];
    bool ok[E];
    df ar[E], ai[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      iu[e] = base + (uint64_t)(e * 256 + threadIdx.x);
      ok[e] = iu[e] < dim;
      T2 a;
      a.x = 0;
      a.y = 0;
      if (ok[e]) a = psi[iu[e]];
      ar[e] = to_df(a.x);
      ai[e] = to_df(a.y);
    }
    for (int g = 0; g < ng; ++g) {
      const GroupDf G = gs[g];
      if (G.xy == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (!ok[e]) continue;
          qsdf::dot_acc pa = qsdf::dot_first(ar[e], ar[e]);    // |alpha_i|^2
          qsdf::dot_add(pa, ai[e], ai[e]);
          const df p2 = qsdf::dot_result(pa);
          for (int n = G.first; n < G.first + G.count; ++n) {
            const bool neg = parity64(iu[e] & ts[n].yz);
            qsdf::dot_add(acc, df{neg ? -ts[n].hh : ts[n].hh, neg ? -ts[n].hl : ts[n].hl}, p2);
          }
        }
        continue;
      }
      if (G.hb >= kTile && (base & G.hb)) continue;     // the whole tile is the upper half
      bool vis[E];
      T2 b[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        vis[e] = ok[e] && !(iu[e] & G.hb);
        b[e].x = 0;
        b[e].y = 0;
        if (vis[e]) b[e] = psi[iu[e] ^ G.xy];
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (!vis[e]) continue;
        const uint64_t ip = iu[e] ^ G.xy;
        const df br = to_df(b[e].x), bi = to_df(b[e].y);
        // q = conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
        qsdf::dot_acc qa = qsdf::dot_first(ar[e], br);
        qsdf::dot_add(qa, ai[e], bi);
        qsdf::dot_acc qb = qsdf::dot_first(ar[e], bi);
        qsdf::dot_add(qb, qsdf::neg(ai[e]), br);
        const df qr = qsdf::dot_result(qa), qi = qsdf::dot_result(qb);
        for (int n = G.first; n < G.first + G.count; ++n) {
          // 2 Re(i^eta q) (-1)^{popc(ip & yz)} h: eta 0 -> qr, 1 -> -qi, 2 -> -qr, 3 -> qi
          const int eta = ts[n].eta;
          const bool neg = parity64(ip & ts[n].yz) != (eta == 1 || eta == 2);
          const float s2 = neg ? -2.0f : 2.0f;                 // exact scaling
          qsdf::dot_add(acc, df{s2 * ts[n].hh, s2 * ts[n].hl}, (eta & 1) ? qi : qr);
        }
      }
    }
    __syncthreads();                        // the prefetched position is visible, the other slot free
  }
  tc.finish();
  const double2 s = block_sum(make_double2(qsdf::finish(acc), 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The same one-pass expectation in native FP64 (complex128 with FP64 or block
// fixed-point arithmetic): products and the per-thread sum in FP64.
template <int E>
__global__ void __launch_bounds__(256) k_expec_sv_f64(const double2* __restrict__ psi, int nq,
                                                      const PauliTerm* __restrict__ terms, int nterms,
                                                      double2* __restrict__ partials,
                                                      const __grid_constant__ TileOrder ord, TileCounter tc) {
  extern __shared__ unsigned char sm_raw[];
  PauliTerm* ts = reinterpret_cast<PauliTerm*>(sm_raw);
  GroupDf* gs = reinterpret_cast<GroupDf*>(ts + nterms);
  __shared__ int ngroups;
  for (int n = threadIdx.x; n < nterms; n += blockDim.x) ts[n] = terms[n];
  __syncthreads();
  if (threadIdx.x == 0) {                 // runs of equal xy, in order
    int ng = 0;
    for (int n = 0; n < nterms; ++n) {
      if (n == 0 || ts[n].xy != ts[n - 1].xy) {
        const uint64_t xy = ts[n].xy;
        gs[ng] = GroupDf{xy, xy ? 1ull << (63 - __clzll((long long)xy)) : 0ull, n, 0};
        ++ng;
      }
      ++gs[ng - 1].count;
    }
    ngroups = ng;
  }
  __syncthreads();
  const int ng = ngroups;
  double acc = 0.0;
  constexpr uint64_t kTile = 256ull * E;
  const uint64_t dim = 1ull << nq;
  const uint64_t ntiles = dim > kTile ? dim / kTile : 1;
  __shared__ uint64_t s_v[2];
  tc.first(s_v);
  for (int it = 0;; ++it) {
    const uint64_t vt = s_v[it & 1];
    if (vt >= ntiles) break;
    tc.prefetch(s_v, it);
    const uint64_t base = ordered_tile(vt, ord) * kTile;
    uint64_t iu[E];
    bool ok[E];
    double2 a[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      iu[e] = base + (uint64_t)(e * 256 + threadIdx.x);
      ok[e] = iu[e] < dim;
      a[e] = ok[e] ? psi[iu[e]] : make_double2(0.0, 0.0);
    }
    for (int g = 0; g < ng; ++g) {
      const GroupDf G = gs[g];
      if (G.xy == 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (!ok[e]) continue;
          const double p2 = fma(a[e].x, a[e].x, a[e].y * a[e].y);
          for (int n = G.first; n < G.first + G.count; ++n)
            acc = fma(parity64(iu[e] & ts[n].yz) ? -ts[n].h : ts[n].h, p2, acc);
        }
        continue;
      }
      if (G.hb >= kTile && (base & G.hb)) continue;     // the whole tile is the upper half
      bool vis[E];
      double2 b[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        vis[e] = ok[e] && !(iu[e] & G.hb);
        b[e] = vis[e] ? psi[iu[e] ^ G.xy] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (!vis[e]) continue;
        const uint64_t ip = iu[e] ^ G.xy;
        // q = conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
        const double qr = fma(a[e].x, b[e].x, a[e].y * b[e].y);
        const double qi = fma(a[e].x, b[e].y, -(a[e].y * b[e].x));
        for (int n = G.first; n < G.first + G.count; ++n) {
          const int eta = ts[n].eta;
          const bool neg = parity64(ip & ts[n].yz) != (eta == 1 || eta == 2);
          acc = fma(neg ? -2.0 * ts[n].h : 2.0 * ts[n].h, (eta & 1) ? qi : qr, acc);
        }
      }
    }
    __syncthreads();                        // the prefetched position is visible, the other slot free
  }
  tc.finish();
  const double2 s = block_sum(make_double2(acc, 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The diagonal (I/Z) terms of a statevector Pauli sum, many at a time:
// sum_n h_n sum_i |alpha_i|^2 (-1)^{popc(i & z_n)}.  A warp holds 32
// consecutive amplitudes i = base + m; a Walsh-Hadamard transform over its
// lanes gives W_j = sum_m |alpha_{base+m}|^2 (-1)^{popc(j & m)} in lane j, so
// the tile's share of term n is (-1)^{popc(base & z_n)} W_{z_n mod 32}: five
// butterfly steps per amplitude and one multiply-add per 32 terms replace one
// add per term.  All in double-float (no FP64 in the loop; each thread rounds
// its sum once).  Needs N >= 5 (whole warps of amplitudes).
__device__ __forceinline__ qsdf::df df_add(qsdf::df a, qsdf::df b) {
  const float s = a.h + b.h;                    // TwoSum of the high parts
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + (a.l + b.l);
  const float h = s + e;                        // renormalise
  return qsdf::df{h, e - (h - s)};
}

// A diagonal term in shared memory: its Z mask and the two halves of its
// coefficient (16 bytes: one load per lane).
struct ZTermDf {
  uint64_t z;
  float hh, hl;
};

// A warp takes tiles of 32 U consecutive amplitudes (U transforms whose loads
// are all in flight together), so each term is read from shared memory once
// per U transforms.
template <typename R, int U>
__global__ void __launch_bounds__(256) k_expec_sv_diag(const typename Cplx<R>::T* __restrict__ psi, int nq,
                                                       const PauliTerm* __restrict__ terms, int nterms,
                                                       double2* __restrict__ partials) {
  using qsdf::df;
  extern __shared__ ZTermDf tz[];
  for (int n = threadIdx.x; n < nterms; n += blockDim.x) {
    const PauliTerm t = terms[n];
    const df h = qsdf::split(t.h);
    tz[n] = ZTermDf{t.yz, h.h, h.l};
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  qsdf::dot_acc acc{0.0f, 0.0f};
  const uint64_t ntiles = (1ull << nq) / (32 * U);
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < ntiles;
       tile += nwarps) {
    const uint64_t base = tile * (32 * U);
    typename Cplx<R>::T a[U];
#pragma unroll
    for (int k = 0; k < U; ++k) a[k] = psi[base + 32 * k + lane];
    df w[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const df ar = to_df(a[k].x), ai = to_df(a[k].y);
      qsdf::dot_acc pa = qsdf::dot_first(ar, ar);
      qsdf::dot_add(pa, ai, ai);
      w[k] = qsdf::dot_result(pa);
#pragma unroll
      for (int b = 1; b < 32; b <<= 1) {
        // lanes with bit b set keep o - w, the others w + o (one TwoSum each)
        const df o{__shfl_xor_sync(0xFFFFFFFFu, w[k].h, b), __shfl_xor_sync(0xFFFFFFFFu, w[k].l, b)};
        const float sg = (lane & b) ? -1.0f : 1.0f;
        w[k] = df_add(df{sg * w[k].h, sg * w[k].l}, o);
      }
    }
    for (int n0 = 0; n0 < nterms; n0 += 32) {
      const int n = n0 + lane;
      ZTermDf t{0, 0.0f, 0.0f};
      if (n < nterms) t = tz[n];
      const int src = (int)(t.z & 31u);
      const bool odd = parity64(base & t.z);
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const df wz{__shfl_sync(0xFFFFFFFFu, w[k].h, src), __shfl_sync(0xFFFFFFFFu, w[k].l, src)};
        const bool neg = odd ^ (bool)(__popc((unsigned)(32 * k) & (unsigned)t.z) & 1);
        qsdf::dot_add(acc, neg ? qsdf::neg(df{t.hh, t.hl}) : df{t.hh, t.hl}, wz);
      }
    }
  }
  const double2 s = block_sum(make_double2(qsdf::finish(acc), 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// The diagonal-term kernel in native FP64 (butterflies and the sum in FP64).
struct ZTerm64 {
  uint64_t z;
  double h;
};
template <int U>
__global__ void __launch_bounds__(256) k_expec_sv_diag_f64(const double2* __restrict__ psi, int nq,
                                                           const PauliTerm* __restrict__ terms, int nterms,
                                                           double2* __restrict__ partials) {
  extern __shared__ ZTerm64 tz64[];
  for (int n = threadIdx.x; n < nterms; n += blockDim.x) tz64[n] = ZTerm64{terms[n].yz, terms[n].h};
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  const uint64_t ntiles = (1ull << nq) / (32 * U);
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < ntiles;
       tile += nwarps) {
    const uint64_t base = tile * (32 * U);
    double2 a[U];
#pragma unroll
    for (int k = 0; k < U; ++k) a[k] = psi[base + 32 * k + lane];
    double w[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      w[k] = fma(a[k].x, a[k].x, a[k].y * a[k].y);
#pragma unroll
      for (int b = 1; b < 32; b <<= 1) {
        const double o = __shfl_xor_sync(0xFFFFFFFFu, w[k], b);
        w[k] = (lane & b) ? o - w[k] : w[k] + o;
      }
    }
    for (int n0 = 0; n0 < nterms; n0 += 32) {
      const int n = n0 + lane;
      ZTerm64 t{0, 0.0};
      if (n < nterms) t = tz64[n];
      const int src = (int)(t.z & 31u);
      const bool odd = parity64(base & t.z);
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const double wz = __shfl_sync(0xFFFFFFFFu, w[k], src);
        const bool neg = odd ^ (bool)(__popc((unsigned)(32 * k) & (unsigned)t.z) & 1);
        acc = fma(neg ? -t.h : t.h, wz, acc);
      }
    }
  }
  const double2 s = block_sum(make_double2(acc, 0.0));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename R, int U>
static cudaError_t launch_diag(const void* amps, int nq, const PauliTerm* terms, int nterms, double2* partials,
                               cudaStream_t st) {
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(k_expec_sv_diag<R, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(ZTermDf) * kTermChunk));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  k_expec_sv_diag<R, U><<<kReduceBlocks, 256, sizeof(ZTermDf) * (size_t)nterms, st>>>(
      static_cast<const typename Cplx<R>::T*>(amps), nq, terms, nterms, partials);
  return cudaGetLastError();
}

cudaError_t launch_expec_sv_diag(qs_prec prec, const void* amps, int nq, const PauliTerm* terms, int nterms,
                                 double2* partials, cudaStream_t st, bool f64) {
  if (nq < 5 || nterms > kTermChunk) return cudaErrorInvalidValue;
  if (prec == QS_C128 && f64) {
    static bool attr_done = false;
    if (!attr_done) {
      cudaError_t e = cudaFuncSetAttribute(k_expec_sv_diag_f64<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(ZTerm64) * kTermChunk));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_expec_sv_diag_f64<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(ZTerm64) * kTermChunk));
      if (e != cudaSuccess) return e;
      attr_done = true;
    }
    const size_t sm = sizeof(ZTerm64) * (size_t)nterms;
    if (nq >= 7)
      k_expec_sv_diag_f64<4><<<kReduceBlocks, 256, sm, st>>>(static_cast<const double2*>(amps), nq, terms, nterms,
                                                              partials);
    else
      k_expec_sv_diag_f64<1><<<kReduceBlocks, 256, sm, st>>>(static_cast<const double2*>(amps), nq, terms, nterms,
                                                              partials);
    return cudaGetLastError();
  }
  if (prec == QS_C128)
    return nq >= 7 ? launch_diag<double, 4>(amps, nq, terms, nterms, partials, st)
                   : launch_diag<double, 1>(amps, nq, terms, nterms, partials, st);
  return nq >= 7 ? launch_diag<float, 4>(amps, nq, terms, nterms, partials, st)
                 : launch_diag<float, 1>(amps, nq, terms, nterms, partials, st);
}

// Stage two: one block of 1024 threads; thread j adds partials j, j + 1024, ...
__global__ void __launch_bounds__(1024) k_reduce_final(const double2* __restrict__ partials, int n,
                                                       double2* __restrict__ result, int accumulate) {
  double sr = 0.0, si = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    sr += partials[j].x;
    si += partials[j].y;
  }
  const double2 s = block_sum(make_double2(sr, si));
  if (threadIdx.x == 0) {
    if (accumulate) {
      result[0].x += s.x;
      result[0].y += s.y;
    } else {
      result[0] = s;
    }
  }
}

// Stage-one kernels always run exactly kReduceBlocks blocks; blocks with no
// work write a zero partial.
cudaError_t launch_norm(qs_prec prec, const void* amps, int ns, double2* partials, cudaStream_t st, bool f64) {
  const uint64_t n = 1ull << ns;
  if (prec == QS_C128 && f64)
    k_norm_f64<<<kNormBlocks, 256, 0, st>>>(static_cast<const double2*>(amps), n, partials);
  else if (prec == QS_C128)
    k_norm<double><<<kNormBlocks, 256, 0, st>>>(static_cast<const double2*>(amps), n, partials);
  else
    k_norm<float><<<kNormBlocks, 256, 0, st>>>(static_cast<const float2*>(amps), n, partials);
  return cudaGetLastError();
}

cudaError_t launch_trace(qs_prec prec, const void* amps, int nq, double2* partials, cudaStream_t st) {
  if (prec == QS_C128)
    k_trace<double><<<kReduceBlocks, 256, 0, st>>>(static_cast<const double2*>(amps), nq, partials);
  else
    k_trace<float><<<kReduceBlocks, 256, 0, st>>>(static_cast<const float2*>(amps), nq, partials);
  return cudaGetLastError();
}

cudaError_t launch_expec_dm(qs_prec prec, const void* amps, int nq, const PauliTerm* terms, int nterms,
                            double2* partials, cudaStream_t st) {
  if (prec == QS_C128)
    k_expec_dm<double><<<kReduceBlocks, 256, 0, st>>>(static_cast<const double2*>(amps), nq, terms, nterms,
                                                      partials);
  else
    k_expec_dm<float><<<kReduceBlocks, 256, 0, st>>>(static_cast<const float2*>(amps), nq, terms, nterms,
                                                     partials);
  return cudaGetLastError();
}

// Blocks of the statevector expectation kernels: as many as are resident at
// once (at most kReduceBlocks), so that the blocks walk consecutive virtual
// tiles together and a coset of the tile order is processed while it is in
// L2.  The other partial slots are zeroed (the final sum stays in a fixed
// order for a given kernel and GPU).
// The last partial slot holds the kernels' TileCounter (zeroed here with the
// unused slots, and zero again when the kernel ends), so the grid is at most
// kReduceBlocks - 1.
template <typename K>
static cudaError_t resident_grid(K kernel, size_t smem, double2* partials, cudaStream_t st, unsigned* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
  if (e != cudaSuccess) return e;
  const int g = per_sm > 0 ? per_sm * num_sms() : 1;
  *grid = (unsigned)(g < kReduceBlocks - 1 ? g : kReduceBlocks - 1);
  return cudaMemsetAsync(partials + *grid, 0, sizeof(double2) * (kReduceBlocks - *grid), st);
}

static TileCounter tile_counter(double2* partials) {
  return TileCounter{reinterpret_cast<unsigned long long*>(partials + kReduceBlocks - 1)};
}

template <typename R, int E>
static cudaError_t expec_sv_u(const void* amps, int nq, const PauliTerm* terms, int nterms, double2* partials,
                              cudaStream_t st, const TileOrder& ord) {
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(k_expec_sv<R, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)((sizeof(TermDf) + sizeof(GroupDf)) * kTermChunk));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const size_t smem = (sizeof(TermDf) + sizeof(GroupDf)) * (size_t)nterms;
  unsigned grid = kReduceBlocks;
  const cudaError_t e = resident_grid(k_expec_sv<R, E>, smem, partials, st, &grid);
  if (e != cudaSuccess) return e;
  k_expec_sv<R, E><<<grid, 256, smem, st>>>(static_cast<const typename Cplx<R>::T*>(amps), nq, terms, nterms,
                                            partials, ord, tile_counter(partials));
  return cudaGetLastError();
}

cudaError_t launch_expec_sv(qs_prec prec, const void* amps, int nq, const PauliTerm* terms, int nterms,
                            double2* partials, cudaStream_t st, bool f64, const TileOrder& ord) {
  static_assert(256 * 4 == (1 << kExpecTileBits), "tiles of the expectation kernels");
  if (nterms > kTermChunk) return cudaErrorInvalidValue;
  if (prec == QS_C128 && f64) {
    static bool attr_done = false;
    const size_t per = sizeof(PauliTerm) + sizeof(GroupDf);
    if (!attr_done) {
      const cudaError_t e = cudaFuncSetAttribute(k_expec_sv_f64<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(per * kTermChunk));
      if (e != cudaSuccess) return e;
      attr_done = true;
    }
    unsigned grid = kReduceBlocks;
    const cudaError_t e = resident_grid(k_expec_sv_f64<4>, per * (size_t)nterms, partials, st, &grid);
    if (e != cudaSuccess) return e;
    k_expec_sv_f64<4><<<grid, 256, per * (size_t)nterms, st>>>(static_cast<const double2*>(amps), nq, terms, nterms,
                                                                partials, ord, tile_counter(partials));
    return cudaGetLastError();
  }
  // tiles of 1024 amplitudes (28 qubits, 8 random terms: 6.9 ms against 7.5
  // and 8.0 ms for tiles of 512 and 2048)
  return prec == QS_C128 ? expec_sv_u<double, 4>(amps, nq, terms, nterms, partials, st, ord)
                         : expec_sv_u<float, 4>(amps, nq, terms, nterms, partials, st, ord);
}

cudaError_t launch_reduce_final(const double2* partials, double2* result, int accumulate, cudaStream_t st,
                                int nblocks) {
  k_reduce_final<<<1, 1024, 0, st>>>(partials, nblocks, result, accumulate);
  return cudaGetLastError();
}

}  // namespace qsk
