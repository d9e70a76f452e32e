// Dense n-target gates (2 <= n <= 5) for complex128 states on the bf16 tensor
// cores, with error-free integer slicing (the Ozaki scheme; the slicing and
// its bounds are in qs_slices.cuh).
//
// The group update alpha_kj -> sum_l m_jl alpha_kl (Sec. "Many-target gate",
// Eq. (local many-target amplitude update)) over a tile of 128 groups is the
// real GEMM C = A B, A[g, 2l + c'] the interleaved (re, im) amplitudes of group
// g, B the realified matrix (B[2l, 2j] = Re m_jl, B[2l+1, 2j] = -Im m_jl,
// B[2l, 2j+1] = Im m_jl, B[2l+1, 2j+1] = Re m_jl).  Each row of A (scaled by
// its largest exponent) and each column of B is cut into seven balanced bf16
// digit slices; the 28 slice products with s + t <= 6 run as tcgen05
// kind::f16 MMAs whose FP32 accumulation in tensor memory is exact, one
// accumulator per level L = s + t; the epilogue recombines the levels in
// 64-bit integers, converts once to double and applies the two scales.  Two
// targets run as three: the matrix is extended by an identity on one more
// (free) qubit, which changes nothing in the result and fills the MMA's K = 16.
//
// Work mapping: thread (warp w, lane) owns row g = 32 (w mod 4) + lane (the
// tensor-memory lane that warp may read) and the amplitudes l in
// [c EPT, (c+1) EPT), c = w / 4, of that row, for the gather, the slicing and
// the epilogue alike, so the row's exponent and base index stay in registers.
// Pipeline per CTA (persistent, tiles c, c + grid, ...): the loads of the
// next tile are issued right after the current tile's slices are written, so
// they are in flight during the MMAs and the epilogue; with two buffers of
// slices and accumulators (NBUF = 2) the epilogue of tile i - 1 would run
// while the tensor cores work on tile i.  The row maxima of tile i + 1 are
// taken after the epilogue, so a tile costs two CTA barriers.  Thread 0
// issues the MMAs: one per A slice and K chunk, against all the B slices it
// pairs with (see mma_tile).  Every wait is bounded:
// on timeout the kernel records an error code, frees its tensor memory and
// returns.
#include "qs_device.cuh"
#include "qs_slices.cuh"
#include "qs_tc_ptx.cuh"

namespace qsk {
namespace {

using namespace tcptx;

constexpr int kRows = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

__host__ __device__ constexpr uint32_t tmem_cols(uint32_t n) {
  return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}

// two floats holding small integers -> packed bf16 pair (lo in bits 0..15); exact
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// KS (7 or 8) digits of a double as floats
template <int KS>
__device__ __forceinline__ void digits(uint32_t hw, uint32_t lw, int emax, float* f) {
  if constexpr (KS == 8)
    qsoz::digit_floats_t8(qsoz::fixed_t8(hw, lw, emax), f);
  else
    qsoz::digit_floats_t(qsoz::fixed_t(hw, lw, emax), f);
}

// lower bound of a row or column exponent maximum: zeros and subnormals
// (their implicit bit wrongly set) then shift out entirely
template <int KS>
__host__ __device__ constexpr int emax_floor() { return KS == 8 ? 58 : qsoz::kEmaxFloor; }

// KS packed (re, im) digit pairs of one amplitude (words of re and im)
template <int KS>
__device__ __forceinline__ void slice_amp(const uint32_t* w, int emax, uint32_t* out) {
  float fr[KS], fi[KS];
  digits<KS>(w[0], w[1], emax, fr);
  digits<KS>(w[2], w[3], emax, fi);
#pragma unroll
  for (int s = 0; s < KS; ++s) out[s] = pack_bf16(fr[s], fi[s]);
}

// bounded wait on an mbarrier phase; true when it ran out
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity))
    if (++spins > kWaitLimit) return true;
  return false;
}

// entry (k, n) of the realified (and possibly identity-extended) matrix
__device__ __forceinline__ double realified(const TcParams& p, int D, int k, int n) {
  int j = n >> 1, l = k >> 1;
  const int c = n & 1, cp = k & 1;
  if (p.nmat < p.n) {
    if ((j >> p.nmat) != (l >> p.nmat)) return 0.0;
    const int mm = (1 << p.nmat) - 1;
    j &= mm;
    l &= mm;
    D = 1 << p.nmat;
  }
  const double mr = p.mat[2 * (j * D + l)];
  const double mi = p.conj ? -p.mat[2 * (j * D + l) + 1] : p.mat[2 * (j * D + l) + 1];
  return c == 0 ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr);
}

// All slice products of one tile.  B's slices lie back to back in shared
// memory (slice t at t * bbytes), so for A slice s one MMA against the first
// 7 - s slices of B, with its accumulator starting at level s, adds A_s B_t
// into level s + t for every t <= 6 - s at once: each A slice is read once
// per 16-column K chunk.  Products wider than 256 columns are cut into
// 256-column MMAs.  The first MMA (s = 0, first K chunk) initialises all
// levels.  adesc / bdesc: descriptors of slice 0 of A and B; K chunks are
// 256 bytes apart, 8-row groups of B kdim * 16 bytes (encoded address >> 4).
template <int N, int KCH, int KS>
__device__ __forceinline__ void mma_tile(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t abytes) {
  constexpr int K = 16 * KCH;
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    constexpr int kMax = 256;
#pragma unroll
    for (int c0 = 0; c0 < (KS - s) * N; c0 += kMax) {
      const int w = (KS - s) * N - c0 < kMax ? (KS - s) * N - c0 : kMax;
      const uint32_t idesc = idesc_bf16(kRows, w);
#pragma unroll
      for (int kk = 0; kk < KCH; ++kk)
        mma_bf16(d_tmem + (uint32_t)(s * N + c0), adesc + ((s * abytes + kk * 256) >> 4),
                 bdesc + (((uint32_t)c0 * K * 2 + kk * 256) >> 4), idesc, (s | kk) != 0);
    }
  }
}

}  // namespace

template <int NT, int THREADS, int NBUF, int CTAS, int KS>
__global__ void __launch_bounds__(THREADS, CTAS) k_dense_ozaki(double2* __restrict__ psi, const __grid_constant__ TcParams p) {
  constexpr int kS = KS;
  constexpr int D = 1 << NT;
  constexpr int K = 2 * D, N = 2 * D;
  constexpr int CG = THREADS / kRows;         // threads per row
  constexpr int EPT = D / CG;                 // amplitudes per thread
  constexpr int CPW = 2 * EPT;                // accumulator columns per thread
  static_assert(EPT % 4 == 0, "four amplitudes per 16-byte slice store");
  constexpr int ABYTES = kRows * K * 2;       // one bf16 digit slice of A
  constexpr int BBYTES = N * K * 2;
  constexpr uint32_t LCOLS = kS * N;          // accumulator columns of one buffer
  constexpr uint32_t TCOLS = tmem_cols(NBUF * LCOLS);
  static_assert(NBUF * LCOLS <= 512, "tensor memory");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_dig = smem;                                        // NBUF x kS x ABYTES
  unsigned char* b_dig = a_dig + NBUF * kS * ABYTES;                  // kS x BBYTES
  uint64_t* toff = reinterpret_cast<uint64_t*>(b_dig + kS * BBYTES);  // D
  uint64_t* rowoff = toff + D;                                        // kRows
  uint64_t* tile_base = rowoff + kRows;                               // 2
  uint64_t* mbar = tile_base + 2;                                     // 2
  int* csc = reinterpret_cast<int*>(mbar + 2);                        // N: (column exponent - 2100) << 20
  int* rowexp = csc + N;                                              // 2 x kRows: exponent field of the row maximum
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rowexp + 2 * kRows);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B: column maxima of the exponents, then the digit slices (once per CTA)
  for (int n = tid; n < N; n += THREADS) {
    int e = emax_floor<KS>();
    for (int k = 0; k < K; ++k) e = max(e, qsoz::biased_exp((uint32_t)__double2hiint(realified(p, D, k, n))));
    csc[n] = e;
  }
  __syncthreads();
  for (int idx = tid; idx < N * K; idx += THREADS) {
    const int n = idx / K, k = idx % K;
    const double v = realified(p, D, k, n);
    float f[kS];
    digits<KS>((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), csc[n], f);
    const uint32_t off = canon_off16(n, k, K);
#pragma unroll
    for (int s = 0; s < kS; ++s)
      *reinterpret_cast<uint16_t*>(b_dig + s * BBYTES + off) = (uint16_t)(pack_bf16(f[s], 0.0f) & 0xFFFFu);
  }
  for (int j = tid; j < D; j += THREADS) {
    uint64_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q)
      if ((j >> q) & 1) off |= 1ull << p.tpos[q];
    toff[j] = off;
  }
  const int row_bits = p.tile_bits - NT;
  for (int g = tid; g < kRows; g += THREADS) {
    uint64_t off = 0;
    for (int b = 0, r = 0; b < p.tile_bits; ++b)
      if (!((p.tslot_mask >> b) & 1)) {
        if ((g >> r) & 1) off |= 1ull << p.P[b];
        ++r;
      }
    rowoff[g] = off;
    rowexp[g] = 0;
    rowexp[kRows + g] = 0;
  }
  __syncthreads();
  // scale 2^(Ea + Eb - 2046 - 54) (seven slices) or 2^(Ea + Eb - 2046 - 53)
  // (eight: the recombined sum is kept divided by 2^8) with biased Ea, Eb,
  // as an exponent-field increment
  constexpr int kScaleOff = KS == 8 ? 53 : 54;
  for (int n = tid; n < N; n += THREADS) csc[n] = (int)((unsigned)(csc[n] - 2046 - kScaleOff) << 20);
  if (tid == 0) {
    tile_base[0] = insert_zeros(blockIdx.x, p.hi_ins, p.nhi) | p.ctrl_mask;
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(mbar + b, 1);      // one commit per tile
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, TCOLS);
    tmem_relinquish();
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t sbo = K * 16;

  const int g = 32 * (warp & 3) + lane;       // row (tensor-memory lane)
  const int cg = warp >> 2;                   // amplitude / column group of the row
  const int l0 = cg * EPT;
  const bool row_ok = g < (1 << row_bits);
  const uint64_t roff = rowoff[g];
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const int helper = THREADS > kRows ? kRows : 0;   // computes tile bases
  // target offsets of this thread's amplitudes: registers when few
  constexpr bool kRegOff = EPT <= 4;
  uint64_t toffr[kRegOff ? EPT : 1];
  if (kRegOff) {
#pragma unroll
    for (int i = 0; i < (kRegOff ? EPT : 1); ++i) toffr[i] = toff[l0 + i];
  }
  auto tofs = [&](int i) -> uint64_t { return kRegOff ? toffr[kRegOff ? i : 0] : toff[l0 + i]; };

  uint32_t R[EPT][4];
  auto load_tile = [&](uint64_t base) {
    const uint64_t rb = base | roff;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      double2 v = make_double2(0.0, 0.0);
      if (row_ok) v = psi[rb | tofs(i)];
      R[i][0] = (uint32_t)__double2hiint(v.x);
      R[i][1] = (uint32_t)__double2loint(v.x);
      R[i][2] = (uint32_t)__double2hiint(v.y);
      R[i][3] = (uint32_t)__double2loint(v.y);
    }
  };
  // row maximum of the exponents (the CG threads of a row are in different warps)
  // (exponent fields compared in place: 0x7FF00000 of the high words)
  auto row_max = [&](int slot) {
    uint32_t em = (uint32_t)emax_floor<KS>() << 20;
#pragma unroll
    for (int i = 0; i < EPT; ++i) em = max(em, max(R[i][0] & 0x7FF00000u, R[i][2] & 0x7FF00000u));
    atomicMax(rowexp + slot * kRows + g, (int)em);
  };

  // epilogue of one tile: levels -> exact integers -> doubles -> scatter
  auto epilogue = [&](uint32_t tbuf, int egs, uint64_t rb) {
#pragma unroll
    for (int cc = 0; cc < CPW; cc += 8) {
      float v[kS][8];
#pragma unroll
      for (int L = 0; L < kS; ++L) tmem_ld8(tmem + tbuf + lane_addr + (uint32_t)(L * N + cg * CPW + cc), v[L]);
      tmem_wait_ld();
      if (row_ok) {
        const int4 s0 = *reinterpret_cast<const int4*>(csc + cg * CPW + cc);
        const int4 s1 = *reinterpret_cast<const int4*>(csc + cg * CPW + cc + 4);
        const int scl[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        double o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t bits[kS];
#pragma unroll
          for (int L = 0; L < kS; ++L) bits[L] = __float_as_uint(v[L][q] + 12582912.0f);
          const double r = __ll2double_rn(KS == 8 ? qsoz::combine_levels8(bits) : qsoz::combine_levels(bits));
          const int hi = __double2hiint(r);                // 0 only for r = 0, which stays 0
          o[q] = __hiloint2double(hi + (hi != 0 ? egs + scl[q] : 0), __double2loint(r));
        }
#pragma unroll
        for (int q = 0; q < 8; q += 2) psi[rb | tofs((cc + q) >> 1)] = make_double2(o[q], o[q + 1]);
      }
    }
  };

  // prologue: the first tile's amplitudes and row maxima, the second tile's base
  load_tile(tile_base[0]);
  row_max(0);
  if (tid == helper && blockIdx.x + gridDim.x < p.ntiles)
    tile_base[1] = insert_zeros(blockIdx.x + gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
  __syncthreads();

  uint32_t phases = 0;
  bool failed = false;
  int it = 0;
  int eg_prev = 0;
  uint64_t rb_prev = 0;
  for (uint64_t c = blockIdx.x; c < p.ntiles; c += gridDim.x, ++it) {
    const int b = NBUF == 2 ? (it & 1) : 0;
    const int par = it & 1;                   // tile parity: row-maximum and base slots
    const uint64_t rb = tile_base[par] | roff;
    const bool has_next = c + gridDim.x < p.ntiles;
    const int egs = rowexp[par * kRows + g];   // exponent field of the row maximum
    const int eg = egs >> 20;
    // digit slices of this thread's amplitudes, 16 bytes per slice and 4 amplitudes
    unsigned char* A = a_dig + b * (kS * ABYTES);
#pragma unroll
    for (int i = 0; i < EPT; i += 4) {
      uint32_t pk[4][kS];
#pragma unroll
      for (int e = 0; e < 4; ++e) slice_amp<KS>(R[i + e], eg, pk[e]);
      const uint32_t off = canon_off16(g, 2 * (l0 + i), K);
#pragma unroll
      for (int s = 0; s < kS; ++s)
        *reinterpret_cast<uint4*>(A + s * ABYTES + off) = make_uint4(pk[0][s], pk[1][s], pk[2][s], pk[3][s]);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint64_t ad = smem_desc(smem_u32(A), 128, sbo), bd = smem_desc(smem_u32(b_dig), 128, sbo);
      mma_tile<N, K / 16, KS>(tmem + (uint32_t)(b * LCOLS), ad, bd, ABYTES);
      mma_commit(mbar + b);
    }
    if (cg == 0) rowexp[par * kRows + g] = 0;   // read by every thread of the row before the barrier
    // loads of the next tile, in flight during the MMAs and the epilogue
    if (has_next) load_tile(tile_base[par ^ 1]);
    bool timed_out = false;
    if (NBUF == 2) {
      if (it > 0) {
        const int pb = b ^ 1;
        timed_out = wait_phase(mbar + pb, (phases >> pb) & 1u);
        phases ^= 1u << pb;
        fence_after_sync();
        epilogue((uint32_t)(pb * LCOLS), eg_prev, rb_prev);
      }
    } else {
      timed_out = wait_phase(mbar, phases & 1u);
      phases ^= 1u;
      fence_after_sync();
      epilogue(0u, egs, rb);
    }
    eg_prev = egs;
    rb_prev = rb;
    if (has_next) row_max(par ^ 1);
    if (tid == helper && c + 2 * (uint64_t)gridDim.x < p.ntiles)
      tile_base[par] = insert_zeros(c + 2 * (uint64_t)gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    fence_before_sync();
    failed = __syncthreads_or(timed_out) != 0;
    fence_after_sync();
    if (failed) break;
  }
  if (NBUF == 2 && !failed && it > 0) {
    const int pb = (it - 1) & 1;
    const bool timed_out = wait_phase(mbar + pb, (phases >> pb) & 1u);
    fence_after_sync();
    epilogue((uint32_t)(pb * LCOLS), eg_prev, rb_prev);
    fence_before_sync();
    failed = __syncthreads_or(timed_out) != 0;
  }
  if (failed && tid == 0) atomicExch(p.err, 1);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

template <int NT, int THREADS, int NBUF, int CTAS, int kS>
static cudaError_t dense_ozaki_nt(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr int D = 1 << NT, K = 2 * D, N = 2 * D;
  constexpr size_t smem = (size_t)NBUF * kS * (kRows * K * 2) + (size_t)kS * (N * K * 2) + 8 * (D + kRows + 4) +
                          4 * (N + 2 * kRows) + 16;
  static_assert(smem * CTAS <= 227 * 1024, "shared memory");
  static_assert(CTAS * tmem_cols(NBUF * kS * N) <= 512, "tensor memory");
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_ozaki<NT, THREADS, NBUF, CTAS, kS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  // for 3 and 4 targets, eight times the resident CTAs: the late ones even out
  // the SMs' tile counts at the end of the pass (7% and 2% faster measured)
  const uint64_t maxb = (uint64_t)num_sms() * CTAS * (NT <= 4 ? 8 : 1);
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_ozaki<NT, THREADS, NBUF, CTAS, kS><<<g, THREADS, smem, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

// Several independent single-buffered CTAs per SM, whose phases drift apart,
// keep the SM busier than double buffering inside one CTA (measured at 30
// qubits: 3 targets 10.3 ms as four 128-thread CTAs against 12.2 ms as two
// double-buffered 256-thread CTAs; 4 targets 11.2 ms as two 256-thread CTAs
// against 13.9 ms as one double-buffered 512-thread CTA).  Tensor memory
// (seven levels of N columns per buffer) bounds the CTAs per SM.
cudaError_t launch_dense_ozaki(void* amps, const TcParams& p, int slices, cudaStream_t st) {
  if (slices == 8) {
    switch (p.n) {
      case 3: return dense_ozaki_nt<3, 128, 1, 4, 8>(amps, p, st);
      case 4: return dense_ozaki_nt<4, 256, 1, 2, 8>(amps, p, st);
      case 5: return dense_ozaki_nt<5, 512, 1, 1, 8>(amps, p, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.n) {
    case 3: return dense_ozaki_nt<3, 128, 1, 4, 7>(amps, p, st);
    case 4: return dense_ozaki_nt<4, 256, 1, 2, 7>(amps, p, st);
    case 5: return dense_ozaki_nt<5, 512, 1, 1, 7>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qsk
