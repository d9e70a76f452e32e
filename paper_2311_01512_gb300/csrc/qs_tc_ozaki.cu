// Dense n-target gates (2 <= n <= 5) for complex128 states on the bf16 tensor
// cores, with error-free integer slicing (the Ozaki scheme; the slicing and
// its bounds are in qs_slices.cuh).
//
// The group update alpha_kj -> sum_l m_jl alpha_kl (Sec. "Many-target gate",
// Eq. (local many-target amplitude update)) over a tile of 128 groups is the
// real GEMM C = A B, A[g, 2l + c'] the interleaved (re, im) amplitudes of group
// g, B the realified matrix (B[2l, 2j] = Re m_jl, B[2l+1, 2j] = -Im m_jl,
// B[2l, 2j+1] = Im m_jl, B[2l+1, 2j+1] = Re m_jl).  Each row of A (scaled by
// its largest exponent) and each column of B is cut into KS = 7 or 8 balanced
// digit slices; the slice products with s + t < KS run as tcgen05 kind::f16
// MMAs whose FP32 accumulation in tensor memory is exact, one accumulator per
// level L = s + t; the epilogue recombines the levels in integers, converts
// once to double and applies the two scales.  Two targets run as three: the
// matrix is extended by an identity on one more (free) qubit, which changes
// nothing in the result and fills the MMA's K = 16.
//
// The amplitude digits below the top one are stored offset by 192 (their
// bf16 bit patterns are then two shifted fields and a constant); each tile's
// accumulators start at P_L(n), minus the offset's contribution (192 times
// the B column sums of the slices involved) plus, for K <= 32, the magic
// 1.25 2^23 that leaves each level's integer in the low bits of its FP32
// pattern.  One initialising MMA writes them: a constant A whose rows are
// (1, 256, 65536, 0, ...) against a B whose column holds P = p0 + 256 p1 +
// 65536 p2 in three bf16-exact parts.
//
// Two kernels share these pieces.  k_dense_ozaki (below; five targets, and any
// pass of fewer tiles than SMs) runs every phase in every thread;
// k_dense_ozaki_ws (two to four targets) gives gathering and slicing, MMA
// issue and the epilogue to separate warps (its own comment further down).
//
// k_dense_ozaki's work mapping: thread (warp w, lane) owns row g = 32 (w mod 4) + lane (the
// tensor-memory lane that warp may read) and the amplitudes l in
// [c EPT, (c+1) EPT), c = w / 4, of that row, for the gather, the slicing and
// the epilogue alike, so the row's exponent and base index stay in registers.
// Pipeline per CTA (persistent, tiles c, c + grid, ...): the loads of the
// next tile are issued right after the current tile's slices are written, so
// they are in flight during the MMAs and the epilogue; with two buffers of
// slices and accumulators (NBUF = 2) the epilogue of tile i - 1 would run
// while the tensor cores work on tile i.  The row maxima of tile i + 1 are
// taken after the epilogue, so a tile costs two CTA barriers.  Thread 0
// issues the initialising MMA and then one MMA per A slice and K chunk,
// against all the B slices it pairs with (see mma_tile).  Every wait is
// bounded: on timeout the kernel records an error code, frees its tensor
// memory and returns.
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
// KS - s slices of B, with its accumulator starting at level s, adds A_s B_t
// into level s + t for every t <= KS - 1 - s at once: each A slice is read once
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
                 bdesc + (((uint32_t)c0 * K * 2 + kk * 256) >> 4), idesc, 1u);
    }
  }
}


// scale 2^(Ea + Eb - 2046 - 54) (seven slices) or 2^(Ea + Eb - 2046 - 53)
// (eight: the recombined sum is kept divided by 2^8) with biased Ea, Eb
template <int KS>
__host__ __device__ constexpr int scale_off() { return KS == 8 ? 53 : 54; }

// Per-CTA constants of a dense gate: the column exponent maxima of B (in
// csc), B's digit slices, the initialising MMA's operands (A rows
// (1, 256, 65536, 0, ...), B columns holding P_L(n) in three parts), the
// target offsets of the group members and the row offsets of the tile.  Every
// step runs over all (column, row) pairs of B at once, the maxima and the
// digit column sums (colsum: KS x N ints) through shared-memory atomics, so
// the setup is short next to one tile even for small states.
template <int NT, int KS, bool kMagicPre>
__device__ void tile_constants(const TcParams& p, unsigned char* b_dig, unsigned char* a_pre, unsigned char* b_pre,
                               int* csc, int* colsum, uint64_t* toff, uint64_t* rowoff, int tid, int nthr) {
  constexpr int D = 1 << NT, K = 2 * D, N = 2 * D, BBYTES = N * K * 2;
  for (int n = tid; n < N; n += nthr) csc[n] = emax_floor<KS>();
  for (int i = tid; i < KS * N; i += nthr) colsum[i] = 0;
  __syncthreads();
  // column fastest across threads: the lanes of a warp update different
  // columns' maxima and sums (no same-address atomics)
  for (int idx = tid; idx < N * K; idx += nthr) {
    const int n = idx % N, k = idx / N;
    atomicMax(csc + n, qsoz::biased_exp((uint32_t)__double2hiint(realified(p, D, k, n))));
  }
  __syncthreads();
  for (int idx = tid; idx < N * K; idx += nthr) {
    const int n = idx % N, k = idx / N;
    const double v = realified(p, D, k, n);
    float f[KS];
    digits<KS>((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), csc[n], f);
    const uint32_t off = canon_off16(n, k, K);
#pragma unroll
    for (int t = 0; t < KS; ++t) {
      *reinterpret_cast<uint16_t*>(b_dig + t * BBYTES + off) = (uint16_t)(pack_bf16(f[t], 0.0f) & 0xFFFFu);
      if (f[t] != 0.0f) atomicAdd(colsum + t * N + n, (int)f[t]);
    }
  }
  __syncthreads();
  // the start values P_L(n) = M - 192 sum_{t < L} colsum_t(n), one (L, n) per thread
  for (int idx = tid; idx < KS * N; idx += nthr) {
    const int L = idx / N, n = idx % N;
    int corr = 0;
    for (int t = 0; t < L; ++t) corr += colsum[t * N + n];
    int pp[3];
    qsoz::split_start((kMagicPre ? (int)qsoz::kPreMagic : 0) - qsoz::kDigitOffset * corr, pp);
    const int col = L * N + n;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      *reinterpret_cast<uint16_t*>(b_pre + canon_off16(col, k, 16)) =
          (uint16_t)(pack_bf16(k < 3 ? (float)pp[k] : 0.0f, 0.0f) & 0xFFFFu);
  }
  for (int idx = tid; idx < kRows * 16; idx += nthr) {
    const int g = idx >> 4, k = idx & 15;
    *reinterpret_cast<uint16_t*>(a_pre + canon_off16(g, k, 16)) =
        (uint16_t)(pack_bf16(k == 0 ? 1.0f : (k == 1 ? 256.0f : (k == 2 ? 65536.0f : 0.0f)), 0.0f) & 0xFFFFu);
  }
  for (int j = tid; j < D; j += nthr) {
    uint64_t off = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q)
      if ((j >> q) & 1) off |= 1ull << p.tpos[q];
    toff[j] = off;
  }
  for (int g = tid; g < kRows; g += nthr) {
    uint64_t off = 0;
    for (int b = 0, r = 0; b < p.tile_bits; ++b)
      if (!((p.tslot_mask >> b) & 1)) {
        if ((g >> r) & 1) off |= 1ull << p.P[b];
        ++r;
      }
    rowoff[g] = off;
  }
}

// The initialising MMA (every level column of the buffer at dcol starts at its
// P_L(n)) and the slice products of one tile; issued by one thread.
template <int N, int KCH, int KS>
__device__ __forceinline__ void mma_full_tile(uint32_t dcol, const unsigned char* a_pre, const unsigned char* b_pre,
                                              const unsigned char* A, const unsigned char* b_dig) {
  constexpr uint32_t LCOLS = KS * N;
  constexpr uint32_t sbo = KCH * 16 * 16;
  const uint64_t pad = smem_desc(smem_u32(a_pre), 128, 256), pbd = smem_desc(smem_u32(b_pre), 128, 256);
#pragma unroll
  for (uint32_t c0 = 0; c0 < LCOLS; c0 += 256) {
    const uint32_t w = LCOLS - c0 < 256 ? LCOLS - c0 : 256;
    mma_bf16(dcol + c0, pad, pbd + ((c0 * 32) >> 4), idesc_bf16(kRows, (int)w), 0u);
  }
  const uint64_t ad = smem_desc(smem_u32(A), 128, sbo), bd = smem_desc(smem_u32(b_dig), 128, sbo);
  mma_tile<N, KCH, KS>(dcol, ad, bd, kRows * KCH * 16 * 2);
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
  constexpr bool kMagicPre = K <= 32;         // accumulators start at the magic (no add in the epilogue)
  constexpr uint32_t kMB = kMagicPre ? qsoz::kPreMagicBits : qsoz::kFaddMagicBits;
  constexpr int PREA = kRows * 32, PREB = (int)LCOLS * 32;   // initialising operands (K = 16)
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_dig = smem;                                        // NBUF x kS x ABYTES
  unsigned char* b_dig = a_dig + NBUF * kS * ABYTES;                  // kS x BBYTES
  unsigned char* a_pre = b_dig + kS * BBYTES;                         // PREA: rows (1, 256, 65536, 0...)
  unsigned char* b_pre = a_pre + PREA;                                // PREB: (p0, p1, p2, 0...) per column
  uint64_t* toff = reinterpret_cast<uint64_t*>(b_pre + PREB);         // D
  uint64_t* rowoff = toff + D;                                        // kRows
  uint64_t* tile_base = rowoff + kRows;                               // 2
  uint64_t* mbar = tile_base + 2;                                     // 2
  int* csc = reinterpret_cast<int*>(mbar + 2);                        // N: (column exponent - 2100) << 20
  int* rowexp = csc + N;                                              // 2 x kRows: exponent field of the row maximum
  int* colsum = rowexp + 2 * kRows;                                   // KS x N: digit column sums (setup)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(colsum + kS * N);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  tile_constants<NT, KS, kMagicPre>(p, b_dig, a_pre, b_pre, csc, colsum, toff, rowoff, tid, THREADS);
  const int row_bits = p.tile_bits - NT;
  for (int g = tid; g < kRows; g += THREADS) {
    rowexp[g] = 0;
    rowexp[kRows + g] = 0;
  }
  __syncthreads();
  // column scales as exponent-field increments
  for (int n = tid; n < N; n += THREADS) csc[n] = (int)((unsigned)(csc[n] - 2046 - scale_off<KS>()) << 20);
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
          for (int L = 0; L < kS; ++L)
            bits[L] = kMagicPre ? __float_as_uint(v[L][q]) : __float_as_uint(v[L][q] + 12582912.0f);
          const double r = __ll2double_rn(qsoz::combine_pairs_u<KS, kMB>(bits));
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
      for (int e = 0; e < 4; ++e) {
        const uint32_t* w = R[i + e];
        const uint64_t tr = qsoz::fixed_ks<KS>(w[0], w[1], eg), ti = qsoz::fixed_ks<KS>(w[2], w[3], eg);
        pk[e][0] = pack_bf16(qsoz::top_digit<KS>(tr), qsoz::top_digit<KS>(ti));
        qsoz::packed_digits_fast<KS>(tr, ti, pk[e]);
      }
      const uint32_t off = canon_off16(g, 2 * (l0 + i), K);
#pragma unroll
      for (int s = 0; s < kS; ++s)
        *reinterpret_cast<uint4*>(A + s * ABYTES + off) = make_uint4(pk[0][s], pk[1][s], pk[2][s], pk[3][s]);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t dcol = tmem + (uint32_t)(b * LCOLS);
      mma_full_tile<N, K / 16, KS>(dcol, a_pre, b_pre, A, b_dig);
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
  constexpr size_t smem = (size_t)NBUF * kS * (kRows * K * 2) + (size_t)kS * (N * K * 2) + kRows * 32 +
                          (size_t)kS * N * 32 + 8 * (D + kRows + 4) + 4 * (N + 2 * kRows + kS * N) + 16;
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

// ---------------------------------------------------------------------------
// Warp-specialised form for two to four targets (K <= 32, so the accumulators
// start at the magic and the epilogue reads level bit patterns directly).
// Eight producer warps gather tiles with cp.async into a ring of S staging
// slots (several tiles of loads in flight), take the row maxima (two threads
// per row, one shuffle) and write the digit slices into a ring of NA operand
// buffers; one thread issues the initialising MMA and the slice MMAs of each
// tile into a ring of NTM tensor-memory buffers; eight epilogue warps (two per
// lane quarter, each half of a row's columns) recombine, convert and store.
// Hand-offs are mbarriers: afull (producers -> MMA), aempty and accfull
// (MMA completion -> producers, epilogue), tempty (epilogue -> MMA) and
// mready (MMA thread -> epilogue, releasing onward the row exponents that the
// producers wrote into one of NM = NA + NTM metadata slots; a slot is
// rewritten only after the epilogue has finished the tile that used it).
// Every role steps its tile base by a masked add: with the inserted (target,
// row and control) bit positions filled with ones, adding the grid stride
// spread over the free positions carries through them.  Every wait is bounded
// and gives up when another role has.
// ---------------------------------------------------------------------------
namespace {
constexpr int kWsE = 8, kWsP = 8;                   // epilogue and producer warps
constexpr int kWsThreads = 32 * (kWsE + kWsP + 1);  // and the MMA warp

__device__ __forceinline__ bool wait_ring(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if (spins > kWaitLimit || ((spins & 255u) == 0 && *abort_flag)) return true;
  }
  return false;
}

// the same for a whole warp: every lane gets the same answer, so a warp
// leaves its loop as one (its shuffles and tcgen05.ld need all lanes)
__device__ __forceinline__ bool wait_ring_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return __any_sync(0xFFFFFFFFu, wait_ring(bar, parity, abort_flag)) != 0;
}

template <int NT, int KS>
struct Ws {
  static constexpr int D = 1 << NT, K = 2 * D, N = 2 * D;
  static constexpr int LCOLS = KS * N;
  static constexpr int NTM = NT == 3 ? 4 : 2;        // accumulator buffers
  static constexpr int TSTRIDE = 512 / NTM;          // their column stride
  static constexpr int NA = NT == 3 ? 4 : 2;         // operand buffers
  static constexpr int NM = NA + NTM;                // metadata slots
  static constexpr int S = NT == 3 ? 4 : 2;          // staging slots (64 KB of loads in flight)
  static constexpr int PT = 32 * kWsP;               // producer threads
  static constexpr int EPP = D / 2;                  // amplitudes per producer thread (two per row)
  static constexpr int EPE = D / 2;                  // amplitudes per epilogue thread (two per row)
  static constexpr int ABYTES = kRows * K * 2, BBYTES = N * K * 2;
  static constexpr int SLOT = PT * EPP * 16;
  static constexpr size_t a_off = 0;
  static constexpr size_t b_off = a_off + (size_t)NA * KS * ABYTES;
  static constexpr size_t apre_off = b_off + (size_t)KS * BBYTES;
  static constexpr size_t bpre_off = apre_off + kRows * 32;
  static constexpr size_t stg_off = bpre_off + (size_t)LCOLS * 32;
  static constexpr size_t toff_off = stg_off + (size_t)S * SLOT;
  static constexpr size_t rowoff_off = toff_off + 8 * D;
  static constexpr size_t bar_off = rowoff_off + 8 * kRows;
  static constexpr size_t csc_off = bar_off + 8 * (2 * NA + 2 * NTM + NM);
  static constexpr size_t ex_off = csc_off + 4 * N;
  static constexpr size_t colsum_off = ex_off + 4 * (size_t)NM * kRows;
  static constexpr size_t slot_off = colsum_off + 4 * (size_t)KS * N;
  static constexpr size_t bytes = slot_off + 16;
  static_assert(LCOLS <= TSTRIDE && NTM * TSTRIDE <= 512, "tensor memory");
  static_assert(bytes <= 227 * 1024, "shared memory");
  static_assert(K <= 32 && EPP % 4 == 0 && PT / kRows == 2, "mapping");
};

}  // namespace

template <int NT, int KS>
__global__ void __launch_bounds__(kWsThreads, 1) k_dense_ozaki_ws(double2* __restrict__ psi, const __grid_constant__ TcParams p) {
  using W = Ws<NT, KS>;
  constexpr int K = W::K, N = W::N, NA = W::NA, NTM = W::NTM, NM = W::NM, S = W::S;
  constexpr int EPP = W::EPP, EPE = W::EPE, PT = W::PT;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_dig = smem + W::a_off;
  unsigned char* b_dig = smem + W::b_off;
  unsigned char* a_pre = smem + W::apre_off;
  unsigned char* b_pre = smem + W::bpre_off;
  unsigned char* stg = smem + W::stg_off;
  uint64_t* toff = reinterpret_cast<uint64_t*>(smem + W::toff_off);
  uint64_t* rowoff = reinterpret_cast<uint64_t*>(smem + W::rowoff_off);
  uint64_t* afull = reinterpret_cast<uint64_t*>(smem + W::bar_off);
  uint64_t* aempty = afull + NA;
  uint64_t* accfull = aempty + NA;
  uint64_t* tempty = accfull + NTM;
  uint64_t* mready = tempty + NTM;
  int* csc = reinterpret_cast<int*>(smem + W::csc_off);
  int* meta_ex = reinterpret_cast<int*>(smem + W::ex_off);
  int* colsum = reinterpret_cast<int*>(smem + W::colsum_off);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + W::slot_off);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + W::slot_off + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  tile_constants<NT, KS, true>(p, b_dig, a_pre, b_pre, csc, colsum, toff, rowoff, tid, kWsThreads);
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      mbar_init(afull + j, kWsP);        // one arrival per producer warp
      mbar_init(aempty + j, 1);
    }
#pragma unroll
    for (int k = 0; k < NTM; ++k) {
      mbar_init(accfull + k, 1);
      mbar_init(tempty + k, kWsE);       // one arrival per epilogue warp
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) mbar_init(mready + m, 1);
    *abort_flag = 0;
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  for (int n = tid; n < N; n += kWsThreads) csc[n] = (int)((unsigned)(csc[n] - 2046 - scale_off<KS>()) << 20);
  __syncthreads();
  const uint32_t tmem = *tmem_slot;
  const int row_bits = p.tile_bits - NT;
  const uint64_t grid = gridDim.x;
  // tile bases: x(c) = insert_zeros(c); x(c + d) = ((x(c) | hole) + insert_zeros(d)) & ~hole
  uint64_t hole = 0;
  for (int q = 0; q < p.nhi; ++q) hole |= 1ull << p.hi_ins[q];
  const uint64_t gstep = insert_zeros(grid, p.hi_ins, p.nhi);
  auto step = [&](uint64_t x, uint64_t d) -> uint64_t { return ((x | hole) + d) & ~hole; };

  if (warp < kWsE) {
    // ---- epilogue: row g (tensor-memory lane), amplitudes [eh EPE, (eh + 1) EPE) ----
    const int q = warp & 3, eh = warp >> 2;
    const int g = 32 * q + lane;
    const bool row_ok = g < (1 << row_bits);
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    uint64_t te[EPE];                         // byte offsets of this thread's amplitudes in a tile
#pragma unroll
    for (int i = 0; i < EPE; ++i) te[i] = (rowoff[g] | toff[eh * EPE + i]) << 4;
    uint64_t xb = insert_zeros(blockIdx.x, p.hi_ins, p.nhi);
    for (int i = 0;; ++i, xb = step(xb, gstep)) {
      const uint64_t c = blockIdx.x + (uint64_t)i * grid;
      if (c >= p.ntiles) break;
      const int k = i % NTM, m = i % NM;
      if (wait_ring_warp(mready + m, (uint32_t)(i / NM) & 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      const int egs = meta_ex[m * kRows + g];
      char* tp = reinterpret_cast<char*>(psi) + ((xb | p.ctrl_mask) << 4);
      if (wait_ring_warp(accfull + k, (uint32_t)(i / NTM) & 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      fence_after_sync();
      const uint32_t tb = tmem + (uint32_t)(k * W::TSTRIDE) + lane_addr + (uint32_t)(eh * 2 * EPE);
#pragma unroll
      for (int cc = 0; cc < 2 * EPE; cc += 8) {
        float v[KS][8];
#pragma unroll
        for (int L = 0; L < KS; ++L) tmem_ld8(tb + (uint32_t)(L * N + cc), v[L]);
        tmem_wait_ld();
        if (cc + 8 == 2 * EPE) {                // the buffer is read: hand it back to the MMA thread
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty + k);
        }
        if (row_ok) {
          const int4 s0 = *reinterpret_cast<const int4*>(csc + eh * 2 * EPE + cc);
          const int4 s1 = *reinterpret_cast<const int4*>(csc + eh * 2 * EPE + cc + 4);
          const int scl[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
          double o[8];
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) {
            uint32_t bits[KS];
#pragma unroll
            for (int L = 0; L < KS; ++L) bits[L] = __float_as_uint(v[L][qq]);
            const double r = __ll2double_rn(qsoz::combine_pairs_u<KS, qsoz::kPreMagicBits>(bits));
            const int hi = __double2hiint(r);   // 0 only for r = 0, which stays 0
            o[qq] = __hiloint2double(hi != 0 ? hi + egs + scl[qq] : 0, __double2loint(r));
          }
#pragma unroll
          for (int qq = 0; qq < 8; qq += 2)
            *reinterpret_cast<double2*>(tp + te[(cc + qq) >> 1]) = make_double2(o[qq], o[qq + 1]);
        }
      }
    }
  } else if (warp < kWsE + kWsP) {
    // ---- producers: row g, part h (amplitudes [h EPP, (h + 1) EPP)) ----
    const int pt = tid - 32 * kWsE, pw = pt >> 5;
    const int g = 16 * pw + (lane >> 1), h = lane & 1;
    const bool row_ok = g < (1 << row_bits);
    uint64_t tp[EPP];                         // byte offsets of this thread's amplitudes in a tile
#pragma unroll
    for (int i = 0; i < EPP; ++i) tp[i] = (rowoff[g] | toff[h * EPP + i]) << 4;
    const uint32_t stg_addr = smem_u32(stg) + (uint32_t)pt * 16u;
    auto issue = [&](uint64_t x, int slot) {
      const char* base = reinterpret_cast<const char*>(psi) + ((x | p.ctrl_mask) << 4);
#pragma unroll
      for (int i = 0; i < EPP; ++i)
        cp_async16(stg_addr + (uint32_t)(slot * W::SLOT + i * PT * 16), row_ok ? (const void*)(base + tp[i]) : psi,
                   row_ok ? 16u : 0u);
    };
    uint64_t xi = insert_zeros(blockIdx.x, p.hi_ins, p.nhi);   // base of the next tile to issue
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const uint64_t c = blockIdx.x + (uint64_t)sl * grid;
      if (c < p.ntiles) issue(xi, sl);
      cp_async_commit();
      xi = step(xi, gstep);
    }
    for (int i = 0;; ++i) {
      const uint64_t c = blockIdx.x + (uint64_t)i * grid;
      if (c >= p.ntiles) break;
      const int slot = i % S, j = i % NA, m = i % NM;
      cp_async_wait<S - 1>();
      uint32_t R[EPP][4];
#pragma unroll
      for (int i2 = 0; i2 < EPP; ++i2) {
        uint4 v;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"(stg_addr + (uint32_t)(slot * W::SLOT + i2 * PT * 16)));
        R[i2][0] = v.y;
        R[i2][1] = v.x;
        R[i2][2] = v.w;
        R[i2][3] = v.z;
      }
      // row maximum of the exponent fields (the row's other part is the neighbouring lane)
      uint32_t em = (uint32_t)emax_floor<KS>() << 20;
#pragma unroll
      for (int i2 = 0; i2 < EPP; ++i2) em = max(em, max(R[i2][0] & 0x7FF00000u, R[i2][2] & 0x7FF00000u));
      em = max(em, __shfl_xor_sync(0xFFFFFFFFu, em, 1));
      // the slot's contents are in registers (used above): refill it S tiles ahead
      {
        const uint64_t c2 = c + (uint64_t)S * grid;
        if (c2 < p.ntiles) issue(xi, slot);
        cp_async_commit();
        xi = step(xi, gstep);
      }
      if (wait_ring_warp(aempty + j, ((uint32_t)(i / NA) & 1u) ^ 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      if (h == 0) meta_ex[m * kRows + g] = (int)em;
      const int eg = (int)(em >> 20);
      unsigned char* A = a_dig + j * (KS * W::ABYTES);
#pragma unroll
      for (int i2 = 0; i2 < EPP; i2 += 4) {
        uint32_t pk[4][KS];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t* w = R[i2 + e];
          const uint64_t tr = qsoz::fixed_ks<KS>(w[0], w[1], eg), ti = qsoz::fixed_ks<KS>(w[2], w[3], eg);
          pk[e][0] = pack_bf16(qsoz::top_digit<KS>(tr), qsoz::top_digit<KS>(ti));
          qsoz::packed_digits_fast<KS>(tr, ti, pk[e]);
        }
        const uint32_t off = canon_off16(g, 2 * (h * EPP + i2), K);
#pragma unroll
        for (int sl = 0; sl < KS; ++sl)
          *reinterpret_cast<uint4*>(A + sl * W::ABYTES + off) = make_uint4(pk[0][sl], pk[1][sl], pk[2][sl], pk[3][sl]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(afull + j);
    }
    cp_async_wait<0>();
  } else if (lane == 0) {
    // ---- MMA issue ----
    int last = -1;
    for (int i = 0;; ++i) {
      const uint64_t c = blockIdx.x + (uint64_t)i * grid;
      if (c >= p.ntiles) break;
      const int j = i % NA, k = i % NTM, m = i % NM;
      if (wait_ring(afull + j, (uint32_t)(i / NA) & 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      mbar_arrive(mready + m);              // the producers' metadata, released onward to the epilogue
      if (wait_ring(tempty + k, ((uint32_t)(i / NTM) & 1u) ^ 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      fence_after_sync();
      mma_full_tile<N, K / 16, KS>(tmem + (uint32_t)(k * W::TSTRIDE), a_pre, b_pre, a_dig + j * (KS * W::ABYTES),
                                   b_dig);
      mma_commit(aempty + j);
      mma_commit(accfull + k);
      last = i;
    }
    // the last tile's MMAs are complete before the tensor memory is freed
    if (last >= 0 && wait_ring(aempty + last % NA, (uint32_t)(last / NA) & 1u, abort_flag)) *abort_flag = 1;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (tid == 0 && *abort_flag) atomicExch(p.err, 1);
  if (warp == 0) tmem_dealloc(tmem, 512);
}

template <int NT, int KS>
static cudaError_t dense_ozaki_ws(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr size_t smem = Ws<NT, KS>::bytes;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dense_ozaki_ws<NT, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const uint64_t maxb = (uint64_t)num_sms();
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_ozaki_ws<NT, KS><<<g, kWsThreads, smem, st>>>(static_cast<double2*>(amps), p);
  return cudaGetLastError();
}

// Several independent single-buffered CTAs per SM, whose phases drift apart,
// keep the SM busier than double buffering inside one CTA (measured at 30
// qubits: 3 targets 10.3 ms as four 128-thread CTAs against 12.2 ms as two
// double-buffered 256-thread CTAs; 4 targets 11.2 ms as two 256-thread CTAs
// against 13.9 ms as one double-buffered 512-thread CTA).  Tensor memory
// (seven levels of N columns per buffer) bounds the CTAs per SM.
// Passes of fewer tiles than SMs (small states) go to the single-CTA kernels,
// whose setup is lighter than the warp-specialised kernel's (one tile per CTA
// leaves nothing to pipeline).
cudaError_t launch_dense_ozaki(void* amps, const TcParams& p, int slices, cudaStream_t st) {
  const bool small = p.ntiles < (uint64_t)num_sms();
  if (slices == 8) {
    switch (p.n) {
      case 3: return small ? dense_ozaki_nt<3, 128, 1, 4, 8>(amps, p, st) : dense_ozaki_ws<3, 8>(amps, p, st);
      case 4: return small ? dense_ozaki_nt<4, 256, 1, 2, 8>(amps, p, st) : dense_ozaki_ws<4, 8>(amps, p, st);
      case 5: return dense_ozaki_nt<5, 512, 1, 1, 8>(amps, p, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.n) {
    case 3: return small ? dense_ozaki_nt<3, 128, 1, 4, 7>(amps, p, st) : dense_ozaki_ws<3, 7>(amps, p, st);
    case 4: return small ? dense_ozaki_nt<4, 256, 1, 2, 7>(amps, p, st) : dense_ozaki_ws<4, 7>(amps, p, st);
    case 5: return dense_ozaki_nt<5, 512, 1, 1, 7>(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qsk
