// Dense n-target gates on the 5th-generation tensor cores (tcgen05) for
// complex64 states: the group update alpha_kj -> sum_l m_jl alpha_kl
// (Sec. "Many-target gate", Eq. (local many-target amplitude update)) is, over
// a tile of 128 groups, the real GEMM
//   C[g, 2j + c] = sum_{l, c'} A[g, 2l + c'] B[2l + c', 2j + c]
// with A the groups' interleaved (re, im) amplitudes and B the realified
// matrix (B[2l, 2j] = Re m_jl, B[2l+1, 2j] = -Im m_jl, B[2l, 2j+1] = Im m_jl,
// B[2l+1, 2j+1] = Re m_jl).  It runs as 3xTF32: A = Ah + Al, B = Bh + Bl with
// Ah, Bh exact TF32 values, C = Ah Bh + Ah Bl + Al Bh accumulated in FP32 in
// tensor memory, which keeps FP32-level accuracy.
//
// Work mapping and pipeline as in the complex128 kernel (qs_tc_ozaki.cu):
// thread (warp w, lane) owns tile row g = 32 (w mod 4) + lane (its
// tensor-memory lane) and amplitudes [c EPT, (c+1) EPT), c = w / 4, for the
// gather, the split and the epilogue; operands are written in the canonical
// K-major no-swizzle layout (8-row x 16-byte core matrices) as 16-byte
// vectors; with two operand and accumulator buffers, the loads of tile i + 1
// are issued before the epilogue of tile i - 1, which runs while the tensor
// cores work on tile i.  One thread issues the MMAs and commits them to an
// mbarrier.  Every wait is bounded: on timeout the kernel records an error
// code, frees its tensor memory and returns.
#include "qs_device.cuh"
#include "qs_tc_ptx.cuh"

namespace qsk {
namespace {

using namespace tcptx;

constexpr int kRows = 128;
constexpr uint32_t kWaitLimit = 1u << 26;

__host__ __device__ constexpr uint32_t tc_cols(uint32_t n) {
  return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity))
    if (++spins > kWaitLimit) return true;
  return false;
}

}  // namespace

template <int NT, int THREADS, int NBUF, int CTAS>
__global__ void __launch_bounds__(THREADS, CTAS) k_dense_tc(float2* __restrict__ psi, const __grid_constant__ TcParams p) {
  constexpr int D = 1 << NT;
  constexpr int K = 2 * D;                   // real inputs per group
  constexpr int N = 2 * D;                   // real outputs per group
  constexpr int CG = THREADS / kRows;        // threads per row
  constexpr int EPT = D / CG;                // amplitudes per thread
  constexpr int CPW = 2 * EPT;               // accumulator columns per thread
  static_assert(EPT % 4 == 0, "eight accumulator columns per epilogue step");
  constexpr int OPB = kRows * K * 4;         // bytes of one A operand (hi or lo)
  constexpr int BPB = N * K * 4;             // bytes of one B operand
  constexpr uint32_t TCOLS = tc_cols(NBUF * N);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_op = smem;                                         // NBUF x (hi, lo)
  unsigned char* b_hi = a_op + NBUF * 2 * OPB;
  unsigned char* b_lo = b_hi + BPB;
  uint64_t* toff = reinterpret_cast<uint64_t*>(b_lo + BPB);          // D
  uint64_t* rowoff = toff + D;                                        // kRows
  uint64_t* tile_base = rowoff + kRows;                               // 2
  uint64_t* mbar = tile_base + 2;                                     // 2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B = realified matrix, split into TF32 halves, once per CTA.
  for (int e = tid; e < N * K; e += THREADS) {
    const int n = e / K, k = e % K;
    int j = n >> 1, l = k >> 1, Dm = D;
    const int c = n & 1, cp = k & 1;
    double v = 0.0;
    if (p.nmat < p.n) {                       // identity on the extra targets
      Dm = 1 << p.nmat;
      if ((j >> p.nmat) != (l >> p.nmat)) Dm = 0;
      j &= (1 << p.nmat) - 1;
      l &= (1 << p.nmat) - 1;
    }
    if (Dm) {
      const double mr = p.mat[2 * (j * Dm + l)];
      const double mi = p.conj ? -p.mat[2 * (j * Dm + l) + 1] : p.mat[2 * (j * Dm + l) + 1];
      v = (c == 0) ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr);
    }
    const float f = (float)v;
    const float h = tf32_hi(f);
    const uint32_t off = canon_off(n, k, K);
    *reinterpret_cast<float*>(b_hi + off) = h;
    *reinterpret_cast<float*>(b_lo + off) = f - h;
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
  }
  if (tid == 0) {
    tile_base[0] = insert_zeros(blockIdx.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    if (blockIdx.x + gridDim.x < p.ntiles)
      tile_base[1] = insert_zeros(blockIdx.x + gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(mbar + b, 1);
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
  const uint32_t idesc = idesc_tf32(kRows, N);
  constexpr uint32_t sbo = K * 32;

  const int g = 32 * (warp & 3) + lane;       // row (tensor-memory lane)
  const int cg = warp >> 2;
  const int l0 = cg * EPT;
  const bool row_ok = g < (1 << row_bits);
  const uint64_t roff = rowoff[g];
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const int helper = THREADS > kRows ? kRows : 0;
  uint64_t toffr[EPT];
#pragma unroll
  for (int i = 0; i < EPT; ++i) toffr[i] = toff[l0 + i];
  // When the lowest target bits are the lowest qubits in order, a thread's
  // amplitudes are consecutive in memory (and start on an even index): move
  // them two at a time (16 bytes).  The test depends on l mod EPT only, so it
  // is the same in every thread.
  bool vec = true;
#pragma unroll
  for (int i = 1; i < EPT; ++i) vec = vec && toffr[i] == toffr[0] + (uint64_t)i;

  float2 R[EPT];
  auto load_tile = [&](uint64_t base) {
    const uint64_t rb = base | roff;
    if (vec) {
#pragma unroll
      for (int i = 0; i < EPT; i += 2) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (row_ok) v = *reinterpret_cast<const float4*>(psi + (rb | toffr[i]));
        R[i] = make_float2(v.x, v.y);
        R[i + 1] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < EPT; ++i) R[i] = row_ok ? psi[rb | toffr[i]] : make_float2(0.0f, 0.0f);
    }
  };
  auto epilogue = [&](uint32_t tbuf, uint64_t rb) {
#pragma unroll
    for (int cc = 0; cc < CPW; cc += 8) {
      float v[8];
      tmem_ld8(tmem + tbuf + lane_addr + (uint32_t)(cg * CPW + cc), v);
      tmem_wait_ld();
      if (row_ok) {
        if (vec) {
#pragma unroll
          for (int q = 0; q < 8; q += 4)
            *reinterpret_cast<float4*>(psi + (rb | toffr[(cc + q) >> 1])) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; q += 2) psi[rb | toffr[(cc + q) >> 1]] = make_float2(v[q], v[q + 1]);
        }
      }
    }
  };

  load_tile(tile_base[0]);
  uint32_t phases = 0;
  bool failed = false;
  int it = 0;
  uint64_t rb_prev = 0;
  for (uint64_t c = blockIdx.x; c < p.ntiles; c += gridDim.x, ++it) {
    const int b = NBUF == 2 ? (it & 1) : 0;
    const int par = it & 1;
    const uint64_t rb = tile_base[par] | roff;
    const bool has_next = c + gridDim.x < p.ntiles;
    // TF32 halves of this thread's amplitudes, 16 bytes (two amplitudes) per store
    unsigned char* ahi = a_op + b * (2 * OPB);
    unsigned char* alo = ahi + OPB;
#pragma unroll
    for (int i = 0; i < EPT; i += 2) {
      const float hx0 = tf32_hi(R[i].x), hy0 = tf32_hi(R[i].y);
      const float hx1 = tf32_hi(R[i + 1].x), hy1 = tf32_hi(R[i + 1].y);
      const uint32_t off = canon_off(g, 2 * (l0 + i), K);
      *reinterpret_cast<float4*>(ahi + off) = make_float4(hx0, hy0, hx1, hy1);
      *reinterpret_cast<float4*>(alo + off) =
          make_float4(R[i].x - hx0, R[i].y - hy0, R[i + 1].x - hx1, R[i + 1].y - hy1);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint64_t dah = smem_desc(smem_u32(ahi), 128, sbo), dal = smem_desc(smem_u32(alo), 128, sbo);
      const uint64_t dbh = smem_desc(smem_u32(b_hi), 128, sbo), dbl = smem_desc(smem_u32(b_lo), 128, sbo);
      const uint32_t d = tmem + (uint32_t)(b * N);
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk)     // Al Bh
        mma_tf32(d, dal + (kk * 256 >> 4), dbh + (kk * 256 >> 4), idesc, kk != 0);
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk)     // Ah Bl
        mma_tf32(d, dah + (kk * 256 >> 4), dbl + (kk * 256 >> 4), idesc, 1);
#pragma unroll
      for (int kk = 0; kk < K / 8; ++kk)     // Ah Bh
        mma_tf32(d, dah + (kk * 256 >> 4), dbh + (kk * 256 >> 4), idesc, 1);
      mma_commit(mbar + b);
    }
    // loads of the next tile, in flight during the MMAs and the epilogue
    if (has_next) load_tile(tile_base[par ^ 1]);
    bool timed_out = false;
    if (NBUF == 2) {
      if (it > 0) {
        const int pb = b ^ 1;
        timed_out = tc_wait(mbar + pb, (phases >> pb) & 1u);
        phases ^= 1u << pb;
        fence_after_sync();
        epilogue((uint32_t)(pb * N), rb_prev);
      }
    } else {
      timed_out = tc_wait(mbar, phases & 1u);
      phases ^= 1u;
      fence_after_sync();
      epilogue(0u, rb);
    }
    rb_prev = rb;
    if (tid == helper && c + 2 * (uint64_t)gridDim.x < p.ntiles)
      tile_base[par] = insert_zeros(c + 2 * (uint64_t)gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    fence_before_sync();
    failed = __syncthreads_or(timed_out) != 0;
    fence_after_sync();
    if (failed) break;
  }
  if (NBUF == 2 && !failed && it > 0) {
    const int pb = (it - 1) & 1;
    const bool timed_out = tc_wait(mbar + pb, (phases >> pb) & 1u);
    fence_after_sync();
    epilogue((uint32_t)(pb * N), rb_prev);
    fence_before_sync();
    failed = __syncthreads_or(timed_out) != 0;
  }
  if (failed && tid == 0) atomicExch(p.err, 1);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// ---------------------------------------------------------------------------
// Six targets (K = N = 128).  3xTF32 operands would need 256 KB of shared
// memory, so A and B are cut into three bf16 slices each instead: x = x0 + x1
// + x2, each slice the bf16 rounding of what the previous ones left (8
// significant bits each, exact remainders in FP32).  The six products with
// s + t <= 2 accumulate in FP32 in tensor memory (kind::f16, bf16 inputs); the
// dropped products are below 2^-26 of |A| |B|.  The leading product x0 y0 has
// an accumulator of its own and the five corrections share a second one, 2^-8
// smaller, so the tensor cores' accumulation rounding acts mostly on eight
// steps of the leading sum; the epilogue adds the two.  Same mapping and
// bounded waits as above; one buffer of slices (192 KB), one CTA of 512
// threads per SM.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// three packed (re, im) bf16 slices of one amplitude
__device__ __forceinline__ void bf16_slices(float2 v, uint32_t* out) {
  float r = v.x, i = v.y;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const uint32_t w = bf16x2_rn(r, i);
    out[s] = w;
    r -= __uint_as_float(w << 16);
    i -= __uint_as_float(w & 0xFFFF0000u);
  }
}
}  // namespace

__global__ void __launch_bounds__(512, 1) k_dense_tc6(float2* __restrict__ psi, const __grid_constant__ TcParams p) {
  constexpr int NT = 6, D = 64, K = 128, N = 128, THREADS = 512;
  constexpr int CG = THREADS / kRows;        // 4
  constexpr int EPT = D / CG;                // 16 amplitudes per thread
  constexpr int CPW = 2 * EPT;               // 32 accumulator columns per thread
  constexpr int SL = kRows * K * 2;          // one bf16 slice of A (32 KB)
  constexpr int SB = N * K * 2;              // one bf16 slice of B (32 KB)
  constexpr uint32_t TCOLS = 256;             // leading product | corrections
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_sl = smem;                                           // 3 x SL
  unsigned char* b_sl = a_sl + 3 * SL;                                  // 3 x SB
  uint64_t* toff = reinterpret_cast<uint64_t*>(b_sl + 3 * SB);          // D
  uint64_t* rowoff = toff + D;                                          // kRows
  uint64_t* tile_base = rowoff + kRows;                                 // 2
  uint64_t* mbar = tile_base + 2;                                       // 1 (+1 pad)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < N * K; e += THREADS) {
    const int n = e / K, k = e % K;
    const int j = n >> 1, c = n & 1, l = k >> 1, cp = k & 1;
    const double mr = p.mat[2 * (j * D + l)];
    const double mi = p.conj ? -p.mat[2 * (j * D + l) + 1] : p.mat[2 * (j * D + l) + 1];
    float v = (float)((c == 0) ? (cp == 0 ? mr : -mi) : (cp == 0 ? mi : mr));
    const uint32_t off = canon_off16(n, k, K);
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      const uint32_t w = bf16x2_rn(v, 0.0f);
      *reinterpret_cast<uint16_t*>(b_sl + sl * SB + off) = (uint16_t)(w & 0xFFFFu);
      v -= __uint_as_float(w << 16);
    }
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
  }
  if (tid == 0) {
    tile_base[0] = insert_zeros(blockIdx.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    if (blockIdx.x + gridDim.x < p.ntiles)
      tile_base[1] = insert_zeros(blockIdx.x + gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    mbar_init(mbar, 1);
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
  const uint32_t idesc = idesc_bf16(kRows, N);
  constexpr uint32_t sbo = K * 16;

  const int g = 32 * (warp & 3) + lane;
  const int cg = warp >> 2;
  const int l0 = cg * EPT;
  const bool row_ok = g < (1 << row_bits);
  const uint64_t roff = rowoff[g];
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  const int helper = kRows;

  float2 R[EPT];
  auto load_tile = [&](uint64_t base) {
    const uint64_t rb = base | roff;
#pragma unroll
    for (int i = 0; i < EPT; ++i) R[i] = row_ok ? psi[rb | toff[l0 + i]] : make_float2(0.0f, 0.0f);
  };

  load_tile(tile_base[0]);
  uint32_t phase = 0;
  bool failed = false;
  int it = 0;
  for (uint64_t c = blockIdx.x; c < p.ntiles; c += gridDim.x, ++it) {
    const int par = it & 1;
    const uint64_t rb = tile_base[par] | roff;
    const bool has_next = c + gridDim.x < p.ntiles;
#pragma unroll
    for (int i = 0; i < EPT; i += 4) {
      uint32_t w[4][3];
#pragma unroll
      for (int e = 0; e < 4; ++e) bf16_slices(R[i + e], w[e]);
      const uint32_t off = canon_off16(g, 2 * (l0 + i), K);
#pragma unroll
      for (int sl = 0; sl < 3; ++sl)
        *reinterpret_cast<uint4*>(a_sl + sl * SL + off) = make_uint4(w[0][sl], w[1][sl], w[2][sl], w[3][sl]);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint64_t da = smem_desc(smem_u32(a_sl), 128, sbo), db = smem_desc(smem_u32(b_sl), 128, sbo);
      // products (s, t) with s + t <= 2: (0, 0) into columns 0..127, the rest into 128..255
      constexpr int PS[6] = {0, 0, 1, 0, 1, 2}, PT[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int pr = 0; pr < 6; ++pr)
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk)
          mma_bf16(tmem + (pr == 0 ? 0u : (uint32_t)N), da + ((PS[pr] * SL + kk * 256) >> 4),
                   db + ((PT[pr] * SB + kk * 256) >> 4), idesc, (pr > 1 || kk != 0) ? 1u : 0u);
      mma_commit(mbar);
    }
    if (has_next) load_tile(tile_base[par ^ 1]);
    const bool timed_out = tc_wait(mbar, phase);
    phase ^= 1u;
    fence_after_sync();
#pragma unroll
    for (int cc = 0; cc < CPW; cc += 8) {
      float v[8], w[8];
      tmem_ld8(tmem + lane_addr + (uint32_t)(cg * CPW + cc), v);
      tmem_ld8(tmem + lane_addr + (uint32_t)(N + cg * CPW + cc), w);
      tmem_wait_ld();
      if (row_ok) {
#pragma unroll
        for (int q = 0; q < 8; q += 2)
          psi[rb | toff[l0 + ((cc + q) >> 1)]] = make_float2(v[q] + w[q], v[q + 1] + w[q + 1]);
      }
    }
    if (tid == helper && c + 2 * (uint64_t)gridDim.x < p.ntiles)
      tile_base[par] = insert_zeros(c + 2 * (uint64_t)gridDim.x, p.hi_ins, p.nhi) | p.ctrl_mask;
    fence_before_sync();
    failed = __syncthreads_or(timed_out) != 0;
    fence_after_sync();
    if (failed) break;
  }
  if (failed && tid == 0) atomicExch(p.err, 1);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

static cudaError_t dense_tc6(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr size_t smem = 3 * (size_t)kRows * 128 * 2 + 3 * (size_t)128 * 128 * 2 + 8 * (64 + kRows + 4) + 16;
  static_assert(smem <= 227 * 1024, "shared memory");
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc6, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const uint64_t maxb = (uint64_t)num_sms();
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_tc6<<<g, 512, smem, st>>>(static_cast<float2*>(amps), p);
  return cudaGetLastError();
}

template <int NT, int THREADS, int NBUF, int CTAS>
static cudaError_t dense_tc_nt(void* amps, const TcParams& p, cudaStream_t st) {
  constexpr int D = 1 << NT, K = 2 * D, N = 2 * D;
  constexpr size_t smem = (size_t)NBUF * 2 * kRows * K * 4 + 2 * (size_t)N * K * 4 + 8 * (D + kRows + 4) + 16;
  static_assert(smem * CTAS <= 227 * 1024, "shared memory");
  static_assert(CTAS * tc_cols(NBUF * N) <= 512, "tensor memory");
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc<NT, THREADS, NBUF, CTAS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const uint64_t maxb = (uint64_t)num_sms() * CTAS;
  const unsigned g = (unsigned)(p.ntiles < maxb ? p.ntiles : maxb);
  k_dense_tc<NT, THREADS, NBUF, CTAS><<<g, THREADS, smem, st>>>(static_cast<float2*>(amps), p);
  return cudaGetLastError();
}

// Launch shapes measured at 30 qubits (random targets): 3 targets 2.59 ms as
// six single-buffered 128-thread CTAs per SM (3.26 ms as three double-buffered
// 256-thread ones), 4 targets 3.17 ms as two double-buffered 512-thread CTAs,
// 5 targets 3.28 ms as two single-buffered 256-thread CTAs (3.65 ms as one
// double-buffered 512-thread CTA).
cudaError_t launch_dense_tc(void* amps, const TcParams& p, cudaStream_t st) {
  switch (p.n) {
    case 3: return dense_tc_nt<3, 128, 1, 6>(amps, p, st);
    case 4: return dense_tc_nt<4, 512, 2, 2>(amps, p, st);
    case 5: return dense_tc_nt<5, 256, 1, 2>(amps, p, st);
    case 6: return dense_tc6(amps, p, st);
    default: return cudaErrorInvalidValue;
  }
}

// A test of the bounded-wait path: one thread waits on an mbarrier that
// nothing arrives at, gives up after `polls` polls, and sets the error word as
// the tensor-core kernels do when a wait runs out.
__global__ void k_test_wait_timeout(int* err, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tcptx::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    uint32_t spins = 0;
    bool ran_out = false;
    while (!tcptx::mbar_try_wait(&bar, 0u))
      if (++spins > polls) {
        ran_out = true;
        break;
      }
    if (ran_out) atomicExch(err, 1);
  }
}

cudaError_t launch_test_wait_timeout(int* err, uint32_t polls, cudaStream_t st) {
  k_test_wait_timeout<<<1, 32, 0, st>>>(err, polls);
  return cudaGetLastError();
}

}  // namespace qsk
