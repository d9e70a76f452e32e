// Composition of consecutive gates into one dense block matrix, in FP64.
//
// A block acts on k <= 6 qubits.  Its matrix is built column by column: start
// from the identity and apply each of the block's gates, in circuit order, to
// every column, as if each column were a k-qubit statevector.  The gate
// updates are the paper's (Sec. "Many-control one-target gate", "Many-target
// gate", "Pauli gadget"), on block-local bit positions.  One CTA per block;
// the matrix lives in shared memory (64 x 64 complex128 = 64 KiB), double
// buffered so that every entry of the next matrix is computed from the last.
#include "qs_device.cuh"

namespace qsk {

__global__ void __launch_bounds__(256) k_block_compose(const ComposeBlock* __restrict__ blocks,
                                                       const ComposeInstr* __restrict__ instrs,
                                                       const double* __restrict__ data, double* __restrict__ out) {
  extern __shared__ __align__(16) double2 sm[];
  const ComposeBlock blk = blocks[blockIdx.x];
  const int D = 1 << blk.k;
  double2* cur = sm;            // column-major: cur[c * D + r]
  double2* nxt = sm + D * D;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int c = e / D, r = e % D;
    cur[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int ii = 0; ii < blk.count; ++ii) {
    const ComposeInstr in = instrs[blk.first + ii];
    uint32_t tmask = 0;
    for (int q = 0; q < in.n; ++q) tmask |= 1u << in.tbit[q];
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
      const int c = e / D, r = e % D;
      const double2* col = cur + c * D;
      double2 v;
      if (in.kind == 0) {                 // dense gate with controls
        if (((uint32_t)r & in.ctrl_mask) != in.ctrl_mask) {
          v = col[r];
        } else {
          int j = 0;
          for (int q = 0; q < in.n; ++q) j |= ((r >> in.tbit[q]) & 1) << q;
          const int rbase = r & ~(int)tmask;
          const int dn = 1 << in.n;
          const double* m = data + in.data_off + 2 * j * dn;
          double sr = 0.0, si = 0.0;
          for (int l = 0; l < dn; ++l) {
            int rr = rbase;
            for (int q = 0; q < in.n; ++q) rr |= ((l >> q) & 1) << in.tbit[q];
            const double2 x = col[rr];
            const double mr = m[2 * l], mi = m[2 * l + 1];
            sr += mr * x.x - mi * x.y;
            si += mr * x.y + mi * x.x;
          }
          v = make_double2(sr, si);
        }
      } else if (in.kind == 1) {          // diagonal
        int j = 0;
        for (int q = 0; q < in.n; ++q) j |= ((r >> in.tbit[q]) & 1) << q;
        const double dr = data[in.data_off + 2 * j], di = data[in.data_off + 2 * j + 1];
        const double2 x = col[r];
        v = make_double2(dr * x.x - di * x.y, dr * x.y + di * x.x);
      } else {                            // Pauli gadget: c x_r + i s beta_{r'} x_{r'}
        const int rp = r ^ in.xy;
        const double2 x = col[r];
        double2 y = rot_i(col[rp], (in.eta + 1) & 3);
        const double sg = (__popc((uint32_t)(rp & in.yz)) & 1) ? -in.s : in.s;
        v = make_double2(in.c * x.x + sg * y.x, in.c * x.y + sg * y.y);
      }
      nxt[e] = v;
    }
    __syncthreads();
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  double* o = out + blk.out_off;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int r = e / D, c = e % D;      // row-major output
    const double2 v = cur[c * D + r];
    o[2 * e] = v.x;
    o[2 * e + 1] = v.y;
  }
}

cudaError_t launch_block_compose(const ComposeBlock* blocks, int nblocks, const ComposeInstr* instrs,
                                 const double* data, double* out, cudaStream_t st) {
  const size_t smem = 2 * sizeof(double2) * 64 * 64;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_block_compose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (nblocks == 0) return cudaSuccess;
  k_block_compose<<<nblocks, 256, smem, st>>>(blocks, instrs, data, out);
  return cudaGetLastError();
}

}  // namespace qsk
