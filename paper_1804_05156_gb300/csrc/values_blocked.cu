// Owner-computes value kernel: one CTA per block of rows (see blockplan.cu).
//
// 1. Stage the coordinates of every vertex the block's elements use in shared memory (each vertex is
//    read from HBM once per block, coalesced through the block's vertex list).
// 2. For sub-batches of the block's element list: compute the local stiffness and load entries of
//    each element into shared memory, then let each owned row add the entries of its incidences in
//    this sub-batch into its shared-memory accumulator, in ascending element order.
// 3. Write every owned row once: val[row_ptr[R] + p] (coalesced along the row) and b[R].
// No atomics; the summation order of every CSR entry is fixed by the plan (deterministic).
#include <cuda_runtime.h>

#include "common.cuh"
#include "element.cuh"

namespace fem {

namespace {

constexpr int BT = 256;  // threads per CTA

struct BlkArgs {
  int64_t N, NT, E;
  int V, SB;
  const int32_t* order;
  const int32_t* rec_off;
  const uint8_t* dpos;
  const int32_t* eoff;
  const int32_t* voff;
  const int32_t* elist;
  const uint16_t* lelem;
  const int32_t* vlist;
  const uint32_t* rec;
  const int32_t* row_ptr;
  int xs_bytes, ev_bytes, acc_bytes;  // shared-memory carve-up
};

struct RowMeta {
  int off, cur, end, rp, R, rl_dp;  // accumulator offset, record cursor/end, row_ptr, vertex, rowlen | dpos << 8
};

template <int D>
__global__ void __launch_bounds__(BT) k_blocked(BlkArgs a, const double* __restrict__ node, const double* __restrict__ k,
                                                int f_kind, const double* __restrict__ f_arg, double* __restrict__ val,
                                                double* __restrict__ bvec, int* __restrict__ err) {
  constexpr int D1 = D + 1, U = D1 * (D1 + 1) / 2, W = U + D1;
  extern __shared__ __align__(16) unsigned char sm[];
  double* xs = reinterpret_cast<double*>(sm);
  double* ev = reinterpret_cast<double*>(sm + a.xs_bytes);
  double* acc = reinterpret_cast<double*>(sm + a.xs_bytes + a.ev_bytes);
  double* bacc = reinterpret_cast<double*>(sm + a.xs_bytes + a.ev_bytes + a.acc_bytes);
  RowMeta* meta = reinterpret_cast<RowMeta*>(bacc + a.V);
  __shared__ int scan_tmp[BT];

  const int blk = blockIdx.x;
  const int e0 = a.eoff[blk], ne = a.eoff[blk + 1] - e0;
  const int v0 = a.voff[blk], nv = a.voff[blk + 1] - v0;
  const int64_t p0 = (int64_t)blk * a.V;
  const int nown = (int)((a.N - p0) < a.V ? (a.N - p0) : a.V);
  const int tid = threadIdx.x;

  for (int v = tid; v < nv; v += BT) {
    const int64_t R = a.vlist[v0 + v];
#pragma unroll
    for (int m = 0; m < D; ++m) xs[v * D + m] = __ldg(node + R * D + m);
  }
  // owned rows: contiguous chunk of rows per thread for the offset scan
  const int rpt = (nown + BT - 1) / BT;
  const int r0 = tid * rpt, r1 = (r0 + rpt < nown) ? r0 + rpt : nown;
  int mysum = 0;
  for (int r = r0; r < r1; ++r) {
    const int R = a.order[p0 + r];
    const int rp = a.row_ptr[R];
    const int rl = a.row_ptr[R + 1] - rp;
    meta[r].cur = a.rec_off[p0 + r];
    meta[r].end = a.rec_off[p0 + r + 1];
    meta[r].rp = rp;
    meta[r].R = R;
    meta[r].rl_dp = rl | ((int)a.dpos[p0 + r] << 8);
    mysum += rl;
  }
  scan_tmp[tid] = mysum;
  __syncthreads();
  for (int o = 1; o < BT; o <<= 1) {
    const int v = (tid >= o) ? scan_tmp[tid - o] : 0;
    __syncthreads();
    scan_tmp[tid] += v;
    __syncthreads();
  }
  int off = scan_tmp[tid] - mysum;
  const int total_acc = scan_tmp[BT - 1];
  for (int r = r0; r < r1; ++r) {
    meta[r].off = off;
    off += meta[r].rl_dp & 0xff;
  }
  for (int q = tid; q < total_acc; q += BT) acc[q] = 0.0;
  for (int r = tid; r < nown; r += BT) bacc[r] = 0.0;
  __syncthreads();

  const bool want_a = val != nullptr, want_b = bvec != nullptr;
  for (int sb = 0; sb < ne; sb += a.SB) {
    const int nb = (ne - sb < a.SB) ? ne - sb : a.SB;
    for (int e = tid; e < nb; e += BT) {
      const int64_t idx = e0 + sb + e;
      const int64_t t = a.elist[idx];
      double x[D1][D];
#pragma unroll
      for (int i = 0; i < D1; ++i) {
        const int lv = a.lelem[(int64_t)i * a.E + idx];
#pragma unroll
        for (int m = 0; m < D; ++m) x[i][m] = xs[lv * D + m];
      }
      Local<D> L;
      if (!element_local<D>(x, k ? __ldg(k + t) : 1.0, want_a, want_b, f_kind, f_arg, t, L)) report(err, FEM_ERR_DEGENERATE);
      double* dst = ev + (int64_t)e * W;
      if (want_a) {
#pragma unroll
        for (int c = 0; c < U; ++c) dst[c] = L.a[c];
      }
      if (want_b) {
#pragma unroll
        for (int i = 0; i < D1; ++i) dst[U + i] = L.bt[i];
      }
    }
    __syncthreads();
    const int sb_end = sb + nb;
    for (int r = tid; r < nown; r += BT) {
      RowMeta m = meta[r];
      const int dp = m.rl_dp >> 8;
      double ba = bacc[r];
      int c = m.cur;
      for (; c < m.end; ++c) {
        const uint32_t rc = a.rec[c];
        const int e = (int)(rc & 0x7fff);
        if (e >= sb_end) break;
        const double* src = ev + (int64_t)(e - sb) * W;
        const int i = (rc >> 15) & 3;
        if (want_a) {
          acc[m.off + dp] += src[pidx_rt<D>(i, i)];
          int sh = 17;
#pragma unroll
          for (int j = 0; j < D1; ++j) {
            if (j == i) continue;
            const int pos = (rc >> sh) & 31;
            acc[m.off + pos] += src[pidx_rt<D>(i, j)];
            sh += 5;
          }
        }
        if (want_b) ba += src[U + i];
      }
      meta[r].cur = c;
      bacc[r] = ba;
    }
    __syncthreads();
  }
  // write-out: flattened over the block's accumulator entries, coalesced along each row
  if (want_a) {
    for (int q = tid; q < total_acc; q += BT) {
      int lo = 0, hi = nown - 1;  // last row with off <= q
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (meta[mid].off <= q) lo = mid;
        else hi = mid - 1;
      }
      val[meta[lo].rp + (q - meta[lo].off)] = acc[q];
    }
  }
  if (want_b)
    for (int r = tid; r < nown; r += BT) bvec[meta[r].R] = bacc[r];
}

}  // namespace

int assemble_blocked(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                     double* val, double* b, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  const BlockPlan& B = P->blk;
  if (P->NT == 0 || B.nblocks == 0) {
    if (val && P->nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P->nnz, s));
    if (b && P->N > 0) FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * P->N, s));
    return FEM_OK;
  }
  const int D = P->d, D1 = D + 1, W = D1 * (D1 + 1) / 2 + D1;
  BlkArgs a;
  a.N = P->N;
  a.NT = P->NT;
  a.E = B.E;
  a.V = B.V;
  a.order = B.order;
  a.rec_off = B.rec_off;
  a.dpos = B.dpos;
  a.eoff = B.eoff;
  a.voff = B.voff;
  a.elist = B.elist;
  a.lelem = B.lelem;
  a.vlist = B.vlist;
  a.rec = B.rec;
  a.row_ptr = P->row_ptr;
  const int budget = 200 * 1024;
  a.xs_bytes = ((B.max_v * D * 8) + 15) / 16 * 16;
  a.acc_bytes = ((B.max_acc * 8) + 15) / 16 * 16;
  const int fixed = a.xs_bytes + a.acc_bytes + B.V * 8 + B.V * (int)sizeof(RowMeta);
  int sbmax = (budget - fixed) / (W * 8);
  if (sbmax < 32) return set_error(FEM_ERR_STATE, "block too large for shared memory");
  a.SB = sbmax < B.max_e ? (sbmax / 32) * 32 : B.max_e;
  if (a.SB < 1) a.SB = 1;
  a.ev_bytes = ((a.SB * W * 8) + 15) / 16 * 16;
  const int smem = fixed + a.ev_bytes;
  if (D == 2) {
    FEM_CUDA(cudaFuncSetAttribute(k_blocked<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FEM_LAUNCH(k_blocked<2>, B.nblocks, BT, smem, s, a, node, k, f_kind, f_arg, val, b, err);
  } else {
    FEM_CUDA(cudaFuncSetAttribute(k_blocked<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    FEM_LAUNCH(k_blocked<3>, B.nblocks, BT, smem, s, a, node, k, f_kind, f_arg, val, b, err);
  }
  return FEM_OK;
}

}  // namespace fem
