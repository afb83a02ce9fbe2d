// Owner-computes value kernel: one CTA per block of rows (see blockplan.cu), float-float arithmetic.
//
// 1. Stage every vertex the block's elements use in shared memory, once per block: the exact
//    three-float split of its coordinates and, for the sine-product load, sin/cos(pi x/2) of each
//    coordinate (the edge midpoints then need only angle additions).
// 2. For sub-batches of the block's element list: compute each element's local stiffness and load
//    entries (element_df.cuh) into shared memory, then let each owned row add the entries of its
//    incidences in this sub-batch into its shared-memory accumulator, in ascending element order.
// 3. Write every owned row once: val[row_ptr[R] + p] (coalesced along the row) and b[R], converting
//    float-float to double with integer operations.
// No atomics and no FP64 instructions; the summation order of every CSR entry is fixed by the plan.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "common.cuh"
#include "element_df.cuh"

namespace fem {

namespace {

static __device__ float4 g_sincos_tab[kSinTabN + 1];
std::mutex g_tab_mu;
bool g_tab_ready[64] = {false};

// sin(pi k/2048), cos(pi k/2048) for k = 0..1024, as float pairs, on the current device (once).
int ensure_sincos_table() {
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(FEM_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (g_tab_ready[dev]) return FEM_OK;
  static float4 host[kSinTabN + 1];
  const double pi = 3.14159265358979323846;
  for (int k = 0; k <= kSinTabN; ++k) {
    const double a = pi * (double)k / 2048.0;
    const double s = std::sin(a), c = std::cos(a);
    const float sh = (float)s, ch = (float)c;
    host[k] = make_float4(sh, (float)(s - (double)sh), ch, (float)(c - (double)ch));
  }
  // exact values where they are known
  host[0] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  host[kSinTabN] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
  FEM_CUDA(cudaMemcpyToSymbol(g_sincos_tab, host, sizeof(host)));
  g_tab_ready[dev] = true;
  return FEM_OK;
}

}  // namespace

// Device address of the sin/cos table on the current device (filled on first use); nullptr on failure.
const float4* sincos_table_device() {
  static std::atomic<const float4*> addr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (const float4* p = addr[dev].load(std::memory_order_acquire)) return p;
  if (ensure_sincos_table() != FEM_OK) return nullptr;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_sincos_tab) != cudaSuccess) return nullptr;
  addr[dev].store(static_cast<const float4*>(p), std::memory_order_release);
  return static_cast<const float4*>(p);
}

namespace {

struct BlkArgs {
  int N, NT, E;
  int V, SB, nblocks;
  const int32_t* order;
  const int32_t* rec_off;
  const int32_t* rowp;    // row_ptr of each owned row, locality order
  const uint16_t* rldp;   // row length | diagonal position << 8, locality order
  const int32_t* eoff;
  const int32_t* voff;
  const int32_t* elist;
  const uint16_t* lelem;
  const int32_t* vlist;
  const uint32_t* rec;
  const int32_t* row_ptr;
  int xs_bytes, sc_bytes, ev_bytes, acc_bytes;  // shared-memory carve-up
  int rec_bytes, el_bytes, max_e;                // block records; per-element coefficient, id, local vertices
};

struct RowMeta {
  int off, cur, end, rp, R, rl_dp;  // accumulator offset, record cursor/end, row_ptr, vertex, rowlen | dpos << 8
};

template <int D, int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB) k_blocked_df(BlkArgs a, const double* __restrict__ node, const double* __restrict__ k,
                                                   int f_kind, const double* __restrict__ f_arg, double* __restrict__ val,
                                                   double* __restrict__ bvec, int* __restrict__ err,
                                                   int* __restrict__ work) {
  constexpr int D1 = D + 1, U = D1 * (D1 + 1) / 2, W = U + D1;
  extern __shared__ __align__(16) unsigned char sm[];
  VtxDF<D>* xs = reinterpret_cast<VtxDF<D>*>(sm);
  SC* scs = reinterpret_cast<SC*>(sm + a.xs_bytes);
  df2* ev = reinterpret_cast<df2*>(sm + a.xs_bytes + a.sc_bytes);
  df2* acc = reinterpret_cast<df2*>(sm + a.xs_bytes + a.sc_bytes + a.ev_bytes);
  df2* bacc = reinterpret_cast<df2*>(sm + a.xs_bytes + a.sc_bytes + a.ev_bytes + a.acc_bytes);
  RowMeta* meta = reinterpret_cast<RowMeta*>(bacc + a.V);
  unsigned char* tail = reinterpret_cast<unsigned char*>(meta + a.V);
  uint32_t* srec = reinterpret_cast<uint32_t*>(tail);                            // the block's records
  double* sk = reinterpret_cast<double*>(tail + a.rec_bytes);                  // k of each listed element
  int* st = reinterpret_cast<int*>(tail + a.rec_bytes + a.max_e * 8);          // element ids
  uint16_t* slv = reinterpret_cast<uint16_t*>(tail + a.rec_bytes + a.max_e * 12);  // local vertex ids
  int* gidx = reinterpret_cast<int*>(tail + a.rec_bytes + a.el_bytes);  // CSR position of each acc entry
  __shared__ int warp_tot[BT / 32];
  const float4* tab = g_sincos_tab;
  __shared__ int s_blk;
  // One block per CTA, or (work != nullptr) a persistent CTA that takes blocks from a device counter
  // until none are left: CTAs that draw small blocks take more of them.
  for (int it = 0;; ++it) {
  if (work) {
    __syncthreads();
    if (threadIdx.x == 0) s_blk = atomicAdd(work, 1);
    __syncthreads();
  } else if (it > 0) {
    break;
  }
  const int blk = work ? s_blk : (int)blockIdx.x;
  if (blk >= a.nblocks) break;
  const int e0 = a.eoff[blk], ne = a.eoff[blk + 1] - e0;
  const int v0 = a.voff[blk], nv = a.voff[blk + 1] - v0;
  const int p0 = blk * a.V;
  const int nown = (a.N - p0) < a.V ? (a.N - p0) : a.V;
  const int tid = threadIdx.x;
  const bool sinprod2 = (D == 2) && f_kind == FEM_F_SINPROD;

  for (int v = tid; v < nv; v += BT) {
    const int R = a.vlist[v0 + v];
    VtxDF<D> x;
    stage_vertex<D>(x, node + (size_t)R * D);
    xs[v] = x;
    if constexpr (D == 2) {
      if (sinprod2) {
        df2 Pv[4];
        sin_products(sincospi_half(split3(x.x[0]), tab), sincospi_half(split3(x.x[1]), tab), Pv);
#pragma unroll
        for (int c = 0; c < 4; ++c) reinterpret_cast<df2*>(scs)[v * 4 + c] = Pv[c];
      }
    }
  }
  // the block's records and element data, loaded once, coalesced (their latency overlaps the staging)
  const int rbase = a.rec_off[p0];
  const int nrec = a.rec_off[p0 + nown] - rbase;
  for (int q = tid; q < nrec; q += BT) srec[q] = __ldg(a.rec + rbase + q);
  const bool want_k = (k != nullptr) && (val != nullptr);
  for (int e = tid; e < ne; e += BT) {
    const int t = __ldg(a.elist + e0 + e);
    st[e] = t;
#pragma unroll
    for (int i = 0; i < D1; ++i) slv[e * D1 + i] = __ldg(a.lelem + i * a.E + e0 + e);
    if (want_k) sk[e] = __ldg(k + t);
  }
  // owned rows: contiguous chunk of rows per thread for the offset scan
  const int rpt = (nown + BT - 1) / BT;
  const int r0 = tid * rpt, r1 = (r0 + rpt < nown) ? r0 + rpt : nown;
  int mysum = 0;
  for (int r = r0; r < r1; ++r) {
    const int rl_dp = a.rldp[p0 + r];
    meta[r].cur = a.rec_off[p0 + r];
    meta[r].end = a.rec_off[p0 + r + 1];
    meta[r].rp = a.rowp[p0 + r];
    meta[r].R = a.order[p0 + r];
    meta[r].rl_dp = rl_dp;
    mysum += rl_dp & 0xff;
  }
  // block-wide exclusive scan of the row lengths (warp shuffles, then the warp totals)
  const int lane = tid & 31, wid = tid >> 5;
  int inc = mysum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < BT / 32) ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    if (lane < BT / 32) warp_tot[lane] = wi - w;
  }
  __syncthreads();
  int off = warp_tot[wid] + inc - mysum;
  for (int r = r0; r < r1; ++r) {
    meta[r].off = off;
    const int rl = meta[r].rl_dp & 0xff;
    const int rp = meta[r].rp;
    for (int q = 0; q < rl; ++q) gidx[off + q] = rp + q;
    off += rl;
  }
  __syncthreads();
  const int total_acc = meta[nown - 1].off + (meta[nown - 1].rl_dp & 0xff);
  for (int q = tid; q < total_acc; q += BT) acc[q] = df2{0.0f, 0.0f};
  for (int r = tid; r < nown; r += BT) bacc[r] = df2{0.0f, 0.0f};
  __syncthreads();

  const bool want_a = val != nullptr, want_b = bvec != nullptr;
  int fst = FEM_OK;  // the constant load's range status, given to every element
  const df2 fconst = (f_kind == FEM_F_CONST && f_arg) ? coef_df(__ldg(f_arg), fst) : df2{1.0f, 0.0f};
  for (int sb = 0; sb < ne; sb += a.SB) {
    const int nb = (ne - sb < a.SB) ? ne - sb : a.SB;
    for (int e = tid; e < nb; e += BT) {
      const int el = sb + e;
      const int t = st[el];
      int lv[D1];
#pragma unroll
      for (int i = 0; i < D1; ++i) lv[i] = slv[el * D1 + i];
      int st = fst;
      const df2 kt = want_k ? coef_df(sk[el], st) : df2{1.0f, 0.0f};
      LocalDF<D> L;
      if constexpr (D == 2) {
        const VtxDF<2>* const V[3] = {&xs[lv[0]], &xs[lv[1]], &xs[lv[2]]};
        const df2* sp = reinterpret_cast<const df2*>(scs);
        const df2* const Pv[3] = {sp + lv[0] * 4, sp + lv[1] * 4, sp + lv[2] * 4};
        st = worst(st, element_df2(V, Pv, kt, want_a, want_b, f_kind, fconst, f_arg, t, L));
      } else {
        const VtxDF<3>* const V[4] = {&xs[lv[0]], &xs[lv[1]], &xs[lv[2]], &xs[lv[3]]};
        st = worst(st, element_df3(V, kt, want_a, want_b, f_kind, fconst, f_arg, t, tab, L));
      }
      if (st != FEM_OK) report(err, st);
      df2* dst = ev + e * W;
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
      df2 ba = bacc[r];
      int c = m.cur;
      for (; c < m.end; ++c) {
        const uint32_t rc = srec[c - rbase];
        const int e = (int)(rc & 0x7fff);
        if (e >= sb_end) break;
        const df2* src = ev + (e - sb) * W;
        const int i = (rc >> 15) & 3;
        if (want_a) {
          acc[m.off + dp] = df_acc(acc[m.off + dp], src[pidx_rt<D>(i, i)]);
          int sh = 17;
#pragma unroll
          for (int j = 0; j < D1; ++j) {
            if (j == i) continue;
            const int pos = (rc >> sh) & 31;
            acc[m.off + pos] = df_acc(acc[m.off + pos], src[pidx_rt<D>(i, j)]);
            sh += 5;
          }
        }
        if (want_b) ba = df_acc(ba, src[U + i]);
      }
      meta[r].cur = c;
      bacc[r] = ba;
    }
    __syncthreads();
  }
  // write-out: flattened over the block's accumulator entries, coalesced along each row
  if (want_a) {
    for (int q = tid; q < total_acc; q += BT) val[gidx[q]] = df_to_double(acc[q]);
  }
  if (want_b)
    for (int r = tid; r < nown; r += BT) bvec[meta[r].R] = df_to_double(bacc[r]);
  }  // blocks
}

}  // namespace

int blocked_smem_budget(int ctas_per_sm) {
  // 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
  const int per = (228 * 1024) / ctas_per_sm - 1024 - 2048;
  return per < 220 * 1024 ? per : 220 * 1024;
}

int blocked_smem_need(const BlockPlan& B, int d, bool sinprod) {
  const int W = (d + 1) * (d + 2) / 2 + d + 1;
  return B.max_v * vtx_bytes(d) + (sinprod && d == 2 ? B.max_v * d * (int)sizeof(SC) : 0) + B.max_acc * 12 + B.V * (8 + 24) +
         B.max_rec * 4 + B.max_e * 20 + 32 * W * 8 + 256;
}

int assemble_blocked(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                     double* val, double* b, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  int rc = ensure_sincos_table();
  if (rc) return rc;
  const BlockPlan& B = P->blk;
  if (P->NT == 0 || B.nblocks == 0) {
    if (val && P->nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P->nnz, s));
    if (b && P->N > 0) FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * P->N, s));
    return FEM_OK;
  }
  const int D = P->d, D1 = D + 1, W = D1 * (D1 + 1) / 2 + D1;
  BlkArgs a;
  a.N = (int)P->N;
  a.NT = (int)P->NT;
  a.nblocks = B.nblocks;
  a.E = (int)B.E;
  a.V = B.V;
  a.order = B.order;
  a.rec_off = B.rec_off;
  a.rowp = B.rowp;
  a.rldp = B.rldp;
  a.eoff = B.eoff;
  a.voff = B.voff;
  a.elist = B.elist;
  a.lelem = B.lelem;
  a.vlist = B.vlist;
  a.rec = B.rec;
  a.row_ptr = P->row_ptr;
  // Shared memory per CTA: what the plan's launch shape (threads x CTAs per SM) leaves per CTA.
  const int budget = blocked_smem_budget(B.minb);
  a.xs_bytes = ((B.max_v * vtx_bytes(D)) + 15) / 16 * 16;
  a.sc_bytes = (D == 2 && f_kind == FEM_F_SINPROD) ? ((B.max_v * D * (int)sizeof(SC)) + 15) / 16 * 16 : 0;
  a.acc_bytes = ((B.max_acc * 8) + 15) / 16 * 16;
  a.rec_bytes = ((B.max_rec * 4) + 15) / 16 * 16;
  a.max_e = B.max_e;
  a.el_bytes = ((B.max_e * 20) + 15) / 16 * 16;  // 8 B k + 4 B id + up to 4 x 2 B local vertices
  const int fixed = a.xs_bytes + a.sc_bytes + a.acc_bytes + B.V * 8 + B.V * (int)sizeof(RowMeta) + a.rec_bytes +
                    a.el_bytes + ((B.max_acc * 4 + 15) / 16) * 16;
  const int sbmax = (budget - fixed) / (W * 8);
  if (sbmax < 32) return assemble_values(P, node, k, f_kind, f_arg, val, b, FEM_DETERMINISTIC, s);
  if (sbmax >= B.max_e) {
    a.SB = B.max_e;
  } else {  // equal sub-batches for the largest block
    const int nsb = (B.max_e + sbmax - 1) / sbmax;
    a.SB = (B.max_e + nsb - 1) / nsb;
  }
  if (a.SB < 1) a.SB = 1;
  a.ev_bytes = ((a.SB * W * 8) + 15) / 16 * 16;
  const int smem = fixed + a.ev_bytes;
  // persistent launch: one resident wave of CTAs drawing blocks from a counter reset in-stream
  int* work = nullptr;
  int grid = B.nblocks;
  if (B.persistent) {
    work = P->work_counter;
    if (!work) return set_error(FEM_ERR_STATE, "pattern has no work counter");
    FEM_CUDA(cudaMemsetAsync(work, 0, sizeof(int), s));
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    grid = nsm * B.minb < B.nblocks ? nsm * B.minb : B.nblocks;
  }
#define FEM_BLK_LAUNCH(DD, TT, MB)                                                                                \
  do {                                                                                                            \
    FEM_CUDA(cudaFuncSetAttribute(k_blocked_df<DD, TT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));   \
    FEM_LAUNCH((k_blocked_df<DD, TT, MB>), grid, TT, smem, s, a, node, k, f_kind, f_arg, val, b, err, work);        \
  } while (0)
  const int shape = B.threads * 16 + B.minb;
  if (D == 2) {
    if (shape == 256 * 16 + 4) FEM_BLK_LAUNCH(2, 256, 4);
    else if (shape == 256 * 16 + 2) FEM_BLK_LAUNCH(2, 256, 2);
    else FEM_BLK_LAUNCH(2, 512, 2);
  } else {
    if (shape == 256 * 16 + 2) FEM_BLK_LAUNCH(3, 256, 2);
    else if (shape == 256 * 16 + 1) FEM_BLK_LAUNCH(3, 256, 1);
    else FEM_BLK_LAUNCH(3, 512, 1);
  }
#undef FEM_BLK_LAUNCH
  return FEM_OK;
}

}  // namespace fem
