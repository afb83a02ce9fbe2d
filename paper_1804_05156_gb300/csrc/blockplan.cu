// Locality plan for the owner-computes value kernel.
//
// The vertices (rows) are ordered by a locality key (a Morton code of the coordinates when the caller
// gives them, else the vertex id) and cut into blocks of V consecutive vertices. One CTA owns one
// block: it computes every element that touches one of its rows (elements on a block boundary are
// computed by each block they touch) and sums the rows' entries on chip in a fixed order, so every
// CSR entry is written once, by its owner, with no atomics.
//
// Per block the plan stores: its element list (ascending caller element id), the vertices those
// elements use (ascending id; local vertex ids are positions in it), each element's local vertex ids,
// and for every owned row its incidences in ascending element order, packed as
//   e (15 bits, position in the block's element list) | i << 15 (2 bits, local vertex of the row)
//   | in-row position of column elem[t][j] for the d vertices j != i, ascending j, 5 bits each.
// Limits of the packed form: <= 32768 elements per block and <= 32 entries per row; a mesh outside
// them keeps the two-pass path.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace fem {

int radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, cudaStream_t s, uint64_t** result);
int unique_u64(const uint64_t* keys, int64_t n, uint64_t* out, int64_t* n_out, cudaStream_t s);
int segment_starts(const uint64_t* keys, int64_t n, int64_t nseg, int32_t* seg_off, cudaStream_t s);

namespace {

__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered(unsigned long long u) {
  return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

// Bounding box of the coordinates: per-thread, then per-warp min/max, then one atomic per warp and
// coordinate on the order-preserving bit pattern.
__global__ void k_bbox(const double* __restrict__ node, int64_t N, int d, unsigned long long* __restrict__ lo,
                       unsigned long long* __restrict__ hi) {
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    for (int m = 0; m < d; ++m) {
      const unsigned long long u = ordered_bits(node[v * d + m]);
      mn[m] = u < mn[m] ? u : mn[m];
      mx[m] = u > mx[m] ? u : mx[m];
    }
  for (int m = 0; m < d; ++m) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn[m], o), b = __shfl_xor_sync(0xffffffffu, mx[m], o);
      mn[m] = a < mn[m] ? a : mn[m];
      mx[m] = b > mx[m] ? b : mx[m];
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(lo + m, mn[m]);
      atomicMax(hi + m, mx[m]);
    }
  }
}

__device__ __forceinline__ uint32_t spread2(uint32_t x) {  // 12 bits -> every other bit
  x &= 0xfff;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // 8 bits -> every third bit
  x &= 0xff;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// key = group (8 bits) << 56 | morton (24 bits) << 32 | vertex id
__global__ void k_vertex_keys(const double* __restrict__ node, const int32_t* __restrict__ group, int64_t N, int d,
                              const unsigned long long* __restrict__ lo, const unsigned long long* __restrict__ hi,
                              uint64_t* __restrict__ keys) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    uint32_t code = 0;
    if (node) {
      const int bits = (d == 2) ? 12 : 8;
      const double cells = (double)(1 << bits);
      uint32_t q[3] = {0, 0, 0};
      for (int m = 0; m < d; ++m) {
        const double a = from_ordered(lo[m]), b = from_ordered(hi[m]);
        double u = (b > a) ? (node[v * d + m] - a) / (b - a) : 0.0;
        u = fmin(fmax(u * cells, 0.0), cells - 1.0);
        q[m] = (uint32_t)u;
      }
      code = (d == 2) ? (spread2(q[0]) | (spread2(q[1]) << 1))
                      : (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2));
    }
    const uint64_t g = group ? (uint64_t)(group[v] & 255) : 0;
    keys[v] = (g << 56) | ((uint64_t)(code & 0xffffff) << 32) | (uint64_t)v;
  }
}

__global__ void k_order_from_keys(const uint64_t* __restrict__ keys, int64_t N, int V, int32_t* __restrict__ order,
                                  int32_t* __restrict__ vblock) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)(keys[p] & 0xffffffffu);
    order[p] = v;
    vblock[v] = (int32_t)(p / V);
  }
}

// (block of elem[t][i], t) for every incidence
__global__ void k_elem_keys(const int32_t* __restrict__ elem, int64_t total, int d1, const int32_t* __restrict__ vblock,
                            uint64_t* __restrict__ keys) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x)
    keys[p] = ((uint64_t)vblock[elem[p]] << 32) | (uint64_t)(p / d1);
}

// (block, elem[t][i]) for every listed element and i
__global__ void k_vert_keys(const uint64_t* __restrict__ ekeys, int64_t E, const int32_t* __restrict__ elem, int d1,
                            uint64_t* __restrict__ keys) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E * d1; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / d1;
    const int i = (int)(q - e * d1);
    const uint64_t k = ekeys[e];
    const int64_t t = (int64_t)(k & 0xffffffffu);
    keys[q] = (k & 0xffffffff00000000ull) | (uint64_t)(uint32_t)elem[t * d1 + i];
  }
}

__device__ __forceinline__ int lower_bound_low32(const uint64_t* __restrict__ keys, int lo, int hi, uint32_t x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((uint32_t)(keys[mid] & 0xffffffffu) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_split_lists(const uint64_t* __restrict__ ekeys, int64_t E, const uint64_t* __restrict__ vkeys,
                              int64_t VT, const int32_t* __restrict__ elem, int d1, const int32_t* __restrict__ voff,
                              int32_t* __restrict__ elist, uint16_t* __restrict__ lelem, int32_t* __restrict__ vlist,
                              int* __restrict__ bad) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ekeys[q];
    const int b = (int)(k >> 32);
    const int32_t t = (int32_t)(k & 0xffffffffu);
    elist[q] = t;
    const int lo = voff[b], hi = voff[b + 1];
    for (int i = 0; i < d1; ++i) {
      const int pos = lower_bound_low32(vkeys, lo, hi, (uint32_t)elem[(int64_t)t * d1 + i]);
      const int l = pos - lo;
      if (l > 65535) atomicOr(bad, 1);
      lelem[(int64_t)i * E + q] = (uint16_t)l;
    }
  }
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < VT; q += (int64_t)gridDim.x * blockDim.x)
    vlist[q] = (int32_t)(vkeys[q] & 0xffffffffu);
}

__global__ void k_sorted_degrees(const int32_t* __restrict__ order, const int32_t* __restrict__ inc_ptr, int64_t N,
                                 int32_t* __restrict__ deg) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int v = order[p];
    deg[p] = inc_ptr[v + 1] - inc_ptr[v];
  }
}

// per owned row (position p in the locality order): local index, diagonal position, records
__global__ void k_records(const int32_t* __restrict__ order, int64_t N, int V, int d1, int64_t NT,
                          const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc,
                          const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ slot,
                          const int32_t* __restrict__ eoff, const int32_t* __restrict__ elist,
                          const int32_t* __restrict__ voff, const int32_t* __restrict__ vlist,
                          const int32_t* __restrict__ rec_off, uint16_t* __restrict__ own_local,
                          int32_t* __restrict__ rowp, uint16_t* __restrict__ rldp, uint32_t* __restrict__ rec,
                          int* __restrict__ bad) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int R = order[p];
    const int b = (int)(p / V);
    // local index of R in the block's vertex list
    int lo = voff[b], hi = voff[b + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (vlist[mid] < R) lo = mid + 1;
      else hi = mid;
    }
    own_local[p] = (uint16_t)(lo - voff[b]);
    const int rp = row_ptr[R];
    if (row_ptr[R + 1] - rp > 32) atomicOr(bad, 2);
    const int e0 = eoff[b], e1 = eoff[b + 1];
    if (e1 - e0 > 32768) atomicOr(bad, 4);
    int w = rec_off[p];
    uint8_t dp = 0;
    for (int q = inc_ptr[R]; q < inc_ptr[R + 1]; ++q, ++w) {
      const int pp = inc[q];
      const int t = pp / d1, i = pp - t * d1;
      int a = e0, c = e1;
      while (a < c) {
        const int mid = (a + c) >> 1;
        if (elist[mid] < t) a = mid + 1;
        else c = mid;
      }
      uint32_t r = (uint32_t)((a - e0) & 0x7fff) | ((uint32_t)i << 15);
      int sh = 17;
      for (int j = 0; j < d1; ++j) {
        const int pos = slot[(int64_t)(i * d1 + j) * NT + t] - rp;
        if (j == i) {
          dp = (uint8_t)pos;
          continue;
        }
        r |= (uint32_t)(pos & 31) << sh;
        sh += 5;
      }
      rec[w] = r;
    }
    rowp[p] = rp;
    rldp[p] = (uint16_t)(((row_ptr[R + 1] - rp) & 0xff) | ((int)dp << 8));
  }
}

__global__ void k_block_maxima(const int32_t* __restrict__ eoff, const int32_t* __restrict__ voff,
                               const int32_t* __restrict__ order, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ rec_off, int64_t N, int V, int nblocks,
                               int* __restrict__ mx) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblocks; b += gridDim.x * blockDim.x) {
    atomicMax(mx + 0, eoff[b + 1] - eoff[b]);
    atomicMax(mx + 1, voff[b + 1] - voff[b]);
    int s = 0;
    const int64_t p1 = ((int64_t)(b + 1) * V < N) ? (int64_t)(b + 1) * V : N;
    for (int64_t p = (int64_t)b * V; p < p1; ++p) s += row_ptr[order[p] + 1] - row_ptr[order[p]];
    atomicMax(mx + 2, s);
    atomicMax(mx + 3, rec_off[p1] - rec_off[(int64_t)b * V]);
  }
}

}  // namespace

void free_block_plan(BlockPlan& B) {
  cudaFree(B.order);
  cudaFree(B.rec_off);
  cudaFree(B.own_local);
  cudaFree(B.rowp);
  cudaFree(B.rldp);
  cudaFree(B.eoff);
  cudaFree(B.voff);
  cudaFree(B.elist);
  cudaFree(B.lelem);
  cudaFree(B.vlist);
  cudaFree(B.rec);
  B = BlockPlan();
}

int build_block_plan(const Pattern* P, const double* node_hint, const int32_t* group, int V, BlockPlan* out,
                     cudaStream_t s) {
  const int d = P->d, d1 = P->d1;
  const int64_t N = P->N, NT = P->NT, total = NT * d1;
  BlockPlan B;
  B.V = V;
  B.nblocks = (int)((N + V - 1) / V);
  if (N == 0 || NT == 0) {
    *out = B;
    return FEM_OK;
  }
  int rc = FEM_OK;
  uint64_t *k1 = nullptr, *k2 = nullptr, *sorted = nullptr, *ek = nullptr, *vk = nullptr;
  int32_t *vblock = nullptr, *deg = nullptr;
  int* dev_int = nullptr;  // [0] bad flag, [1..4] maxima
  unsigned long long* bbox = nullptr;
  auto cleanup = [&]() {
    cudaFreeAsync(k1, s);
    cudaFreeAsync(k2, s);
    cudaFreeAsync(ek, s);
    cudaFreeAsync(vk, s);
    cudaFreeAsync(vblock, s);
    cudaFreeAsync(deg, s);
    cudaFreeAsync(dev_int, s);
    cudaFreeAsync(bbox, s);
  };
#define BP_TRY(x)              \
  do {                         \
    cudaError_t e_ = (x);      \
    if (e_ != cudaSuccess) {   \
      cleanup();               \
      free_block_plan(B);      \
      return cuda_error(e_, #x); \
    }                          \
  } while (0)
#define BP_RC(x)             \
  do {                       \
    rc = (x);                \
    if (rc) {                \
      cleanup();             \
      free_block_plan(B);    \
      return rc;             \
    }                        \
  } while (0)
  const int64_t big = std::max<int64_t>(N, total);
  BP_TRY(cudaMallocAsync((void**)&k1, sizeof(uint64_t) * big, s));
  BP_TRY(cudaMallocAsync((void**)&k2, sizeof(uint64_t) * big, s));
  BP_TRY(cudaMallocAsync((void**)&vblock, sizeof(int32_t) * N, s));
  BP_TRY(cudaMallocAsync((void**)&dev_int, sizeof(int) * 5, s));
  BP_TRY(cudaMallocAsync((void**)&bbox, sizeof(unsigned long long) * 6, s));
  BP_TRY(cudaMallocAsync((void**)&B.order, sizeof(int32_t) * N, s));
  BP_TRY(cudaMemsetAsync(dev_int, 0, sizeof(int) * 5, s));
  // 1. locality order of the vertices
  if (node_hint) {
    unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
    BP_TRY(cudaMemcpyAsync(bbox, init, sizeof(init), cudaMemcpyHostToDevice, s));
    FEM_LAUNCH(k_bbox, grid_for(N, 256, 1024), 256, 0, s, node_hint, N, d, bbox, bbox + 3);
  }
  FEM_LAUNCH(k_vertex_keys, grid_for(N, 256), 256, 0, s, node_hint, group, N, d, bbox, bbox + 3, k1);
  BP_RC(radix_sort_u64(k1, k2, N, s, &sorted));
  FEM_LAUNCH(k_order_from_keys, grid_for(N, 256), 256, 0, s, sorted, N, V, B.order, vblock);
  // 2. element lists: unique (block, t) over all incidences
  FEM_LAUNCH(k_elem_keys, grid_for(total, 256), 256, 0, s, P->elem, total, d1, vblock, k1);
  BP_RC(radix_sort_u64(k1, k2, total, s, &sorted));
  int64_t E = 0;
  BP_TRY(cudaMallocAsync((void**)&ek, sizeof(uint64_t) * total, s));
  BP_RC(unique_u64(sorted, total, ek, &E, s));
  BP_TRY(cudaMallocAsync((void**)&B.eoff, sizeof(int32_t) * (B.nblocks + 1), s));
  BP_RC(segment_starts(ek, E, B.nblocks, B.eoff, s));
  // 3. vertex lists: unique (block, vertex) over the listed elements' vertices
  const int64_t nvk = E * d1;
  uint64_t *k3 = nullptr, *k4 = nullptr;
  BP_TRY(cudaMallocAsync((void**)&k3, sizeof(uint64_t) * nvk, s));
  BP_TRY(cudaMallocAsync((void**)&k4, sizeof(uint64_t) * nvk, s));
  FEM_LAUNCH(k_vert_keys, grid_for(nvk, 256), 256, 0, s, ek, E, P->elem, d1, k3);
  BP_RC(radix_sort_u64(k3, k4, nvk, s, &sorted));
  int64_t VT = 0;
  BP_TRY(cudaMallocAsync((void**)&vk, sizeof(uint64_t) * nvk, s));
  BP_RC(unique_u64(sorted, nvk, vk, &VT, s));
  cudaFreeAsync(k3, s);
  cudaFreeAsync(k4, s);
  BP_TRY(cudaMallocAsync((void**)&B.voff, sizeof(int32_t) * (B.nblocks + 1), s));
  BP_RC(segment_starts(vk, VT, B.nblocks, B.voff, s));
  // 4. element list, local vertex ids, vertex list
  BP_TRY(cudaMallocAsync((void**)&B.elist, sizeof(int32_t) * E, s));
  BP_TRY(cudaMallocAsync((void**)&B.lelem, sizeof(uint16_t) * E * d1, s));
  BP_TRY(cudaMallocAsync((void**)&B.vlist, sizeof(int32_t) * VT, s));
  FEM_LAUNCH(k_split_lists, grid_for(std::max(E, VT), 256), 256, 0, s, ek, E, vk, VT, P->elem, d1, B.voff, B.elist,
             B.lelem, B.vlist, dev_int);
  // 5. records of the owned rows
  BP_TRY(cudaMallocAsync((void**)&deg, sizeof(int32_t) * N, s));
  BP_TRY(cudaMallocAsync((void**)&B.rec_off, sizeof(int32_t) * (N + 1), s));
  FEM_LAUNCH(k_sorted_degrees, grid_for(N, 256), 256, 0, s, B.order, P->inc_ptr, N, deg);
  BP_RC(exclusive_scan(deg, B.rec_off, N, nullptr, s));
  BP_TRY(cudaMallocAsync((void**)&B.own_local, sizeof(uint16_t) * N, s));
  BP_TRY(cudaMallocAsync((void**)&B.rowp, sizeof(int32_t) * N, s));
  BP_TRY(cudaMallocAsync((void**)&B.rldp, sizeof(uint16_t) * N, s));
  BP_TRY(cudaMallocAsync((void**)&B.rec, sizeof(uint32_t) * total, s));
  FEM_LAUNCH(k_records, grid_for(N, 256), 256, 0, s, B.order, N, V, d1, NT, P->inc_ptr, P->inc, P->row_ptr, P->slot,
             B.eoff, B.elist, B.voff, B.vlist, B.rec_off, B.own_local, B.rowp, B.rldp, B.rec, dev_int);
  FEM_LAUNCH(k_block_maxima, grid_for(B.nblocks, 256), 256, 0, s, B.eoff, B.voff, B.order, P->row_ptr, B.rec_off, N,
             V, B.nblocks, dev_int + 1);
  int hs[5] = {0, 0, 0, 0, 0};
  BP_TRY(cudaMemcpyAsync(hs, dev_int, sizeof(hs), cudaMemcpyDeviceToHost, s));
  BP_TRY(cudaStreamSynchronize(s));
  B.E = E;
  B.VT = VT;
  B.max_e = hs[1];
  B.max_v = hs[2];
  B.max_acc = hs[3];
  B.max_rec = hs[4];
  B.ok = (hs[0] == 0);
  cleanup();
#undef BP_TRY
#undef BP_RC
  *out = B;
  return FEM_OK;
}

// Launch shapes (threads per CTA, CTAs per SM) the value kernel is compiled for.
static const int kShapes2[][2] = {{512, 2}, {256, 4}, {256, 2}};
static const int kShapes3[][2] = {{512, 1}, {256, 2}, {256, 1}};

int rebuild_block_plan(Pattern* P, const double* node_hint, const int32_t* group, cudaStream_t s) {
  free_block_plan(P->blk);
  free_tile_plan(P->tile);
  P->use_tiles = false;
  const int d = P->d;
  const bool sinprod = (d == 2);  // the tuning workload: the 2-D sine-product load, 3-D constant load
  // Without coordinates there is nothing to time: take the first feasible block size, default shape.
  if (!node_hint) {
    for (int V = (d == 2) ? 256 : 512; V >= 32; V >>= 1) {
      BlockPlan B;
      int rc = build_block_plan(P, nullptr, group, V, &B, s);
      if (rc) return rc;
      B.threads = (d == 2) ? 512 : 512;
      B.minb = (d == 2) ? 2 : 1;
      while (B.minb > 1 && blocked_smem_need(B, d, sinprod) > blocked_smem_budget(B.minb)) B.minb >>= 1;
      if (B.ok && blocked_smem_need(B, d, sinprod) <= blocked_smem_budget(B.minb)) {
        P->blk = B;
        break;
      }
      free_block_plan(B);
    }
    // the two-phase path on the same vertex order (identity order if no blocked plan was feasible)
    TilePlan T;
    int rc = build_tile_plan(P, P->blk.order, 256, &T, s);
    if (rc) return rc;
    if (T.ok) {
      P->tile = T;
      P->use_tiles = true;
    } else {
      free_tile_plan(T);
    }
    enforce_one_launch(P);
    return FEM_OK;
  }
  // With coordinates: time every feasible (block size, launch shape) on the device, keep the fastest.
  // The timing runs may report degenerate elements (the coordinates are only an ordering hint), so
  // the device error word is saved first and restored afterwards.
  int* errw = device_error_word();
  if (!errw) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  int saved_err = 0;
  FEM_CUDA(cudaMemcpyAsync(&saved_err, errw, sizeof(int), cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  double *val = nullptr, *bb = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&val, sizeof(double) * (P->nnz > 0 ? P->nnz : 1), s));
  FEM_CUDA(cudaMallocAsync((void**)&bb, sizeof(double) * (P->N > 0 ? P->N : 1), s));
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  BlockPlan best;
  float best_ms = 1e30f;
  const int Vs[] = {512, 256, 128};
  const int (*shapes)[2] = (d == 2) ? kShapes2 : kShapes3;
  const int nshapes = 3;
  int rc = FEM_OK;
  for (int vi = 0; vi < 3 && rc == FEM_OK; ++vi) {
    BlockPlan B;
    rc = build_block_plan(P, node_hint, group, Vs[vi], &B, s);
    if (rc) break;
    bool kept = false;
    for (int si = P->one_launch ? nshapes : 0; si < 2 * nshapes && B.ok; ++si) {
      B.threads = shapes[si % nshapes][0];
      B.minb = shapes[si % nshapes][1];
      B.persistent = si >= nshapes;
      if (blocked_smem_need(B, d, sinprod) > blocked_smem_budget(B.minb)) continue;
      Pattern Q = *P;  // same pattern, candidate plan
      Q.blk = B;
      const int fk = sinprod ? FEM_F_SINPROD : FEM_F_CONST;
      rc = assemble_blocked(&Q, node_hint, nullptr, fk, nullptr, val, bb, s);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && rc == FEM_OK; ++r) rc = assemble_blocked(&Q, node_hint, nullptr, fk, nullptr, val, bb, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "tuning run");
      if (rc) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= 3.0f;
      if (ms < best_ms) {
        if (best.order && !kept) free_block_plan(best);
        best_ms = ms;
        best = B;
        best.tuned_ms = ms;
        kept = true;
      }
    }
    if (!kept) free_block_plan(B);
  }
  // The two-phase path on the chosen vertex order: time each tile size in both launch forms (two
  // launches, or one fused cooperative launch), keep the fastest if it beats the blocked plan.
  TilePlan bestT;
  for (int ti = 0; ti < 2 && rc == FEM_OK; ++ti) {
    const int TEs[] = {256, 128};
    TilePlan T;
    rc = build_tile_plan(P, best.order, TEs[ti], &T, s);
    if (rc) break;
    if (!T.ok) {
      free_tile_plan(T);
      continue;
    }
    float t_best = 1e30f;
    bool f_best = false;
    for (int fu = P->one_launch ? 1 : 0; fu < 2 && rc == FEM_OK; ++fu) {
      T.fused = fu == 1;
      if (T.fused && tile_fused_smem(T, d) == 0) continue;
      Pattern Q = *P;
      Q.tile = T;
      const int fk = sinprod ? FEM_F_SINPROD : FEM_F_CONST;
      rc = assemble_tiles(&Q, node_hint, nullptr, fk, nullptr, val, bb, s);  // warm-up
      if (rc == FEM_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && rc == FEM_OK; ++r) rc = assemble_tiles(&Q, node_hint, nullptr, fk, nullptr, val, bb, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_error(cudaGetLastError(), "tuning run");
      }
      if (rc == FEM_OK) {
        float ms = 1e30f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.0f;
        if (ms < t_best) {
          t_best = ms;
          f_best = T.fused;
        }
      }
    }
    T.fused = f_best;
    if (rc == FEM_OK && t_best < bestT.tuned_ms) {
      free_tile_plan(bestT);
      bestT = T;
      bestT.tuned_ms = t_best;
    } else {
      free_tile_plan(T);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(val, s);
  cudaFreeAsync(bb, s);
  cudaMemcpyAsync(errw, &saved_err, sizeof(int), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  if (rc) {
    if (best.order) free_block_plan(best);
    free_tile_plan(bestT);
    return rc;
  }
  if (best.order) P->blk = best;
  if (bestT.ok && bestT.tuned_ms < 1e29f && (!best.order || bestT.tuned_ms < best_ms)) {
    P->tile = bestT;
    P->use_tiles = true;
  } else {
    free_tile_plan(bestT);
  }
  enforce_one_launch(P);
  return FEM_OK;
}

void enforce_one_launch(Pattern* P) {
  if (!P->one_launch) return;
  if (P->use_tiles && !P->tile.fused) {
    if (tile_fused_smem(P->tile, P->d) != 0) {
      P->tile.fused = true;
      return;
    }
    P->use_tiles = false;
  }
  if (!P->use_tiles && P->blk.ok) P->blk.persistent = true;
}

}  // namespace fem
