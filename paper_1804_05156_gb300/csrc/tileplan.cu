// Tile plan of the two-phase float-float value path (values_tiles.cu).
//
// Elements are put in a locality order (by the earliest position, in the vertex locality order, of
// any of their vertices) and cut into tiles of TE consecutive elements; each element belongs to
// exactly one tile, so nothing is computed twice. Per tile the plan stores the vertices its elements
// use (ascending id) and each element's local vertex ids. For the reduction phase it stores, per
// incidence q of the vertex-to-element lists (inc order: rows ascending, elements ascending within a
// row), the in-row positions of the element's other d columns (8 bits each, ascending local index),
// and per row the in-row position of the diagonal. The element phase writes the local entries of
// element t, row i, to packet ipos(t, i) = the index q of incidence (t, i), so every row reads its
// packets contiguously and sums them in ascending element order.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace fem {

int radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, cudaStream_t s, uint64_t** result);
int unique_u64(const uint64_t* keys, int64_t n, uint64_t* out, int64_t* n_out, cudaStream_t s);
int segment_starts(const uint64_t* keys, int64_t n, int64_t nseg, int32_t* seg_off, cudaStream_t s);

namespace {

__global__ void k_positions(const int32_t* __restrict__ order, int64_t N, int32_t* __restrict__ pos) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
    pos[order ? order[p] : p] = (int32_t)p;
}

// key = (earliest vertex position of t) << 32 | t
__global__ void k_tile_elem_keys(const int32_t* __restrict__ elem, int64_t NT, int d1, const int32_t* __restrict__ pos,
                                 uint64_t* __restrict__ keys) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t m = pos[elem[t * d1]];
    for (int i = 1; i < d1; ++i) m = min(m, pos[elem[t * d1 + i]]);
    keys[t] = ((uint64_t)(uint32_t)m << 32) | (uint64_t)t;
  }
}

// elist[j] = t of the j-th element in tile order; (tile, vertex) keys of every element-vertex
__global__ void k_tile_vert_keys(const uint64_t* __restrict__ ekeys, int64_t NT, const int32_t* __restrict__ elem,
                                 int d1, int TE, int32_t* __restrict__ elist, uint64_t* __restrict__ vkeys) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < NT; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = (int32_t)(ekeys[j] & 0xffffffffu);
    elist[j] = t;
    const uint64_t tile = (uint64_t)(j / TE);
    for (int i = 0; i < d1; ++i) vkeys[j * d1 + i] = (tile << 32) | (uint64_t)(uint32_t)elem[(int64_t)t * d1 + i];
  }
}

__global__ void k_inverse_inc(const int32_t* __restrict__ inc, int64_t total, int32_t* __restrict__ inv) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    inv[inc[q]] = (int32_t)q;
}

// local vertex ids (binary search in the tile's vertex list) and packet indices, SoA by local index i
__global__ void k_tile_local(const int32_t* __restrict__ elist, int64_t NT, const int32_t* __restrict__ elem, int d1,
                             int TE, const uint64_t* __restrict__ vk, const int32_t* __restrict__ voff,
                             const int32_t* __restrict__ inv, uint16_t* __restrict__ lelem, int32_t* __restrict__ ipos,
                             int* __restrict__ bad) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < NT; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = elist[j];
    const int tile = (int)(j / TE);
    const int v0 = voff[tile], v1 = voff[tile + 1];
    for (int i = 0; i < d1; ++i) {
      const uint32_t x = (uint32_t)elem[t * d1 + i];
      int lo = v0, hi = v1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint32_t)(vk[mid] & 0xffffffffu) < x) lo = mid + 1;
        else hi = mid;
      }
      if (lo - v0 > 65535) atomicOr(bad, 1);
      lelem[(int64_t)i * NT + j] = (uint16_t)(lo - v0);
      ipos[(int64_t)i * NT + j] = inv[t * d1 + i];
    }
  }
}

__global__ void k_low32(const uint64_t* __restrict__ vk, int64_t n, int32_t* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = (int32_t)(vk[q] & 0xffffffffu);
}

// per row: positions of the other columns of each incidence, and of the diagonal
template <typename PW>
__global__ void k_row_words(int64_t N, int d1, int64_t NT, const int32_t* __restrict__ inc_ptr,
                            const int32_t* __restrict__ inc, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ slot, PW* __restrict__ pw, uint8_t* __restrict__ rdp,
                            int* __restrict__ mx, int* __restrict__ bad) {
  for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < N; R += (int64_t)gridDim.x * blockDim.x) {
    const int rp = row_ptr[R], rl = row_ptr[R + 1] - rp;
    if (rl > 256) atomicOr(bad, 2);
    atomicMax(mx, rl);
    uint8_t dp = 0;
    for (int q = inc_ptr[R]; q < inc_ptr[R + 1]; ++q) {
      const int p = inc[q];
      const int t = p / d1, i = p - t * d1;
      uint32_t w = 0;
      int sh = 0;
      for (int j = 0; j < d1; ++j) {
        const int pos = slot[(int64_t)(i * d1 + j) * NT + t] - rp;
        if (j == i) {
          dp = (uint8_t)pos;
          continue;
        }
        w |= (uint32_t)(pos & 0xff) << sh;
        sh += 8;
      }
      pw[q] = (PW)w;
    }
    rdp[R] = dp;
  }
}

__global__ void k_tile_max_v(const int32_t* __restrict__ voff, int ntiles, int* __restrict__ mx) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ntiles; b += gridDim.x * blockDim.x)
    atomicMax(mx, voff[b + 1] - voff[b]);
}

}  // namespace

void free_tile_plan(TilePlan& T) {
  cudaFree(T.elist);
  cudaFree(T.lelem);
  cudaFree(T.voff);
  cudaFree(T.vlist);
  cudaFree(T.ipos);
  cudaFree(T.pw);
  cudaFree(T.rdp);
  cudaFree(T.pk);
  T = TilePlan();
}

int build_tile_plan(const Pattern* P, const int32_t* order, int TE, TilePlan* out, cudaStream_t s) {
  const int d1 = P->d1;
  const int64_t N = P->N, NT = P->NT, total = NT * d1;
  TilePlan T;
  T.TE = TE;
  T.ntiles = (int)((NT + TE - 1) / TE);
  if (N == 0 || NT == 0) {
    *out = T;
    return FEM_OK;
  }
  uint64_t *k1 = nullptr, *k2 = nullptr, *vk = nullptr, *sorted = nullptr;
  int32_t *pos = nullptr, *inv = nullptr;
  int* dev_int = nullptr;  // [0] bad flags, [1] longest row, [2] most tile vertices
  auto cleanup = [&]() {
    cudaFreeAsync(k1, s);
    cudaFreeAsync(k2, s);
    cudaFreeAsync(vk, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(inv, s);
    cudaFreeAsync(dev_int, s);
  };
#define TP_TRY(x)                \
  do {                           \
    cudaError_t e_ = (x);        \
    if (e_ != cudaSuccess) {     \
      cleanup();                 \
      free_tile_plan(T);         \
      return cuda_error(e_, #x); \
    }                            \
  } while (0)
#define TP_RC(x)          \
  do {                    \
    int rc_ = (x);        \
    if (rc_) {            \
      cleanup();          \
      free_tile_plan(T);  \
      return rc_;         \
    }                     \
  } while (0)
  TP_TRY(cudaMallocAsync((void**)&k1, sizeof(uint64_t) * total, s));
  TP_TRY(cudaMallocAsync((void**)&k2, sizeof(uint64_t) * total, s));
  TP_TRY(cudaMallocAsync((void**)&pos, sizeof(int32_t) * N, s));
  TP_TRY(cudaMallocAsync((void**)&dev_int, sizeof(int) * 3, s));
  TP_TRY(cudaMemsetAsync(dev_int, 0, sizeof(int) * 3, s));
  // 1. element order
  FEM_LAUNCH(k_positions, grid_for(N, 256), 256, 0, s, order, N, pos);
  FEM_LAUNCH(k_tile_elem_keys, grid_for(NT, 256), 256, 0, s, P->elem, NT, d1, pos, k1);
  TP_RC(radix_sort_u64(k1, k2, NT, s, &sorted));
  // 2. tile vertex lists
  uint64_t* vkeys = (sorted == k1) ? k2 : k1;
  TP_TRY(cudaMallocAsync((void**)&T.elist, sizeof(int32_t) * NT, s));
  FEM_LAUNCH(k_tile_vert_keys, grid_for(NT, 256), 256, 0, s, sorted, NT, P->elem, d1, TE, T.elist, vkeys);
  uint64_t* other = (vkeys == k1) ? k2 : k1;
  TP_RC(radix_sort_u64(vkeys, other, total, s, &sorted));
  TP_TRY(cudaMallocAsync((void**)&vk, sizeof(uint64_t) * total, s));
  int64_t VT = 0;
  TP_RC(unique_u64(sorted, total, vk, &VT, s));
  TP_TRY(cudaMallocAsync((void**)&T.voff, sizeof(int32_t) * (T.ntiles + 1), s));
  TP_RC(segment_starts(vk, VT, T.ntiles, T.voff, s));
  TP_TRY(cudaMallocAsync((void**)&T.vlist, sizeof(int32_t) * VT, s));
  FEM_LAUNCH(k_low32, grid_for(VT, 256), 256, 0, s, vk, VT, T.vlist);
  // 3. local vertex ids and packet indices
  TP_TRY(cudaMallocAsync((void**)&inv, sizeof(int32_t) * total, s));
  FEM_LAUNCH(k_inverse_inc, grid_for(total, 256), 256, 0, s, P->inc, total, inv);
  TP_TRY(cudaMallocAsync((void**)&T.lelem, sizeof(uint16_t) * total, s));
  TP_TRY(cudaMallocAsync((void**)&T.ipos, sizeof(int32_t) * total, s));
  FEM_LAUNCH(k_tile_local, grid_for(NT, 256), 256, 0, s, T.elist, NT, P->elem, d1, TE, vk, T.voff, inv, T.lelem,
             T.ipos, dev_int);
  // 4. per-incidence column positions and per-row diagonal positions
  TP_TRY(cudaMallocAsync((void**)&T.rdp, sizeof(uint8_t) * N, s));
  if (P->d == 2) {
    TP_TRY(cudaMallocAsync(&T.pw, sizeof(uint16_t) * total, s));
    FEM_LAUNCH(k_row_words<uint16_t>, grid_for(N, 256), 256, 0, s, N, d1, NT, P->inc_ptr, P->inc, P->row_ptr, P->slot,
               (uint16_t*)T.pw, T.rdp, dev_int + 1, dev_int);
  } else {
    TP_TRY(cudaMallocAsync(&T.pw, sizeof(uint32_t) * total, s));
    FEM_LAUNCH(k_row_words<uint32_t>, grid_for(N, 256), 256, 0, s, N, d1, NT, P->inc_ptr, P->inc, P->row_ptr, P->slot,
               (uint32_t*)T.pw, T.rdp, dev_int + 1, dev_int);
  }
  FEM_LAUNCH(k_tile_max_v, grid_for(T.ntiles, 256), 256, 0, s, T.voff, T.ntiles, dev_int + 2);
  // 5. packets: four float pairs (32 bytes) per incidence
  TP_TRY(cudaMallocAsync((void**)&T.pk, sizeof(float4) * 2 * total, s));
  int hs[3] = {0, 0, 0};
  TP_TRY(cudaMemcpyAsync(hs, dev_int, sizeof(hs), cudaMemcpyDeviceToHost, s));
  TP_TRY(cudaStreamSynchronize(s));
  T.VT = VT;
  T.max_row = hs[1];
  T.max_v = hs[2];
  T.ok = (hs[0] == 0);
  cleanup();
#undef TP_TRY
#undef TP_RC
  *out = T;
  return FEM_OK;
}

}  // namespace fem
