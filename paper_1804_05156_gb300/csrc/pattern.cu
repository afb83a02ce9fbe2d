// Pattern build: the structural CSR pattern of the P1 matrix and the per-element slot map.
//
// Sec. 2.2: `sparse(i, j, s, m, n)` sorts the (i, j) pairs and merges duplicates. Here the pairs are
// never materialised as 64-bit keys. The sort is a two-digit MSD radix sort: the first digit is the
// row (a counting sort of the (element, local vertex) incidences by vertex, i.e. one radix pass with
// radix N), the second digit is the column, ranked inside each row bucket by a warp. The ranks give
// the unique columns (col_idx) and, for every (t, i, j), the CSR position of (elem[t][i], elem[t][j])
// (the slot map), so the value kernels never search.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fem {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one int64 per thread (blockDim.x == SCAN_THREADS); returns the
// exclusive prefix and writes the block total to *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
    int64_t ti = warp_incl_scan(t);
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;
    if (lane == 31) *total = ti;
  }
  __syncthreads();
  int64_t r = warp_tot[w] + inc - v;
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q)
    if (base + q < n) s += in[base + q];
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place; sums[ntiles] = grand total.
__global__ void k_scan_sums(int64_t* sums, int64_t ntiles) {
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t c = 0; c < ntiles; c += SCAN_THREADS) {
    int64_t i = c + threadIdx.x;
    int64_t v = (i < ntiles) ? sums[i] : 0;
    int64_t ex = block_excl_scan(v, &tot);
    if (i < ntiles) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[ntiles] = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                             const int64_t* __restrict__ sums, int64_t ntiles) {
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    s += v[q];
  }
  int64_t ex = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    if (base + q < n) out[base + q] = (int32_t)ex;
    ex += v[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)sums[ntiles];
}

// ---- pattern kernels -------------------------------------------------------------------------------

// Validates vertex ids (range, no repeats within an element) and counts incidences per vertex.
__global__ void k_degree(const int32_t* __restrict__ elem, int64_t NT, int d1, int64_t N, int32_t* __restrict__ deg,
                         int* __restrict__ err) {
  const int64_t total = NT * d1;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int v = elem[p];
    if (v < 0 || v >= N) {
      report(err, FEM_ERR_INDEX);
      continue;
    }
    const int64_t t = p / d1;
    const int i = (int)(p - t * d1);
    bool dup = false;
    for (int j = 0; j < i; ++j) dup |= elem[t * d1 + j] == v;
    if (dup) report(err, FEM_ERR_INDEX);
    atomicAdd(deg + v, 1);
  }
}

__global__ void k_max(const int32_t* __restrict__ a, int64_t n, int* __restrict__ out) {
  int m = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    m = max(m, a[p]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Counting-sort scatter: incidence p = t*(d+1)+i goes to its vertex's bucket (order within a bucket
// is arbitrary here and fixed by k_sort_bucket).
__global__ void k_fill_inc(const int32_t* __restrict__ elem, int64_t total, const int32_t* __restrict__ inc_ptr,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ inc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int v = elem[p];
    const int pos = atomicAdd(cursor + v, 1);
    inc[inc_ptr[v] + pos] = (int32_t)p;
  }
}

// One warp per vertex: rank-sort its bucket ascending (entries are distinct).
__global__ void k_sort_bucket(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ in,
                              int32_t* __restrict__ out, int64_t N) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < N; r += nw) {
    const int base = inc_ptr[r], len = inc_ptr[r + 1] - base;
    for (int a = lane; a < len; a += 32) {
      const int x = in[base + a];
      int rank = 0;
      for (int b = 0; b < len; ++b) rank += in[base + b] < x;
      out[base + rank] = x;
    }
  }
}

// Candidate columns of row r: for incidence q of the row (element t, local i) and local j, the
// vertex elem[t][j]. Staged per warp in shared memory (capacity cap ints + cap flag bytes).
struct RowStage {
  int32_t* cand;
  uint8_t* first;
};

__device__ __forceinline__ int stage_row(const int32_t* __restrict__ elem, int d1, const int32_t* __restrict__ inc,
                                         int base, int len, RowStage st, int lane) {
  const int K = len * d1;
  for (int a = lane; a < K; a += 32) {
    const int q = a / d1, j = a - q * d1;
    const int p = inc[base + q];
    const int t = p / d1;
    st.cand[a] = elem[(int64_t)t * d1 + j];
  }
  __syncwarp();
  for (int a = lane; a < K; a += 32) {
    const int c = st.cand[a];
    uint8_t f = 1;
    for (int b = 0; b < a; ++b)
      if (st.cand[b] == c) {
        f = 0;
        break;
      }
    st.first[a] = f;
  }
  __syncwarp();
  return K;
}

__global__ void k_row_count(const int32_t* __restrict__ elem, int d1, const int32_t* __restrict__ inc_ptr,
                            const int32_t* __restrict__ inc, int64_t N, int cap, int32_t* __restrict__ rowcnt) {
  extern __shared__ unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  RowStage st{reinterpret_cast<int32_t*>(smem) + (size_t)w * cap,
              smem + (size_t)nwb * cap * sizeof(int32_t) + (size_t)w * cap};
  const int64_t nw = (int64_t)gridDim.x * nwb;
  for (int64_t r = (int64_t)blockIdx.x * nwb + w; r < N; r += nw) {
    const int base = inc_ptr[r], len = inc_ptr[r + 1] - base;
    const int K = stage_row(elem, d1, inc, base, len, st, lane);
    int cnt = 0;
    for (int a = lane; a < K; a += 32) cnt += st.first[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) rowcnt[r] = cnt;
    __syncwarp();
  }
}

__global__ void k_row_fill(const int32_t* __restrict__ elem, int d1, int64_t NT, const int32_t* __restrict__ inc_ptr,
                           const int32_t* __restrict__ inc, int64_t N, int cap, const int32_t* __restrict__ row_ptr,
                           int32_t* __restrict__ col_idx, int32_t* __restrict__ slot) {
  extern __shared__ unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  RowStage st{reinterpret_cast<int32_t*>(smem) + (size_t)w * cap,
              smem + (size_t)nwb * cap * sizeof(int32_t) + (size_t)w * cap};
  const int64_t nw = (int64_t)gridDim.x * nwb;
  for (int64_t r = (int64_t)blockIdx.x * nwb + w; r < N; r += nw) {
    const int base = inc_ptr[r], len = inc_ptr[r + 1] - base;
    const int K = stage_row(elem, d1, inc, base, len, st, lane);
    const int rp = row_ptr[r];
    for (int a = lane; a < K; a += 32) {
      const int c = st.cand[a];
      int rank = 0;
      for (int b = 0; b < K; ++b) rank += (st.first[b] && st.cand[b] < c);
      if (st.first[a]) col_idx[rp + rank] = c;
      const int q = a / d1, j = a - q * d1;
      const int p = inc[base + q];
      const int t = p / d1, i = p - t * d1;
      slot[(int64_t)(i * d1 + j) * NT + t] = rp + rank;
    }
    __syncwarp();
  }
}

template <typename T>
int dalloc(T** p, int64_t n, cudaStream_t s) {
  *p = nullptr;
  if (n <= 0) return FEM_OK;
  cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (size_t)n, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(FEM_ERR_OOM, "device allocation of %lld bytes failed", (long long)(sizeof(T) * n));
  }
  return FEM_OK;
}

}  // namespace

int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* total_host, cudaStream_t s) {
  if (n == 0) {
    FEM_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
    if (total_host) *total_host = 0;
    return FEM_OK;
  }
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* sums = nullptr;
  int rc = dalloc(&sums, ntiles + 1, s);
  if (rc) return rc;
  FEM_LAUNCH(k_tile_sums, (int)ntiles, SCAN_THREADS, 0, s, in, n, sums);
  FEM_LAUNCH(k_scan_sums, 1, SCAN_THREADS, 0, s, sums, ntiles);
  FEM_LAUNCH(k_scan_apply, (int)ntiles, SCAN_THREADS, 0, s, in, out, n, sums, ntiles);
  if (total_host) {
    FEM_CUDA(cudaMemcpyAsync(total_host, sums + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
  }
  FEM_CUDA(cudaFreeAsync(sums, s));
  return FEM_OK;
}

int build_pattern(Pattern* P, const int32_t* elem_in, cudaStream_t s) {
  const int d1 = P->d1;
  const int64_t N = P->N, NT = P->NT, total = NT * d1;
  int rc;
  int32_t *deg = nullptr, *cursor = nullptr, *inc_tmp = nullptr, *rowcnt = nullptr;
  int* dscal = nullptr;  // [0] validation error, [1] max degree
  auto cleanup = [&]() {
    if (deg) cudaFreeAsync(deg, s);
    if (cursor) cudaFreeAsync(cursor, s);
    if (inc_tmp) cudaFreeAsync(inc_tmp, s);
    if (rowcnt) cudaFreeAsync(rowcnt, s);
    if (dscal) cudaFreeAsync(dscal, s);
  };
#define FEM_TRY(x)  \
  do {              \
    rc = (x);       \
    if (rc) {       \
      cleanup();    \
      return rc;    \
    }               \
  } while (0)
  FEM_TRY(dalloc(&P->elem, total, s));
  FEM_TRY(dalloc(&P->row_ptr, N + 1, s));
  FEM_TRY(dalloc(&P->inc_ptr, N + 1, s));
  FEM_TRY(dalloc(&P->inc, total, s));
  FEM_TRY(dalloc(&deg, N, s));
  FEM_TRY(dalloc(&dscal, 2, s));
  if (total > 0) FEM_CUDA(cudaMemcpyAsync(P->elem, elem_in, sizeof(int32_t) * total, cudaMemcpyDeviceToDevice, s));
  if (N > 0) FEM_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * N, s));
  FEM_CUDA(cudaMemsetAsync(dscal, 0, 2 * sizeof(int), s));
  FEM_LAUNCH(k_degree, grid_for(total, 256), 256, 0, s, P->elem, NT, d1, N, deg, dscal);
  FEM_LAUNCH(k_max, grid_for(N, 256, 1024), 256, 0, s, deg, N, dscal + 1);
  int hs[2] = {0, 0};
  FEM_CUDA(cudaMemcpyAsync(hs, dscal, sizeof(hs), cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  if (hs[0] != 0) {
    cleanup();
    return set_error(hs[0], "element array names a vertex outside [0, N) or repeats a vertex");
  }
  const int maxdeg = hs[1];
  const int cap = std::max(1, maxdeg * d1);
  // warps per block for the row kernels, limited by the shared-memory staging (5 bytes per candidate)
  int nwb = 8;
  while (nwb > 1 && (size_t)nwb * cap * 5 > 200 * 1024) nwb >>= 1;
  const size_t row_smem = (size_t)nwb * cap * 5;
  if (row_smem > 200 * 1024) {
    cleanup();
    return set_error(FEM_ERR_ARG, "vertex degree %d too large for the pattern build", maxdeg);
  }
  FEM_TRY(exclusive_scan(deg, P->inc_ptr, N, nullptr, s));
  FEM_TRY(dalloc(&cursor, N, s));
  FEM_TRY(dalloc(&inc_tmp, total, s));
  if (N > 0) FEM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * N, s));
  FEM_LAUNCH(k_fill_inc, grid_for(total, 256), 256, 0, s, P->elem, total, P->inc_ptr, cursor, inc_tmp);
  FEM_LAUNCH(k_sort_bucket, grid_for(N * 32, 256), 256, 0, s, P->inc_ptr, inc_tmp, P->inc, N);
  FEM_TRY(dalloc(&rowcnt, N, s));
  if (row_smem > 48 * 1024) {
    FEM_CUDA(cudaFuncSetAttribute(k_row_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
    FEM_CUDA(cudaFuncSetAttribute(k_row_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
  }
  FEM_LAUNCH(k_row_count, grid_for(N * 32, nwb * 32), nwb * 32, row_smem, s, P->elem, d1, P->inc_ptr, P->inc, N, cap,
             rowcnt);
  int64_t nnz = 0;
  FEM_TRY(exclusive_scan(rowcnt, P->row_ptr, N, &nnz, s));
  if (nnz >= ((int64_t)1 << 31)) {
    cleanup();
    return set_error(FEM_ERR_ARG, "pattern has %lld entries, beyond int32 indexing", (long long)nnz);
  }
  P->nnz = nnz;
  FEM_TRY(dalloc(&P->col_idx, nnz, s));
  FEM_TRY(dalloc(&P->slot, total * d1, s));
  FEM_LAUNCH(k_row_fill, grid_for(N * 32, nwb * 32), nwb * 32, row_smem, s, P->elem, d1, NT, P->inc_ptr, P->inc, N,
             cap, P->row_ptr, P->col_idx, P->slot);
  cleanup();
#undef FEM_TRY
  return FEM_OK;
}

}  // namespace fem
