// Device-wide LSD radix sort of 64-bit keys (8-bit digits, stable), and the unique / segment helpers
// the locality plan is built from. Used at plan time only.
#include <cuda_runtime.h>

#include "common.cuh"

namespace fem {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // keys per tile
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                         int32_t* __restrict__ counts, int64_t ntiles) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: within a tile, keys keep their order among equal digits.
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                            int64_t n, int shift, const int32_t* __restrict__ offsets,
                                                            int64_t ntiles) {
  __shared__ int32_t running[256];
  __shared__ int32_t wc[RS_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  running[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  for (int q = 0; q < RS_WARPS; ++q) wc[q][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    const uint64_t k = valid ? in[i] : 0;
    // invalid slots get digit 256 so they never match a real digit
    const int dig = valid ? (int)((k >> shift) & 255) : 256 + lane;
    const unsigned m = __match_any_sync(0xffffffffu, dig);
    const int lrank = __popc(m & lt);
    if (valid && lrank == 0) wc[w][dig] = __popc(m);
    __syncthreads();
    if (valid) {
      int pos = running[dig] + lrank;
      for (int q = 0; q < w; ++q) pos += wc[q][dig];
      out[pos] = k;
    }
    __syncthreads();
    int tot = 0;
    for (int q = 0; q < RS_WARPS; ++q) {
      tot += wc[q][threadIdx.x];
      wc[q][threadIdx.x] = 0;
    }
    running[threadIdx.x] += tot;
    __syncthreads();
  }
}

// OR and AND of all keys (to skip digits that are the same in every key)
__global__ void k_key_span(const uint64_t* __restrict__ keys, int64_t n, unsigned long long* __restrict__ orv,
                           unsigned long long* __restrict__ andv) {
  unsigned long long o = 0, a = ~0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    o |= keys[i];
    a &= keys[i];
  }
  for (int s = 16; s > 0; s >>= 1) {
    o |= __shfl_xor_sync(0xffffffffu, o, s);
    a &= __shfl_xor_sync(0xffffffffu, a, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(orv, o);
    atomicAnd(andv, a);
  }
}

__global__ void k_unique_flags(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_unique_scatter(const uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ pos,
                                 uint64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (i == 0 || keys[i] != keys[i - 1]) out[pos[i]] = keys[i];
}

// seg_off[s] = first index i with (keys[i] >> 32) >= s, for s in [0, nseg]; keys sorted.
__global__ void k_segment_starts(const uint64_t* __restrict__ keys, int64_t n, int64_t nseg, int32_t* __restrict__ seg_off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cur = (i < n) ? (int64_t)(keys[i] >> 32) : nseg;
    const int64_t prev = (i == 0) ? -1 : (int64_t)(keys[i - 1] >> 32);
    for (int64_t s = prev + 1; s <= cur && s <= nseg; ++s) seg_off[s] = (int32_t)i;
  }
}

}  // namespace

int radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, cudaStream_t s, uint64_t** result) {
  *result = keys;
  if (n <= 1) return FEM_OK;
  unsigned long long* span = nullptr;
  int32_t *counts = nullptr, *offs = nullptr;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  FEM_CUDA(cudaMallocAsync((void**)&span, 2 * sizeof(unsigned long long), s));
  FEM_CUDA(cudaMallocAsync((void**)&counts, sizeof(int32_t) * 256 * ntiles, s));
  FEM_CUDA(cudaMallocAsync((void**)&offs, sizeof(int32_t) * (256 * ntiles + 1), s));
  unsigned long long init[2] = {0ull, ~0ull};
  FEM_CUDA(cudaMemcpyAsync(span, init, sizeof(init), cudaMemcpyHostToDevice, s));
  FEM_LAUNCH(k_key_span, grid_for(n, 256, 1024), 256, 0, s, keys, n, span, span + 1);
  unsigned long long hs[2];
  FEM_CUDA(cudaMemcpyAsync(hs, span, sizeof(hs), cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  const uint64_t differ = hs[0] ^ hs[1];  // bits that are not the same in every key
  uint64_t* a = keys;
  uint64_t* b = tmp;
  for (int shift = 0; shift < 64; shift += 8) {
    if (((differ >> shift) & 255) == 0) continue;
    FEM_LAUNCH(k_radix_hist, (int)ntiles, RS_THREADS, 0, s, a, n, shift, counts, ntiles);
    int rc = exclusive_scan(counts, offs, 256 * ntiles, nullptr, s);
    if (rc) return rc;
    FEM_LAUNCH(k_radix_scatter, (int)ntiles, RS_THREADS, 0, s, a, b, n, shift, offs, ntiles);
    uint64_t* t = a;
    a = b;
    b = t;
  }
  *result = a;
  FEM_CUDA(cudaFreeAsync(span, s));
  FEM_CUDA(cudaFreeAsync(counts, s));
  FEM_CUDA(cudaFreeAsync(offs, s));
  return FEM_OK;
}

int unique_u64(const uint64_t* keys, int64_t n, uint64_t* out, int64_t* n_out, cudaStream_t s) {
  if (n == 0) {
    *n_out = 0;
    return FEM_OK;
  }
  int32_t *flag = nullptr, *pos = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&flag, sizeof(int32_t) * n, s));
  FEM_CUDA(cudaMallocAsync((void**)&pos, sizeof(int32_t) * (n + 1), s));
  FEM_LAUNCH(k_unique_flags, grid_for(n, 256), 256, 0, s, keys, n, flag);
  int rc = exclusive_scan(flag, pos, n, n_out, s);
  if (rc) return rc;
  FEM_LAUNCH(k_unique_scatter, grid_for(n, 256), 256, 0, s, keys, n, pos, out);
  FEM_CUDA(cudaFreeAsync(flag, s));
  FEM_CUDA(cudaFreeAsync(pos, s));
  return FEM_OK;
}

int segment_starts(const uint64_t* keys, int64_t n, int64_t nseg, int32_t* seg_off, cudaStream_t s) {
  if (n == 0) {
    FEM_CUDA(cudaMemsetAsync(seg_off, 0, sizeof(int32_t) * (nseg + 1), s));
    return FEM_OK;
  }
  FEM_LAUNCH(k_segment_starts, grid_for(n + 1, 256), 256, 0, s, keys, n, nseg, seg_off);
  return FEM_OK;
}

}  // namespace fem
