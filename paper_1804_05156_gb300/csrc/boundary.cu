// Boundary vertices and the Dirichlet condition (Sec. 1.2 and Sec. 3.3).
#include <cuda_runtime.h>

#include "common.cuh"

namespace fem {

namespace {

__device__ __forceinline__ void side_vertices(int d, const int32_t* __restrict__ e, int i, int (&sv)[3]) {
  if (d == 2) {
    sv[0] = e[(i + 1) % 3];
    sv[1] = e[(i + 2) % 3];
    sv[2] = -1;
  } else {
    // faces opposite vertex i, 0-based: {1,3,2}, {0,2,3}, {0,3,1}, {0,1,2}
    const int F[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};
    for (int m = 0; m < 3; ++m) sv[m] = e[F[i][m]];
  }
}

// bdflag path: every side flagged 1 marks its vertices.
__global__ void k_mark_flagged(const int32_t* __restrict__ elem, const int8_t* __restrict__ bdflag, int64_t NT, int d,
                               uint8_t* __restrict__ is_bd) {
  const int d1 = d + 1;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NT * d1; p += (int64_t)gridDim.x * blockDim.x) {
    if (bdflag[p] != 1) continue;
    const int64_t t = p / d1;
    int sv[3];
    side_vertices(d, elem + t * d1, (int)(p - t * d1), sv);
    for (int m = 0; m < d; ++m) is_bd[sv[m]] = 1;
  }
}

// whole-boundary path: side (t, i) is a boundary side when no other element contains all its
// vertices; the candidates are the elements incident to the side's first vertex.
__global__ void k_mark_unshared(const int32_t* __restrict__ elem, int64_t NT, int d, const int32_t* __restrict__ inc_ptr,
                                const int32_t* __restrict__ inc, uint8_t* __restrict__ is_bd) {
  const int d1 = d + 1;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < NT * d1; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = p / d1;
    int sv[3];
    side_vertices(d, elem + t * d1, (int)(p - t * d1), sv);
    bool shared = false;
    for (int q = inc_ptr[sv[0]]; q < inc_ptr[sv[0] + 1] && !shared; ++q) {
      const int64_t u = inc[q] / d1;
      if (u == t) continue;
      const int32_t* eu = elem + u * d1;
      bool all = true;
      for (int m = 1; m < d; ++m) {
        bool has = false;
        for (int j = 0; j < d1; ++j) has |= eu[j] == sv[m];
        all &= has;
      }
      shared = all;
    }
    if (!shared)
      for (int m = 0; m < d; ++m) is_bd[sv[m]] = 1;
  }
}

// b <- b - A u (ascending columns, no FMA), then identity rows / zero columns on the boundary.
__global__ void k_dirichlet_rows(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t N,
                                 const uint8_t* __restrict__ is_bd, const double* __restrict__ gD,
                                 double* __restrict__ val, double* __restrict__ b) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int p0 = row_ptr[r], p1 = row_ptr[r + 1];
    const bool rbd = is_bd[r] != 0;
    if (b) {
      double s = 0.0;
      for (int p = p0; p < p1; ++p) {
        const int c = col[p];
        const double u = is_bd[c] ? (gD ? gD[c] : 0.0) : 0.0;
        s = __dadd_rn(s, __dmul_rn(val[p], u));
      }
      b[r] = rbd ? (gD ? gD[r] : 0.0) : __dsub_rn(b[r], s);
    }
    for (int p = p0; p < p1; ++p) {
      const int c = col[p];
      if (rbd) val[p] = (c == r) ? 1.0 : 0.0;
      else if (is_bd[c]) val[p] = 0.0;
    }
  }
}

__global__ void k_free_flags(const uint8_t* __restrict__ is_bd, int64_t N, int32_t* __restrict__ flag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x)
    flag[r] = is_bd[r] ? 0 : 1;
}

__global__ void k_free_scatter(const uint8_t* __restrict__ is_bd, const int32_t* __restrict__ pos, int64_t N,
                               int32_t* __restrict__ free_node) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x)
    if (!is_bd[r]) free_node[pos[r]] = (int32_t)r;
}

}  // namespace

int boundary_nodes(Pattern* P, const int8_t* bdflag, uint8_t* is_bd, cudaStream_t s) {
  const int64_t total = P->NT * P->d1;
  if (bdflag) {
    if (P->N > 0) FEM_CUDA(cudaMemsetAsync(is_bd, 0, (size_t)P->N, s));
    FEM_LAUNCH(k_mark_flagged, grid_for(total, 256), 256, 0, s, P->elem, bdflag, P->NT, P->d, is_bd);
    return FEM_OK;
  }
  if (P->N == 0) return FEM_OK;
  // The whole-boundary mask depends on the topology only: found on the first call, then copied.
  if (!P->bd_whole) {
    uint8_t* m = nullptr;
    FEM_CUDA(cudaMalloc((void**)&m, (size_t)P->N));
    cudaError_t e = cudaMemsetAsync(m, 0, (size_t)P->N, s);
    if (e != cudaSuccess) {
      cudaFree(m);
      return cuda_error(e, "cudaMemsetAsync");
    }
    FEM_LAUNCH(k_mark_unshared, grid_for(total, 256), 256, 0, s, P->elem, P->NT, P->d, P->inc_ptr, P->inc, m);
    P->bd_whole = m;
  }
  FEM_CUDA(cudaMemcpyAsync(is_bd, P->bd_whole, (size_t)P->N, cudaMemcpyDeviceToDevice, s));
  return FEM_OK;
}

int apply_dirichlet(const Pattern* P, const uint8_t* is_bd, const double* gD, double* val, double* b,
                    int32_t* free_node, int64_t* n_free, cudaStream_t s) {
  const int64_t N = P->N;
  FEM_LAUNCH(k_dirichlet_rows, grid_for(N, 256), 256, 0, s, P->row_ptr, P->col_idx, N, is_bd, gD, val, b);
  if (free_node || n_free) {
    int32_t *flag = nullptr, *pos = nullptr;
    FEM_CUDA(cudaMallocAsync((void**)&flag, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), s));
    FEM_CUDA(cudaMallocAsync((void**)&pos, sizeof(int32_t) * (size_t)(N + 1), s));
    FEM_LAUNCH(k_free_flags, grid_for(N, 256), 256, 0, s, is_bd, N, flag);
    int64_t total = 0;
    int rc = exclusive_scan(flag, pos, N, n_free ? &total : nullptr, s);
    if (rc) return rc;
    if (free_node) FEM_LAUNCH(k_free_scatter, grid_for(N, 256), 256, 0, s, is_bd, pos, N, free_node);
    FEM_CUDA(cudaFreeAsync(flag, s));
    FEM_CUDA(cudaFreeAsync(pos, s));
    if (n_free) *n_free = total;
  }
  return FEM_OK;
}

}  // namespace fem
