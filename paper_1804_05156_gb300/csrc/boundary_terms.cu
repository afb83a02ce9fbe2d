// Neumann and Robin sides ("Boundary conditions" and Sec. 3.3), side quadrature points, and the
// pure-Neumann fixes (b - mean(b); the zero-average shift of a solution).
//
// A side is the face of element t opposite local vertex j; bdflag[t][j] = 2 marks it Neumann, 3 Robin
// (du/dn + alpha u = g). Its vertices are the element's other d vertices in ascending local index and its
// measure |s| is the edge length (2-D) or the triangle area (3-D). Load: |s| g / d to each of its
// vertices (the one-point side rule of the paper's Neumann code, at the midpoint / centroid). Robin
// matrix: alpha |s| (1 + delta_ab) / (d (d+1)) to the CSR entry of each pair (a, b) of its vertices.
// One thread per row walks the row's incidences (ascending element) and, for each, the element's
// flagged sides through the row's vertex (ascending j): every b and val entry is updated by one thread
// only, in a fixed order, with uncontracted FP64 operations. This boundary work is small next to the
// assembly, so it stays in FP64.
#include <cuda_runtime.h>

#include "common.cuh"

namespace fem {

namespace {

template <int D>
__device__ __forceinline__ double side_measure(const double* __restrict__ node, const int32_t* __restrict__ e, int j) {
  int32_t v[3] = {0, 0, 0};
  int c = 0;
#pragma unroll
  for (int k = 0; k <= D; ++k)
    if (k != j) v[c++] = e[k];
  if constexpr (D == 2) {
    const double dx = __dsub_rn(__ldg(node + 2 * (size_t)v[1]), __ldg(node + 2 * (size_t)v[0]));
    const double dy = __dsub_rn(__ldg(node + 2 * (size_t)v[1] + 1), __ldg(node + 2 * (size_t)v[0] + 1));
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  } else {
    double u[3], w[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      u[m] = __dsub_rn(__ldg(node + 3 * (size_t)v[1] + m), __ldg(node + 3 * (size_t)v[0] + m));
      w[m] = __dsub_rn(__ldg(node + 3 * (size_t)v[2] + m), __ldg(node + 3 * (size_t)v[0] + m));
    }
    const double x0 = __dsub_rn(__dmul_rn(u[1], w[2]), __dmul_rn(u[2], w[1]));
    const double x1 = __dsub_rn(__dmul_rn(u[2], w[0]), __dmul_rn(u[0], w[2]));
    const double x2 = __dsub_rn(__dmul_rn(u[0], w[1]), __dmul_rn(u[1], w[0]));
    return __dmul_rn(__dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x0, x0), __dmul_rn(x1, x1)), __dmul_rn(x2, x2))), 0.5);
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_boundary_terms(int64_t N, int64_t NT, const int32_t* __restrict__ elem,
                                                        const int32_t* __restrict__ inc_ptr,
                                                        const int32_t* __restrict__ inc,
                                                        const int32_t* __restrict__ slot,
                                                        const double* __restrict__ node,
                                                        const int8_t* __restrict__ bdflag,
                                                        const double* __restrict__ g_side, double g_const,
                                                        double alpha, double* __restrict__ val,
                                                        double* __restrict__ b) {
  constexpr int D1 = D + 1;
  for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < N; R += (int64_t)gridDim.x * blockDim.x) {
    const int q1 = __ldg(inc_ptr + R + 1);
    bool any = false;
    double bR = 0.0;
    for (int q = __ldg(inc_ptr + R); q < q1; ++q) {
      const int p = __ldg(inc + q);
      const int64_t t = p / D1;
      const int i = p - (int)t * D1;
      int fl[D1];
#pragma unroll
      for (int j = 0; j < D1; ++j) fl[j] = __ldg(bdflag + t * D1 + j);
#pragma unroll
      for (int j = 0; j < D1; ++j) {
        if (j == i || (fl[j] != 2 && fl[j] != 3)) continue;
        int32_t e[D1];
#pragma unroll
        for (int k = 0; k < D1; ++k) e[k] = __ldg(elem + t * D1 + k);
        const double m = side_measure<D>(node, e, j);
        if (b) {
          if (!any) bR = b[R];
          any = true;
          const double g = g_side ? __ldg(g_side + t * D1 + j) : g_const;
          bR = __dadd_rn(bR, __ddiv_rn(__dmul_rn(m, g), (double)D));
        }
        if (fl[j] == 3 && val) {
#pragma unroll
          for (int c = 0; c < D1; ++c) {
            if (c == j) continue;
            const int pos = __ldg(slot + (int64_t)(i * D1 + c) * NT + t);
            const double wgt = (c == i) ? 2.0 : 1.0;
            val[pos] = __dadd_rn(val[pos], __ddiv_rn(__dmul_rn(__dmul_rn(alpha, m), wgt), (double)(D * D1)));
          }
        }
      }
    }
    if (any) b[R] = bR;
  }
}

// quadrature point of side (t, j): the mean of its vertices, summed in ascending local index
template <int D>
__global__ void k_side_points(int64_t NT, const int32_t* __restrict__ elem, const double* __restrict__ node,
                              double* __restrict__ pts) {
  constexpr int D1 = D + 1;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < NT * D1; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = s / D1;
    const int j = (int)(s - t * D1);
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < D1; ++k)
        if (k != j) acc = __dadd_rn(acc, __ldg(node + (size_t)__ldg(elem + t * D1 + k) * D + m));
      pts[s * D + m] = __ddiv_rn(acc, (double)D);
    }
  }
}

// ---- deterministic sums: a fixed grid of kRedBlocks blocks, each a fixed tree; then one block ----------

constexpr int kRedBlocks = 1024, kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// partial[blk] = sum of x over block blk's contiguous chunk (each thread sums a strided slice)
__global__ void __launch_bounds__(kRedThreads) k_partial_sum(const double* __restrict__ x, int64_t n,
                                                             double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  const int64_t chunk = (n + kRedBlocks - 1) / kRedBlocks;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) s = __dadd_rn(s, __ldg(x + i));
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// per element: (sum of u over its vertices) * d! |tau| and d! |tau| (2-D |2 area|, 3-D 6 x signed volume);
// the factors 1/(d+1) and 1/d! are applied once to the totals
template <int D>
__global__ void __launch_bounds__(kRedThreads) k_partial_average(int64_t NT, const int32_t* __restrict__ elem,
                                                                 const double* __restrict__ node,
                                                                 const double* __restrict__ u,
                                                                 double* __restrict__ partial) {
  constexpr int D1 = D + 1;
  __shared__ double sh[kRedThreads];
  const int64_t chunk = (NT + kRedBlocks - 1) / kRedBlocks;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < NT ? lo + chunk : NT;
  double num = 0.0, den = 0.0;
  for (int64_t t = lo + threadIdx.x; t < hi; t += kRedThreads) {
    int32_t e[D1];
#pragma unroll
    for (int k = 0; k < D1; ++k) e[k] = __ldg(elem + t * D1 + k);
    double x[D1][D];
#pragma unroll
    for (int k = 0; k < D1; ++k)
#pragma unroll
      for (int m = 0; m < D; ++m) x[k][m] = __ldg(node + (size_t)e[k] * D + m);
    double meas;
    if constexpr (D == 2) {
      const double a2 = __dsub_rn(__dmul_rn(__dsub_rn(x[1][0], x[0][0]), __dsub_rn(x[2][1], x[0][1])),
                                  __dmul_rn(__dsub_rn(x[1][1], x[0][1]), __dsub_rn(x[2][0], x[0][0])));
      meas = fabs(a2);
    } else {
      double a[3], bb[3], c[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        a[m] = __dsub_rn(x[1][m], x[0][m]);
        bb[m] = __dsub_rn(x[2][m], x[0][m]);
        c[m] = __dsub_rn(x[3][m], x[0][m]);
      }
      const double v = __dadd_rn(__dadd_rn(__dmul_rn(__dsub_rn(__dmul_rn(a[1], bb[2]), __dmul_rn(a[2], bb[1])), c[0]),
                                           __dmul_rn(__dsub_rn(__dmul_rn(a[2], bb[0]), __dmul_rn(a[0], bb[2])), c[1])),
                                 __dmul_rn(__dsub_rn(__dmul_rn(a[0], bb[1]), __dmul_rn(a[1], bb[0])), c[2]));
      meas = v;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D1; ++k) s = __dadd_rn(s, __ldg(u + e[k]));
    num = __dadd_rn(num, __dmul_rn(s, meas));
    den = __dadd_rn(den, meas);
  }
  const double tn = block_sum(num, sh) / (double)D1;
  const double td = block_sum(den, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = tn;
    partial[kRedBlocks + blockIdx.x] = td;
  }
}

// out[0] = (sum of partial[0..kRedBlocks)) / divisor  (or / sum of partial[kRedBlocks..2 kRedBlocks) when
// divisor <= 0)
__global__ void __launch_bounds__(kRedThreads) k_finish(const double* __restrict__ partial, double divisor,
                                                        double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double s = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) {
    s = __dadd_rn(s, partial[i]);
    if (divisor <= 0.0) s2 = __dadd_rn(s2, partial[kRedBlocks + i]);
  }
  const double a = block_sum(s, sh);
  const double c = (divisor <= 0.0) ? block_sum(s2, sh) : divisor;
  if (threadIdx.x == 0) out[0] = (c != 0.0) ? __ddiv_rn(a, c) : 0.0;
}

__global__ void k_subtract(double* __restrict__ x, int64_t n, const double* __restrict__ c) {
  const double cv = *c;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __dsub_rn(x[i], cv);
}

}  // namespace

int boundary_terms(const Pattern* P, const double* node, const int8_t* bdflag, const double* g_side, double g_const,
                   double alpha, double* val, double* b, cudaStream_t s) {
  if (P->N == 0 || P->NT == 0) return FEM_OK;
  const int grid = grid_for(P->N, 256);
  if (P->d == 2)
    FEM_LAUNCH(k_boundary_terms<2>, grid, 256, 0, s, P->N, P->NT, P->elem, P->inc_ptr, P->inc, P->slot, node, bdflag,
               g_side, g_const, alpha, val, b);
  else
    FEM_LAUNCH(k_boundary_terms<3>, grid, 256, 0, s, P->N, P->NT, P->elem, P->inc_ptr, P->inc, P->slot, node, bdflag,
               g_side, g_const, alpha, val, b);
  return FEM_OK;
}

int side_points(const Pattern* P, const double* node, double* pts, cudaStream_t s) {
  const int64_t total = P->NT * P->d1;
  if (P->d == 2) FEM_LAUNCH(k_side_points<2>, grid_for(total, 256), 256, 0, s, P->NT, P->elem, node, pts);
  else FEM_LAUNCH(k_side_points<3>, grid_for(total, 256), 256, 0, s, P->NT, P->elem, node, pts);
  return FEM_OK;
}

int mean_shift(double* x, int64_t n, cudaStream_t s) {
  if (n <= 0) return FEM_OK;
  double* tmp = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, sizeof(double) * (kRedBlocks + 1), s));
  FEM_LAUNCH(k_partial_sum, kRedBlocks, kRedThreads, 0, s, x, n, tmp);
  FEM_LAUNCH(k_finish, 1, kRedThreads, 0, s, tmp, (double)n, tmp + kRedBlocks);
  FEM_LAUNCH(k_subtract, grid_for(n, 256), 256, 0, s, x, n, tmp + kRedBlocks);
  FEM_CUDA(cudaFreeAsync(tmp, s));
  return FEM_OK;
}

int zero_average(const Pattern* P, const double* node, double* u, double* c_out, cudaStream_t s) {
  if (P->N == 0) return FEM_OK;
  double* tmp = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, sizeof(double) * (2 * kRedBlocks + 1), s));
  if (P->d == 2) FEM_LAUNCH(k_partial_average<2>, kRedBlocks, kRedThreads, 0, s, P->NT, P->elem, node, u, tmp);
  else FEM_LAUNCH(k_partial_average<3>, kRedBlocks, kRedThreads, 0, s, P->NT, P->elem, node, u, tmp);
  FEM_LAUNCH(k_finish, 1, kRedThreads, 0, s, tmp, 0.0, tmp + 2 * kRedBlocks);
  FEM_LAUNCH(k_subtract, grid_for(P->N, 256), 256, 0, s, u, P->N, tmp + 2 * kRedBlocks);
  if (c_out) FEM_CUDA(cudaMemcpyAsync(c_out, tmp + 2 * kRedBlocks, sizeof(double), cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaFreeAsync(tmp, s));
  return FEM_OK;
}

}  // namespace fem
