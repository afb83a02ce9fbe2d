// Backward of the assembly: gradients of L = w . val + r . b with respect to the node coordinates and
// the per-element coefficients. The basis gradients are recomputed from the coordinates.
//
// With g_i = grad lambda_i = n_i / (d! |tau|) (eq. (dlambda)), a^tau = k |tau| G G^T, and the
// identities d|tau|/dx_m = |tau| g_m, dg_i/dx_m = -g_m g_i^T:
//   dL/dk_t   = |tau| S,                               S = sum_ij W_ij g_i . g_j
//   dL_A/dx_m = k |tau| (S g_m - sum_i Q_im g_i),     Q = (W + W^T) P, P_ij = g_i . g_j
//   dL_b/dx_m = |tau| g_m sum_i r_i c_i + |tau| sum_q w_q lambda_m(q) grad f(x_q) sum_i r_i lambda_i(q)
// where W_ij = w[slot(t, i, j)], c_i = sum_q w_q f(x_q) lambda_i(q) and (w_q, lambda(q)) is the
// element's quadrature rule. Node gradients are gathered per vertex over its incidence list
// (ascending element order), so the result is deterministic.
#include <cuda_runtime.h>

#include "common.cuh"
#include "element.cuh"

namespace fem {

namespace {

template <int D>
__device__ __forceinline__ void grad_f(int f_kind, const double (&p)[D], double (&g)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) g[c] = 0.0;
  if (f_kind != FEM_F_SINPROD) return;
  double sp[D], cp[D];
#pragma unroll
  for (int m = 0; m < D; ++m) sincospi(p[m], &sp[m], &cp[m]);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double v = 3.14159265358979323846 * cp[c];
#pragma unroll
    for (int m = 0; m < D; ++m)
      if (m != c) v *= sp[m];
    g[c] = v;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_backward_elem(const int32_t* __restrict__ elem, int64_t NT,
                                                       const double* __restrict__ node, const double* __restrict__ k,
                                                       int f_kind, const double* __restrict__ f_arg,
                                                       const int32_t* __restrict__ slot, const double* __restrict__ w,
                                                       const double* __restrict__ r, double* __restrict__ gk,
                                                       double* __restrict__ scratch, int* __restrict__ err) {
  constexpr int D1 = D + 1;
  constexpr double DF = (D == 2) ? 2.0 : 6.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    int e[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) e[i] = elem[t * D1 + i];
    double x[D1][D];
    load_coords<D>(node, e, x);
    double n[D1][D], meas;
    bool ok;
    if constexpr (D == 2) {
      ok = normals2(x, n, meas);
      // the backward needs the signed area: reject inverted triangles
      const double a2 = (x[1][0] - x[0][0]) * (x[2][1] - x[0][1]) - (x[1][1] - x[0][1]) * (x[2][0] - x[0][0]);
      ok = ok && a2 > 0.0;
    } else {
      ok = normals3(x, n, meas);
    }
    if (!ok) report(err, FEM_ERR_DEGENERATE);
    double g[D1][D];
    const double inv = 1.0 / (DF * meas);
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int c = 0; c < D; ++c) g[i][c] = n[i][c] * inv;
    double P[D1][D1];
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int j = 0; j < D1; ++j) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += g[i][c] * g[j][c];
        P[i][j] = s;
      }
    const double kt = k ? k[t] : 1.0;
    double out[D1][D];
#pragma unroll
    for (int m = 0; m < D1; ++m)
#pragma unroll
      for (int c = 0; c < D; ++c) out[m][c] = 0.0;
    if (w) {
      double W[D1][D1];
#pragma unroll
      for (int i = 0; i < D1; ++i)
#pragma unroll
        for (int j = 0; j < D1; ++j) W[i][j] = __ldg(w + slot[(int64_t)(i * D1 + j) * NT + t]);
      double S = 0.0;
#pragma unroll
      for (int i = 0; i < D1; ++i)
#pragma unroll
        for (int j = 0; j < D1; ++j) S += W[i][j] * P[i][j];
      if (gk) gk[t] = meas * S;
#pragma unroll
      for (int m = 0; m < D1; ++m) {
        double acc[D];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = S * g[m][c];
#pragma unroll
        for (int i = 0; i < D1; ++i) {
          double q = 0.0;
#pragma unroll
          for (int j = 0; j < D1; ++j) q += (W[i][j] + W[j][i]) * P[j][m];
#pragma unroll
          for (int c = 0; c < D; ++c) acc[c] -= q * g[i][c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) out[m][c] = kt * meas * acc[c];
      }
    } else if (gk) {
      gk[t] = 0.0;
    }
    if (r) {
      double rv[D1];
#pragma unroll
      for (int i = 0; i < D1; ++i) rv[i] = __ldg(r + e[i]);
      double fq[D1];
      f_at_points<D>(x, f_kind, f_arg, t, fq);
      // rule: 2-D midpoints (w_q = 1/3, lambda_i(q) = 1/2 for i != q, 0 for i == q);
      //       3-D (w_q = 1/4, lambda_i(q) = alpha if i == q else beta)
      double lam[D1][D1];
      double wq;
      double pts[D1][D];
      if constexpr (D == 2) {
        wq = 1.0 / 3.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
          for (int i = 0; i < 3; ++i) lam[q][i] = (i == q) ? 0.0 : 0.5;
#pragma unroll
          for (int c = 0; c < 2; ++c) pts[q][c] = (x[(q + 1) % 3][c] + x[(q + 2) % 3][c]) * 0.5;
        }
      } else {
        wq = 0.25;
        const double s5 = 2.23606797749978969641;
        const double alpha = (5.0 + 3.0 * s5) / 20.0, beta = (5.0 - s5) / 20.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int i = 0; i < 4; ++i) lam[q][i] = (i == q) ? alpha : beta;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) s += lam[q][i] * x[i][c];
            pts[q][c] = s;
          }
        }
      }
      double Rb = 0.0;
#pragma unroll
      for (int i = 0; i < D1; ++i) {
        double ci = 0.0;
#pragma unroll
        for (int q = 0; q < D1; ++q) ci += wq * fq[q] * lam[q][i];
        Rb += rv[i] * ci;
      }
      double gf[D1][D], rl[D1];
#pragma unroll
      for (int q = 0; q < D1; ++q) {
        grad_f<D>(f_kind, pts[q], gf[q]);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < D1; ++i) s += rv[i] * lam[q][i];
        rl[q] = s;
      }
#pragma unroll
      for (int m = 0; m < D1; ++m)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          double s2 = 0.0;
#pragma unroll
          for (int q = 0; q < D1; ++q) s2 += wq * lam[q][m] * gf[q][c] * rl[q];
          out[m][c] += meas * g[m][c] * Rb + meas * s2;
        }
    }
#pragma unroll
    for (int m = 0; m < D1; ++m)
#pragma unroll
      for (int c = 0; c < D; ++c) scratch[(int64_t)(m * D + c) * NT + t] = out[m][c];
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_backward_gather(const int32_t* __restrict__ inc_ptr,
                                                         const int32_t* __restrict__ inc, int64_t N, int64_t NT,
                                                         const double* __restrict__ scratch, double* __restrict__ gnode) {
  constexpr int D1 = D + 1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    for (int q = inc_ptr[v]; q < inc_ptr[v + 1]; ++q) {
      const int p = inc[q];
      const int64_t t = p / D1;
      const int m = p - (int)t * D1;
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] = acc[c] + scratch[(int64_t)(m * D + c) * NT + t];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) gnode[v * D + c] = acc[c];
  }
}

}  // namespace

int assemble_backward(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                      const double* w, const double* r, double* gnode, double* gk, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  if (!P->scratch) return set_error(FEM_ERR_STATE, "pattern has no scratch for the backward gather");
  const int64_t NT = P->NT, N = P->N;
  if (NT == 0) {
    if (gnode && N > 0) FEM_CUDA(cudaMemsetAsync(gnode, 0, sizeof(double) * N * P->d, s));
    return FEM_OK;
  }
  const int grid = grid_for(NT, 256, 152 * 16);
  if (P->d == 2) {
    FEM_LAUNCH(k_backward_elem<2>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, w, r, gk, P->scratch,
               err);
    if (gnode) FEM_LAUNCH(k_backward_gather<2>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, N, NT, P->scratch, gnode);
  } else {
    FEM_LAUNCH(k_backward_elem<3>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, w, r, gk, P->scratch,
               err);
    if (gnode) FEM_LAUNCH(k_backward_gather<3>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, N, NT, P->scratch, gnode);
  }
  return FEM_OK;
}

}  // namespace fem
