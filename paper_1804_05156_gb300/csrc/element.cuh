// Per-element geometry and local quantities in FP64 (device functions).
//
// Sec. 3.1.3. 2-D: side vectors ve_i = x_{i+2} - x_{i+1} (indices mod 3; ve_i is the side opposite
// vertex i traversed counter-clockwise), twice the signed area A2 = ve_3 x ve_1 ... written out below,
// and n_i . n_j = ve_i . ve_j. 3-D: n_i = (x_f2 - x_f1) x (x_f3 - x_f1) for the faces
// [2 4 3], [1 3 4], [1 4 2], [1 2 3] (1-based), volume = n_4 . (x_4 - x_1) / 6 (signed).
#pragma once

#include <cuda_runtime.h>

#include "femasm.h"

namespace fem {

// Index of the unique local pair (i, j) in the per-element value list: diagonals first (0..d), then
// the upper off-diagonals in row order.
template <int D>
__host__ __device__ constexpr int pidx(int i, int j) {
  return (i == j) ? i
                  : (D == 2 ? 3 + ((i < j ? i : j) == 0 ? ((i > j ? i : j) - 1) : 2)
                            : 4 + ((i < j ? i : j) == 0   ? ((i > j ? i : j) - 1)
                                   : (i < j ? i : j) == 1 ? ((i > j ? i : j) + 1)
                                                          : 5));
}
// Same map for run-time (i, j): the (d+1)^2 results packed 4 bits each in one 64-bit constant.
template <int D>
__host__ __device__ constexpr uint64_t pidx_table() {
  uint64_t t = 0;
  for (int i = 0; i < D + 1; ++i)
    for (int j = 0; j < D + 1; ++j) t |= (uint64_t)pidx<D>(i, j) << (4 * (i * (D + 1) + j));
  return t;
}
template <int D>
__device__ __forceinline__ int pidx_rt(int i, int j) {
  constexpr uint64_t T = pidx_table<D>();
  return (int)((T >> (4 * (i * (D + 1) + j))) & 15u);
}

template <int D>
struct Local {
  double a[(D + 1) * (D + 2) / 2];  // unique entries, pidx order
  double bt[D + 1];                 // load-vector contributions
  double meas;                      // |tau| (2-D abs area, 3-D signed volume)
};

template <int D>
__device__ __forceinline__ void load_coords(const double* __restrict__ node, const int (&e)[D + 1], double (&x)[D + 1][D]) {
#pragma unroll
  for (int i = 0; i < D + 1; ++i)
#pragma unroll
    for (int m = 0; m < D; ++m) x[i][m] = __ldg(node + (int64_t)e[i] * D + m);
}

// f at a point, for FEM_F_CONST / FEM_F_SINPROD (FEM_F_QPVALUES is read by the caller).
template <int D>
__device__ __forceinline__ double f_point(int f_kind, const double* __restrict__ f_arg, const double (&p)[D]) {
  if (f_kind == FEM_F_CONST) return f_arg ? __ldg(f_arg) : 1.0;
  double v = 1.0;
#pragma unroll
  for (int m = 0; m < D; ++m) v *= sinpi(p[m]);
  return v;
}

// Scaled normals n[i] (D components) and |tau|; returns false for a degenerate element.
__device__ __forceinline__ bool normals2(const double (&x)[3][2], double (&n)[3][2], double& meas) {
  double ve[3][2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    ve[0][m] = x[2][m] - x[1][m];
    ve[1][m] = x[0][m] - x[2][m];
    ve[2][m] = x[1][m] - x[0][m];
  }
  const double a2 = -ve[2][0] * ve[1][1] + ve[2][1] * ve[1][0];
  meas = 0.5 * fabs(a2);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    n[i][0] = -ve[i][1];
    n[i][1] = ve[i][0];
  }
  return meas > 0.0 && meas < INFINITY;
}

__device__ __forceinline__ bool normals3(const double (&x)[4][3], double (&n)[4][3], double& meas) {
  constexpr int F[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double u[3], v[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      u[m] = x[F[i][1]][m] - x[F[i][0]][m];
      v[m] = x[F[i][2]][m] - x[F[i][0]][m];
    }
    n[i][0] = u[1] * v[2] - u[2] * v[1];
    n[i][1] = u[2] * v[0] - u[0] * v[2];
    n[i][2] = u[0] * v[1] - u[1] * v[0];
  }
  meas = (n[3][0] * (x[3][0] - x[0][0]) + n[3][1] * (x[3][1] - x[0][1]) + n[3][2] * (x[3][2] - x[0][2])) / 6.0;
  return meas > 0.0 && meas < INFINITY;
}

// Quadrature points of the element's rule and f there.
template <int D>
__device__ __forceinline__ void f_at_points(const double (&x)[D + 1][D], int f_kind, const double* __restrict__ f_arg,
                                            int64_t t, double (&fq)[D + 1]) {
  if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
    for (int q = 0; q < D + 1; ++q) fq[q] = __ldg(f_arg + t * (D + 1) + q);
    return;
  }
  if (f_kind == FEM_F_CONST) {
    const double c = f_arg ? __ldg(f_arg) : 1.0;
#pragma unroll
    for (int q = 0; q < D + 1; ++q) fq[q] = c;
    return;
  }
  if (D == 2) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double p[D];
#pragma unroll
      for (int m = 0; m < D; ++m) p[m] = (x[(q + 1) % 3][m] + x[(q + 2) % 3][m]) * 0.5;
      fq[q] = f_point<D>(f_kind, f_arg, p);
    }
  } else {
    const double s5 = 2.23606797749978969641;  // sqrt(5)
    const double alpha = (5.0 + 3.0 * s5) / 20.0, beta = (5.0 - s5) / 20.0;
#pragma unroll
    for (int q = 0; q < D + 1; ++q) {
      double p[D];
#pragma unroll
      for (int m = 0; m < D; ++m) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < D + 1; ++i) s += (i == q ? alpha : beta) * x[i][m];
        p[m] = s;
      }
      fq[q] = f_point<D>(f_kind, f_arg, p);
    }
  }
}

// Local stiffness (times k) and load contributions of one element. Returns false if degenerate.
template <int D>
__device__ __forceinline__ bool element_local(const double (&x)[D + 1][D], double kt, bool want_a, bool want_b,
                                              int f_kind, const double* __restrict__ f_arg, int64_t t, Local<D>& L) {
  constexpr int D1 = D + 1;
  double n[D1][D];
  bool ok;
  if constexpr (D == 2) ok = normals2(x, n, L.meas);
  else ok = normals3(x, n, L.meas);
  if (want_a) {
    const double sc = kt / ((D == 2 ? 4.0 : 36.0) * L.meas);
#pragma unroll
    for (int i = 0; i < D1; ++i) L.a[i] = 0.0;
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int j = i + 1; j < D1; ++j) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < D; ++m) s = fma(n[i][m], n[j][m], s);
        const double aij = s * sc;
        L.a[pidx<D>(i, j)] = aij;
        L.a[i] -= aij;
        L.a[j] -= aij;
      }
  }
  if (want_b) {
    double fq[D1];
    f_at_points<D>(x, f_kind, f_arg, t, fq);
    if constexpr (D == 2) {
#pragma unroll
      for (int i = 0; i < 3; ++i) L.bt[i] = L.meas * (fq[(i + 1) % 3] + fq[(i + 2) % 3]) / 6.0;
    } else {
      const double s5 = 2.23606797749978969641;
      const double alpha = (5.0 + 3.0 * s5) / 20.0, beta = (5.0 - s5) / 20.0;
      const double fs = fq[0] + fq[1] + fq[2] + fq[3];
#pragma unroll
      for (int i = 0; i < 4; ++i) L.bt[i] = L.meas * 0.25 * (beta * fs + (alpha - beta) * fq[i]);
    }
  }
  return ok;
}

}  // namespace fem
