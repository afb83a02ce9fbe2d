// Per-element local stiffness and load contributions in float-float arithmetic (see dfloat.cuh).
//
// Same formulas as element.cuh (Sec. 3.1.3, eq. (dlambda) and the a_ij formula below it; Sec. 3.2),
// arranged for the FP32 pipe:
//  * coordinates arrive as exact three-float splits, so every edge vector is formed to ~2^-47 of its
//    own length (f3_diff);
//  * 2-D: ve_0 = x3 - x2, ve_1 = x1 - x3, ve_2 = x2 - x1 (1-based vertices), 2 area = ve_1 x ve_2,
//    a_ij = s ve_i.ve_j, s = k / (2 |2 area|) (the paper's abs() of the area);
//  * 3-D: with e_m = x_{m+1} - x_1, n_1 = e_2 x e_3, n_2 = e_3 x e_1, n_3 = e_1 x e_2 (the paper's faces
//    [1 3 4], [1 4 2], [1 2 3]) and n_0 = (x_4 - x_2) x (x_3 - x_2) (face [2 4 3]); every edge is
//    formed from its own endpoints, so each normal's rounding stays relative to its own face; volume = n_3 . e_3 / 6 (signed);
//    a_ij = s n_i.n_j, s = k / (36 volume);
//  * diagonals are minus the off-diagonal row sums (sum_i n_i = 0).
#pragma once

#include "dfloat.cuh"
#include "element.cuh"

namespace fem {

// Staged vertex: exact splits of the coordinates, and for the sine-product load the values
// sin(pi x/2), cos(pi x/2) of each coordinate (df).
template <int D>
struct __align__(16) VtxDF {  // 16-byte aligned: staged vertices are read with 128-bit accesses
  f3 x[D];
};
struct __align__(16) SC {
  df2 s, c;
};
// bytes of one staged vertex in shared memory
inline int vtx_bytes(int d) { return d == 2 ? (int)sizeof(VtxDF<2>) : (int)sizeof(VtxDF<3>); }

template <int D>
struct LocalDF {
  df2 a[(D + 1) * (D + 2) / 2];  // pidx order
  df2 bt[D + 1];
};

// sin(pi x/2) and cos(pi x/2) from the exact split of x: x/2 = n + r with n = rint(a/2), r exact to
// ~2^-47 of |r| (so values near the zeros of the sine keep their relative accuracy).
__device__ __forceinline__ SC sincospi_half(const f3& x, const float4* __restrict__ tab) {
  const float ah = 0.5f * x.a, bh = 0.5f * x.b, ch = 0.5f * x.c;
  const float n = rintf(ah);
  const df2 r0 = two_sum(__fsub_rn(ah, n), bh);
  const df2 r = fast_two_sum(r0.h, __fadd_rn(r0.l, ch));
  SC o;
  df_sincospi_small(r, tab, o.s, o.c);
  if (__float2int_rn(n) & 1) {
    o.s = df_neg(o.s);
    o.c = df_neg(o.c);
  }
  return o;
}

// sin(pi (u + v)/2) = sin(pi u/2) cos(pi v/2) + cos(pi u/2) sin(pi v/2)
__device__ __forceinline__ df2 sin_mid(const SC& u, const SC& v) { return df_add(df_mul(u.s, v.c), df_mul(u.c, v.s)); }

// want_diag = false leaves L.a[0..2] (the diagonals) unset, for callers that re-form them.
__device__ __forceinline__ bool element_df2(const VtxDF<2>* const (&V)[3], const SC* const (&S)[3], df2 kt, bool want_a,
                                            bool want_b, int f_kind, df2 fconst, const double* __restrict__ f_arg,
                                            int t, LocalDF<2>& L, bool want_diag = true) {
  // side vectors ve_i (side opposite vertex i), each formed from its own endpoints
  df2 e[3][2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    e[0][m] = f3_diff(V[2]->x[m], V[1]->x[m]);
    e[1][m] = f3_diff(V[0]->x[m], V[2]->x[m]);
    e[2][m] = f3_diff(V[1]->x[m], V[0]->x[m]);
  }
  const df2 a2 = df_dot2m(e[1][0], e[2][1], e[1][1], e[2][0]);  // twice the signed area
  const df2 a2abs = a2.h < 0.0f ? df_neg(a2) : a2;
  const bool ok = a2abs.h > 0.0f && a2abs.h < INFINITY;
  if (want_a) {
    const df2 s = df_mul(kt, df_recip(df_scale(a2abs, 2.0f)));
    const df2 a01 = df_mul(s, df_dot<2>(e[0], e[1]));
    const df2 a02 = df_mul(s, df_dot<2>(e[0], e[2]));
    const df2 a12 = df_mul(s, df_dot<2>(e[1], e[2]));
    L.a[3] = a01;
    L.a[4] = a02;
    L.a[5] = a12;
    if (want_diag) {
      L.a[0] = df_neg(df_add(a01, a02));
      L.a[1] = df_neg(df_add(a01, a12));
      L.a[2] = df_neg(df_add(a02, a12));
    }
  }
  if (want_b) {
    const df2 meas = df_scale(a2abs, 0.5f);
    df2 f[3];
    if (f_kind == FEM_F_SINPROD) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int u = (q + 1) % 3, v = (q + 2) % 3;
        f[q] = df_mul(sin_mid(S[u][0], S[v][0]), sin_mid(S[u][1], S[v][1]));
      }
    } else if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = df_from_double(__ldg(f_arg + (size_t)t * 3 + q));
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = fconst;
    }
    const df2 w = df_mul(meas, df2{0.1666666716337204f, -4.9670538793e-09f});  // |tau| / 6
#pragma unroll
    for (int i = 0; i < 3; ++i) L.bt[i] = df_mul(w, df_add(f[(i + 1) % 3], f[(i + 2) % 3]));
  }
  return ok;
}

__device__ __forceinline__ void df_cross(const df2 (&u)[3], const df2 (&v)[3], df2 (&o)[3]) {
  o[0] = df_dot2m(u[1], v[2], u[2], v[1]);
  o[1] = df_dot2m(u[2], v[0], u[0], v[2]);
  o[2] = df_dot2m(u[0], v[1], u[1], v[0]);
}

// want_diag = false leaves L.a[0..3] (the diagonals) unset, for callers that re-form them.
__device__ __forceinline__ bool element_df3(const VtxDF<3>* const (&V)[4], df2 kt, bool want_a, bool want_b,
                                            int f_kind, df2 fconst, const double* __restrict__ f_arg, int t,
                                            const float4* __restrict__ tab, LocalDF<3>& L, bool want_diag = true) {
  df2 e[3][3];  // e[m-1] = x_m - x_0
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int m = 0; m < 3; ++m) e[q][m] = f3_diff(V[q + 1]->x[m], V[0]->x[m]);
  df2 n[4][3];
  df_cross(e[1], e[2], n[1]);
  df_cross(e[2], e[0], n[2]);
  df_cross(e[0], e[1], n[3]);
  {
    df2 u[3], v[3];  // x_3 - x_1 and x_2 - x_1 (0-based), the edges of face [2 4 3]
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      u[m] = f3_diff(V[3]->x[m], V[1]->x[m]);
      v[m] = f3_diff(V[2]->x[m], V[1]->x[m]);
    }
    df_cross(u, v, n[0]);
  }
  const df2 vol6 = df_dot<3>(n[3], e[2]);  // 6 * signed volume
  const bool ok = vol6.h > 0.0f && vol6.h < INFINITY;
  if (want_a) {
    const df2 s = df_mul(kt, df_recip(df_mul_f(vol6, 6.0f)));  // k / (36 vol)
#pragma unroll
    for (int i = 0; i < 4; ++i) L.a[i] = df2{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i + 1; j < 4; ++j) {
        const df2 aij = df_mul(s, df_dot<3>(n[i], n[j]));
        L.a[pidx<3>(i, j)] = aij;
        if (want_diag) {
          L.a[i] = df_sub(L.a[i], aij);
          L.a[j] = df_sub(L.a[j], aij);
        }
      }
  }
  if (want_b) {
    const df2 vol = df_mul(vol6, df2{0.1666666716337204f, -4.9670538793e-09f});
    df2 f[4];
    if (f_kind == FEM_F_SINPROD) {
      // points x_q = sum_i lambda_i(q) x_i; per coordinate, shifted by an integer n near the element
      // so that sin(pi x) keeps its relative accuracy next to integers
      const df2 al = {0.58541017770767212f, 1.8917296174e-08f}, be = {0.13819660246372223f, -1.3387116971e-09f};
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = df_from(1.0f);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float nn = rintf(V[0]->x[m].a);
        df2 y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const df2 ya = two_sum(V[i]->x[m].a, -nn);
          y[i] = df_add(ya, fast_two_sum(V[i]->x[m].b, V[i]->x[m].c));
        }
        const df2 sy = df_add(df_add(y[0], y[1]), df_add(y[2], y[3]));
        const float sgn = (__float2int_rn(nn) & 1) ? -1.0f : 1.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const df2 xq = df_add(df_mul(be, sy), df_mul(df_sub(al, be), y[q]));
          const df2 sv = df_sinpi(xq, tab);
          f[q] = df_mul(f[q], df2{sv.h * sgn, sv.l * sgn});
        }
      }
    } else if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = df_from_double(__ldg(f_arg + (size_t)t * 4 + q));
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = fconst;
    }
    const df2 al = {0.58541017770767212f, 1.8917296174e-08f}, be = {0.13819660246372223f, -1.3387116971e-09f};
    const df2 fs = df_add(df_add(f[0], f[1]), df_add(f[2], f[3]));
    const df2 w = df_scale(vol, 0.25f);
#pragma unroll
    for (int i = 0; i < 4; ++i) L.bt[i] = df_mul(w, df_add(df_mul(be, fs), df_mul(df_sub(al, be), f[i])));
  }
  return ok;
}

// ---- other second-order operators on the same element (values only) --------------------------------
// Mass: m_ij = c |tau| (1 + delta_ij) / ((d+1)(d+2)), the exact integral of c lambda_i lambda_j.
// Anisotropic div(K grad u): a_ij = n_i^T K n_j / (d!^2 |tau|) = |tau| grad lambda_i^T K grad lambda_j
// (eq. (dlambda)), K symmetric given by its upper triangle; the diagonal is left to the caller (the
// row sums vanish, as for the stiffness matrix).
constexpr int kOpStiffness = 0, kOpMass = 1, kOpAniso = 2, kOpApply = 3;  // kOpApply: y = A u, matrix-free

template <int D>
__device__ __forceinline__ void sym_tensor_df(const double* __restrict__ c, df2 (&K)[D][D]) {
  if constexpr (D == 2) {
    K[0][0] = df_from_double(__ldg(c));
    K[0][1] = K[1][0] = df_from_double(__ldg(c + 1));
    K[1][1] = df_from_double(__ldg(c + 2));
  } else {
    K[0][0] = df_from_double(__ldg(c));
    K[0][1] = K[1][0] = df_from_double(__ldg(c + 1));
    K[0][2] = K[2][0] = df_from_double(__ldg(c + 2));
    K[1][1] = df_from_double(__ldg(c + 3));
    K[1][2] = K[2][1] = df_from_double(__ldg(c + 4));
    K[2][2] = df_from_double(__ldg(c + 5));
  }
}

// n^T K m
template <int D>
__device__ __forceinline__ df2 df_quad(const df2 (&n)[D], const df2 (&K)[D][D], const df2 (&m)[D]) {
  df2 Km[D];
#pragma unroll
  for (int a = 0; a < D; ++a) Km[a] = df_dot<D>(K[a], m);
  return df_dot<D>(n, Km);
}

// scaled normals n_i and d! |tau| (2-D: |2 area|, the paper's abs(); 3-D: 6 x signed volume)
template <int D>
__device__ __forceinline__ df2 element_normals_df(const VtxDF<D>* const (&V)[D + 1], df2 (&n)[D + 1][D]) {
  if constexpr (D == 2) {
    df2 e[3][2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      e[0][m] = f3_diff(V[2]->x[m], V[1]->x[m]);
      e[1][m] = f3_diff(V[0]->x[m], V[2]->x[m]);
      e[2][m] = f3_diff(V[1]->x[m], V[0]->x[m]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      n[i][0] = df_neg(e[i][1]);
      n[i][1] = e[i][0];
    }
    const df2 a2 = df_dot2m(e[1][0], e[2][1], e[1][1], e[2][0]);
    return a2.h < 0.0f ? df_neg(a2) : a2;
  } else {
    df2 e[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int m = 0; m < 3; ++m) e[q][m] = f3_diff(V[q + 1]->x[m], V[0]->x[m]);
    df_cross(e[1], e[2], n[1]);
    df_cross(e[2], e[0], n[2]);
    df_cross(e[0], e[1], n[3]);
    df2 u[3], v[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      u[m] = f3_diff(V[3]->x[m], V[1]->x[m]);
      v[m] = f3_diff(V[2]->x[m], V[1]->x[m]);
    }
    df_cross(u, v, n[0]);
    return df_dot<3>(n[3], e[2]);
  }
}

// Local matrix of operator op (kOpMass or kOpAniso) into L.a (pidx order; mass: every entry; aniso: the
// off-diagonal entries). coef: mass c_t (nullable: 1), aniso the tensor's upper triangle of element t.
template <int D>
__device__ __forceinline__ bool element_df_operator(const VtxDF<D>* const (&V)[D + 1], int op,
                                                    const double* __restrict__ coef, LocalDF<D>& L) {
  constexpr int D1 = D + 1;
  df2 n[D1][D];
  const df2 dm = element_normals_df<D>(V, n);  // d! |tau|
  const bool ok = dm.h > 0.0f && dm.h < INFINITY;
  if (op == kOpMass) {
    // c |tau| / ((d+1)(d+2)) = c d! |tau| / (2 * 12) in 2-D, / (6 * 20) in 3-D
    const df2 inv = (D == 2) ? df2{0.041666667908430099f, -1.2417634e-09f} : df2{0.0083333337679505348f, -4.3461720e-10f};
    const df2 c = coef ? df_from_double(__ldg(coef)) : df2{1.0f, 0.0f};
    const df2 off = df_mul(c, df_mul(dm, inv));
    const df2 dia = df_scale(off, 2.0f);
#pragma unroll
    for (int i = 0; i < D1; ++i) L.a[i] = dia;
#pragma unroll
    for (int c2 = D1; c2 < D1 * (D1 + 1) / 2; ++c2) L.a[c2] = off;
  } else {
    df2 K[D][D];
    sym_tensor_df<D>(coef, K);
    const df2 s = df_recip(D == 2 ? df_scale(dm, 2.0f) : df_mul_f(dm, 6.0f));  // 1 / (d!^2 |tau|)
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int j = i + 1; j < D1; ++j) L.a[pidx<D>(i, j)] = df_mul(s, df_quad<D>(n[i], K, n[j]));
  }
  return ok;
}

}  // namespace fem
