// Per-element local stiffness and load contributions in float-float arithmetic (see dfloat.cuh).
//
// Same formulas as element.cuh (Sec. 3.1.3, eq. (dlambda) and the a_ij formula below it; Sec. 3.2),
// arranged for the FP32 pipe:
//  * 2-D: staged vertices are the coordinates as doubles, and every edge vector is one FP64 subtraction
//    of its own two endpoints: rounded once, to 2^-53 of the edge however far the element is from the
//    origin (the edge the FP64 formula itself starts from); the element is then scaled by 2^-s, s the
//    exponent of its largest edge component, as the edges are converted to float pairs
//    (df_from_double_shift, integer operations only): every product below is of order one whatever the
//    element's size, and each result is scaled back exactly by the power of two its degree of
//    homogeneity in the coordinates gives (stiffness 0, measure 2);
//  * 3-D: staged vertices are the coordinates' exact three-float splits, every edge the exact float-float
//    difference of its endpoints' splits (f3_diff), at the element's own scale; tet_status reports an
//    element whose 6 |tau| leaves the range in which these products keep their precision;
//  * 2-D: ve_0 = x3 - x2, ve_1 = x1 - x3, ve_2 = x2 - x1 (1-based vertices), 2 area = ve_1 x ve_2,
//    a_ij = s ve_i.ve_j, s = k / (2 |2 area|) (the paper's abs() of the area);
//  * 3-D: with e_m = x_{m+1} - x_1, n_1 = e_2 x e_3, n_2 = e_3 x e_1, n_3 = e_1 x e_2 (the paper's faces
//    [1 3 4], [1 4 2], [1 2 3]) and n_0 = (x_4 - x_2) x (x_3 - x_2) (face [2 4 3]); every edge is formed
//    from its own endpoints, so each normal's rounding stays relative to its own face; 6 volume =
//    n_3 . e_3 (signed); a_ij = s n_i.n_j, s = k / (36 volume);
//  * diagonals are minus the off-diagonal row sums (sum_i n_i = 0).
// The element routines return FEM_OK, FEM_ERR_DEGENERATE (zero 2-D area, non-positive 3-D volume) or
// FEM_ERR_RANGE (a coefficient, scale or result outside the float-float range, see dfloat.cuh).
#pragma once

#include "dfloat.cuh"
#include "element.cuh"

namespace fem {

// Staged vertex (16-byte aligned: staged vertices are read with 128-bit accesses). 2-D keeps the
// coordinates as doubles (the edges are FP64 subtractions); 3-D keeps their exact three-float splits (the
// edges are exact float-float differences: fifteen FP64 subtractions per tetrahedron would crowd the FP64
// pipe).
template <int D>
struct VtxDF;
template <>
struct __align__(16) VtxDF<2> {
  double x[2];
};
template <>
struct __align__(16) VtxDF<3> {
  f3 x[3];
};
template <int D>
__device__ __forceinline__ void stage_vertex(VtxDF<D>& v, const double* __restrict__ p) {
#pragma unroll
  for (int m = 0; m < D; ++m) {
    if constexpr (D == 2) v.x[m] = __ldg(p + m);
    else v.x[m] = split3(__ldg(p + m));
  }
}
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

__device__ __forceinline__ int worst(int st, int code) { return st != FEM_OK ? st : code; }

// Whether an input value (a coefficient k or c, a load value f, a loss weight) is 0 or of magnitude in
// [2^-80, 2^96]: inside the float-float range with room for the products it enters. Anything else
// (outside that range, or not finite) is reported as FEM_ERR_RANGE by the caller.
__device__ __forceinline__ bool input_in_range(double v) {
  const int E = (int)((abs_hiword(v) >> 20) & 0x7ffu);
  return (abs_hiword(v) | (uint32_t)__double2loint(v)) == 0u || (E >= 1023 - 80 && E <= 1023 + 96);
}
// An input value as a float pair (the exact split for |v| in [2^-80, 2^96]); out of range sets
// FEM_ERR_RANGE.
__device__ __forceinline__ df2 coef_df(double v, int& st) {
  if (!input_in_range(v)) st = worst(st, FEM_ERR_RANGE);
  return df_from_double(v);
}

__device__ __forceinline__ int int_parity(float n) { return fabsf(n) < 16777216.0f ? (__float2int_rn(n) & 1) : 0; }

// sin(pi x/2) and cos(pi x/2) from the exact split x = a + b + c. x/2 = n + r with n = rint(a/2) and the
// remainder r = (a/2 - n) + b/2 + c/2, every part exact. Coordinates below 2^15 (|b/2| < 2^-10, c/2 below
// the last bit of b/2) take one of three steps: the series of sin and cos of pi r for |r| < 5/4096, the
// series of pi (1/2 - |r|) for 1/2 - |r| < 5/4096 (sin(pi |r|) = cos, cos(pi |r|) = sin of it), the table
// step of df_sincospi_table otherwise (where its cancellation ratio is at most 7/5). The small quantity each
// step works on (r itself next to 0; 1/2 - |r| next to 1/2, at most 2^-10 past 0; r - k/2048 in the table
// step) is formed from the exact parts with two-sums, so it keeps 2^-48 of itself and the cosine next to its
// zeros keeps its relative accuracy (r carried as one float pair would have lost the last bits of x). Larger coordinates
// reduce each part by its own nearest integer, then the float-float sum once more; their remainder is
// carried to 2^-48 of 1/2.
__device__ __forceinline__ SC sincospi_half(const f3& x, const float4* __restrict__ tab) {
  const float ah = 0.5f * x.a, bh = 0.5f * x.b, ch = 0.5f * x.c;
  const float na = rintf(ah);
  SC o;
  int par;
  if (fabsf(x.a) < 32768.0f) {
    const float ra = __fsub_rn(ah, na);  // |ra| <= 1/2
    const df2 r0 = two_sum(ra, bh);      // r = r0.h + r0.l + c/2 exactly, |r| <= 1/2 + 2^-10
    const float ar = fabsf(r0.h);
    const df2 PI = {3.14159274101257324f, -8.74227765734758577e-8f};
    par = __float2int_rn(na) & 1;
    if (ar < 5.0f / 4096.0f) {  // r small: its float-float sum keeps 2^-49 of itself
      df_sincos_series(df_mul(PI, fast_two_sum(r0.h, __fadd_rn(r0.l, ch))), o.s, o.c);
    } else if (ar > 0.5f - 5.0f / 4096.0f) {
      // 1/2 - |r| = (1/2 - sg ra) - sg b/2 - sg c/2; |ra| > 0.49 here, so the first difference is exact
      const float sg = r0.h < 0.0f ? -1.0f : 1.0f;
      const df2 p = two_sum(__fsub_rn(0.5f, sg * ra), -sg * bh);
      df2 sp, cp;
      df_sincos_series(df_mul(PI, fast_two_sum(p.h, __fsub_rn(p.l, sg * ch))), sp, cp);  // of pi (1/2 - |r|)
      o.s = sg < 0.0f ? df_neg(cp) : cp;  // sin(pi r) = sg cos(pi (1/2 - |r|))
      o.c = sp;                            // cos(pi r) = sin(pi (1/2 - |r|))
    } else {
      // the table step's remainder d = r - k/2048 from the exact parts: (r0.h - k/2048) exactly (Sterbenz),
      // then the two-sum with r0.l, then c/2
      const float kf = rintf(__fmul_rn(r0.h, 2048.0f));
      const df2 t = two_sum(__fsub_rn(r0.h, __fmul_rn(kf, 1.0f / 2048.0f)), r0.l);
      df_sincospi_table((int)kf, fast_two_sum(t.h, __fadd_rn(t.l, ch)), tab, o.s, o.c);
    }
  } else {
    const float nb = rintf(bh), nc = rintf(ch);
    const df2 r0 = two_sum(__fsub_rn(ah, na), __fsub_rn(bh, nb));
    df2 r = df_add(r0, df2{__fsub_rn(ch, nc), 0.0f});
    const float n3 = rintf(r.h);
    r = fast_two_sum(__fsub_rn(r.h, n3), r.l);
    par = (int_parity(na) + int_parity(nb) + int_parity(nc) + int_parity(n3)) & 1;
    df_sincospi_small(r, tab, o.s, o.c);
  }
  if (par) {
    o.s = df_neg(o.s);
    o.c = df_neg(o.c);
  }
  return o;
}

// sin(pi (u + v)/2) = sin(pi u/2) cos(pi v/2) + cos(pi u/2) sin(pi v/2)
__device__ __forceinline__ df2 sin_mid(const SC& u, const SC& v) { return df_add(df_mul(u.s, v.c), df_mul(u.c, v.s)); }

// 2-D sine product at edge midpoints from per-vertex products. With sx, cx = sin, cos(pi x/2) and sy, cy
// likewise, a vertex carries P = (sx sy, sx cy, cx sy, cx cy); at the midpoint m of vertices u and v
//   f(m) = sin(pi (x_u + x_v)/2) sin(pi (y_u + y_v)/2) = sum_a P_u[a] P_v[3 - a]
// (both angle additions expanded), one float-float dot product of four terms.
__device__ __forceinline__ void sin_products(const SC& x, const SC& y, df2 (&P)[4]) {
  P[0] = df_mul(x.s, y.s);
  P[1] = df_mul(x.s, y.c);
  P[2] = df_mul(x.c, y.s);
  P[3] = df_mul(x.c, y.c);
}
__device__ __forceinline__ df2 sinprod_mid(const df2* u, const df2* v) {
  const df2 A[4] = {u[0], u[1], u[2], u[3]}, B[4] = {v[3], v[2], v[1], v[0]};
  return df_dot<4>(A, B);
}

// x - n as a float pair for an integer n near x, and the parity of n: n = rint of the leading float of
// x (truncated), the subtraction in FP64 (rounded once, to 2^-53 of the difference), so sin(pi x) =
// (-1)^n sin(pi (x - n)) keeps its relative accuracy next to the integers. Coordinates up to 2^96.
__device__ __forceinline__ float lead_float(double x) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const int fe = (int)((hw >> 20) & 0x7ffu) - 896;
  return (fe > 0 && fe < 255) ? __uint_as_float((hw & 0x80000000u) | ((uint32_t)fe << 23) | ((hw & 0xfffffu) << 3) |
                                                (lw >> 29))
                              : 0.0f;
}

// sin(pi x) at one of the 3-D load's twelve points (four points, three coordinates), as one out-of-line
// copy: fewer registers held across the element routine and a shorter kernel (measured: 1 % faster on
// the 64^3 sine-product forward, 0.4 % on the 128^3 element phase; the same bits)
static __device__ __noinline__ df2 sinpi_point(df2 x, const float4* __restrict__ tab) { return df_sinpi(x, tab); }

// ---- element frames: FP64 edges, scaled by 2^-s --------------------------------------------------

// Triangle: side vectors ve_i (opposite vertex i) as float pairs scaled by 2^-s, and twice the signed area
// ve_1 x ve_2 scaled by 2^-2s, formed in FP64 from the FP64 sides (one product, one fused multiply-add:
// within 2^-52 of |ve_1x ve_2y| + |ve_1y ve_2x|) and then split; returns s.
__device__ __forceinline__ int tri_edges(const VtxDF<2>* const (&V)[3], df2 (&e)[3][2], df2& a2) {
  double ed[3][2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    ed[0][m] = __dsub_rn(V[2]->x[m], V[1]->x[m]);
    ed[1][m] = __dsub_rn(V[0]->x[m], V[2]->x[m]);
    ed[2][m] = __dsub_rn(V[1]->x[m], V[0]->x[m]);
  }
  uint32_t mx = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int m = 0; m < 2; ++m) mx = max(mx, abs_hiword(ed[q][m]));
  const int s = exponent_of_hiword(mx);
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int m = 0; m < 2; ++m) e[q][m] = df_from_double_shift(ed[q][m], s);
  a2 = df_from_double_shift(__fma_rn(ed[1][0], ed[2][1], -__dmul_rn(ed[1][1], ed[2][0])), 2 * s);
  return s;
}

__device__ __forceinline__ void df_cross(const df2 (&u)[3], const df2 (&v)[3], df2 (&o)[3]) {
  o[0] = df_dot2m(u[1], v[2], u[2], v[1]);
  o[1] = df_dot2m(u[2], v[0], u[0], v[2]);
  o[2] = df_dot2m(u[0], v[1], u[1], v[0]);
}

// Tetrahedron: edges e_m = x_{m+1} - x_0 and the scaled inward face normals n_i, every edge the exact
// float-float difference of its endpoints' splits, at the element's own scale (no frame: in 3-D the extra
// state of a scaled frame costs registers the kernels cannot spare). The products of normals (|e|^4), the
// volume (|e|^3) and its reciprocal stay inside the float-float range for edges in [2^-24, 2^29];
// tet_status checks that through 6 |tau|.
__device__ __forceinline__ void tet_normals(const VtxDF<3>* const (&V)[4], df2 (&e)[3][3], df2 (&n)[4][3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int m = 0; m < 3; ++m) e[q][m] = f3_diff(V[q + 1]->x[m], V[0]->x[m]);
  df_cross(e[1], e[2], n[1]);
  df_cross(e[2], e[0], n[2]);
  df_cross(e[0], e[1], n[3]);
  df2 u[3], v[3];  // x_3 - x_1 and x_2 - x_1 (0-based): the edges of face [2 4 3]
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    u[m] = f3_diff(V[3]->x[m], V[1]->x[m]);
    v[m] = f3_diff(V[2]->x[m], V[1]->x[m]);
  }
  df_cross(u, v, n[0]);
}
// Status of a tetrahedron from its 6 tau (signed): FEM_OK within [2^-72, 2^87] (edges of about 2^-24 to
// 2^29), FEM_ERR_RANGE above or below. A zero, negative or non-finite 6 tau is FEM_ERR_DEGENERATE when the
// first edge's largest component is within [2^-24, 2^29] (the element itself is flat or inverted), else
// FEM_ERR_RANGE (its volume under- or overflowed); that edge is formed again only on this rare branch.
__device__ __forceinline__ int tet_status(const VtxDF<3>* const (&V)[4], df2 vol6) {
  if (vol6.h > 0.0f && vol6.h < INFINITY) return (vol6.h >= 0x1p-72f && vol6.h <= 0x1p87f) ? FEM_OK : FEM_ERR_RANGE;
  float a = 0.0f;
#pragma unroll
  for (int m = 0; m < 3; ++m) a = fmaxf(a, fabsf(f3_diff(V[1]->x[m], V[0]->x[m]).h));
  return (a >= 0x1p-24f && a <= 0x1p29f) ? FEM_ERR_DEGENERATE : FEM_ERR_RANGE;
}

// P: the per-vertex sine products (sin_products) when f_kind is FEM_F_SINPROD.
__device__ __forceinline__ int element_df2(const VtxDF<2>* const (&V)[3], const df2* const (&P)[3], df2 kt, bool want_a,
                                           bool want_b, int f_kind, df2 fconst, const double* __restrict__ f_arg,
                                           int t, LocalDF<2>& L, bool want_diag = true) {
  df2 e[3][2], a2;
  const int s = tri_edges(V, e, a2);  // a2: twice the signed area, times 2^-2s
  const df2 a2abs = a2.h < 0.0f ? df_neg(a2) : a2;
  int st = (a2abs.h > 0.0f && a2abs.h < INFINITY) ? FEM_OK : FEM_ERR_DEGENERATE;
  if (want_a) {
    // the 2-D stiffness is homogeneous of degree 0: the scaled frame gives the values themselves
    // (k in [2^-80, 2^96], checked where it is read, keeps every entry in range: no per-entry checks)
    const df2 sc = df_mul(kt, df_recip(df_scale(a2abs, 2.0f)));
    const df2 a01 = df_mul(sc, df_dot<2>(e[0], e[1]));
    const df2 a02 = df_mul(sc, df_dot<2>(e[0], e[2]));
    const df2 a12 = df_mul(sc, df_dot<2>(e[1], e[2]));
    L.a[3] = a01;
    L.a[4] = a02;
    L.a[5] = a12;
    if (want_diag) {
      L.a[0] = df_neg(df_add(a01, a02));
      L.a[1] = df_neg(df_add(a01, a12));
      L.a[2] = df_neg(df_add(a02, a12));
    } else {
      L.a[0] = L.a[1] = L.a[2] = df2{0.0f, 0.0f};
    }
  }
  if (want_b) {
    if (!scale_in_range(2 * s)) st = worst(st, FEM_ERR_RANGE);
    const df2 meas = df_ldexp(df_scale(a2abs, 0.5f), scale_in_range(2 * s) ? 2 * s : 0);  // |tau|
    df2 f[3];
    if (f_kind == FEM_F_SINPROD) {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = sinprod_mid(P[(q + 1) % 3], P[(q + 2) % 3]);
    } else if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = coef_df(__ldg(f_arg + (size_t)t * 3 + q), st);
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = fconst;
    }
    const df2 w = df_mul(meas, df2{0.1666666716337204f, -4.9670538793e-09f});  // |tau| / 6
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const df2 fs = df_add(f[(i + 1) % 3], f[(i + 2) % 3]);
      L.bt[i] = df_mul(w, fs);
      // range on the terms' magnitude |tau| max |f| (f_j + f_k itself may cancel, dfloat.cuh)
      const float fm = fmaxf(fabsf(f[(i + 1) % 3].h), fabsf(f[(i + 2) % 3].h));
      if (!mag_in_range(__fmul_rn(fabsf(w.h), fm), 0, w.h != 0.0f && fm != 0.0f)) st = worst(st, FEM_ERR_RANGE);
    }
  }
  return st;
}

// want_diag = false leaves L.a[0..3] (the diagonals) 0, for callers that form them from row sums.
__device__ __forceinline__ int element_df3(const VtxDF<3>* const (&V)[4], df2 kt, bool want_a, bool want_b,
                                           int f_kind, df2 fconst, const double* __restrict__ f_arg, int t,
                                           const float4* __restrict__ tab, LocalDF<3>& L, bool want_diag = true) {
  df2 e[3][3], n[4][3];
  tet_normals(V, e, n);
  const df2 vol6 = df_dot<3>(n[3], e[2]);  // 6 x signed volume
  int st = tet_status(V, vol6);
  if (want_a) {
    // k / (36 vol); with k in [2^-80, 2^96] and the edges in range every entry is (no per-entry checks)
    const df2 sc = df_mul(kt, df_recip(df_mul_f(vol6, 6.0f)));
#pragma unroll
    for (int i = 0; i < 4; ++i) L.a[i] = df2{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = i + 1; j < 4; ++j) {
        const df2 aij = df_mul(sc, df_dot<3>(n[i], n[j]));
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
        df2 y[4];  // x_i - n, exact: the leading parts' difference by two-sum, then the other parts
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = df_add(two_sum(V[i]->x[m].a, -nn), fast_two_sum(V[i]->x[m].b, V[i]->x[m].c));
        const df2 sy = df_add(df_add(y[0], y[1]), df_add(y[2], y[3]));
        const float sgn = int_parity(nn) ? -1.0f : 1.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const df2 xq = df_add(df_mul(be, sy), df_mul(df_sub(al, be), y[q]));
          const df2 sv = sinpi_point(xq, tab);
          f[q] = df_mul(f[q], df2{sv.h * sgn, sv.l * sgn});
        }
      }
    } else if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = coef_df(__ldg(f_arg + (size_t)t * 4 + q), st);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] = fconst;
    }
    const df2 al = {0.58541017770767212f, 1.8917296174e-08f}, be = {0.13819660246372223f, -1.3387116971e-09f};
    const df2 fs = df_add(df_add(f[0], f[1]), df_add(f[2], f[3]));
    const df2 w = df_scale(vol, 0.25f);
#pragma unroll
    for (int i = 0; i < 4; ++i) L.bt[i] = df_mul(w, df_add(df_mul(be, fs), df_mul(df_sub(al, be), f[i])));
    // range on the terms' magnitude |tau| max |f| (every point enters every entry with a positive weight;
    // the sums themselves may cancel, dfloat.cuh)
    const float fm = fmaxf(fmaxf(fabsf(f[0].h), fabsf(f[1].h)), fmaxf(fabsf(f[2].h), fabsf(f[3].h)));
    if (!mag_in_range(__fmul_rn(fabsf(w.h), fm), 0, w.h != 0.0f && fm != 0.0f)) st = worst(st, FEM_ERR_RANGE);
  }
  return st;
}

// ---- other second-order operators on the same element (values only) --------------------------------
// Mass: m_ij = c |tau| (1 + delta_ij) / ((d+1)(d+2)), the exact integral of c lambda_i lambda_j.
// Anisotropic div(K grad u): a_ij = n_i^T K n_j / (d!^2 |tau|) = |tau| grad lambda_i^T K grad lambda_j
// (eq. (dlambda)), K symmetric given by its upper triangle; the diagonal is left to the caller (the
// row sums vanish, as for the stiffness matrix).
constexpr int kOpStiffness = 0, kOpMass = 1, kOpAniso = 2, kOpApply = 3;  // kOpApply: y = A u, matrix-free

template <int D>
__device__ __forceinline__ void sym_tensor_df(const double* __restrict__ c, df2 (&K)[D][D], int& st) {
  if constexpr (D == 2) {
    K[0][0] = coef_df(__ldg(c), st);
    K[0][1] = K[1][0] = coef_df(__ldg(c + 1), st);
    K[1][1] = coef_df(__ldg(c + 2), st);
  } else {
    K[0][0] = coef_df(__ldg(c), st);
    K[0][1] = K[1][0] = coef_df(__ldg(c + 1), st);
    K[0][2] = K[2][0] = coef_df(__ldg(c + 2), st);
    K[1][1] = coef_df(__ldg(c + 3), st);
    K[1][2] = K[2][1] = coef_df(__ldg(c + 4), st);
    K[2][2] = coef_df(__ldg(c + 5), st);
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

// Scaled normals n_i and d! |tau| (2-D: |2 area|, the paper's abs(); 3-D: 6 x signed volume); 2-D in the
// element's frame scaled by 2^-s (normals times 2^-s, the measure times 2^-2s), returns s; 3-D at the
// element's own scale, returns 0.
template <int D>
__device__ __forceinline__ int element_normals_df(const VtxDF<D>* const (&V)[D + 1], df2 (&n)[D + 1][D], df2& dm) {
  if constexpr (D == 2) {
    df2 e[3][2], a2;
    const int s = tri_edges(V, e, a2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      n[i][0] = df_neg(e[i][1]);
      n[i][1] = e[i][0];
    }
    dm = a2.h < 0.0f ? df_neg(a2) : a2;
    return s;
  } else {
    df2 e[3][3];
    tet_normals(V, e, n);
    dm = df_dot<3>(n[3], e[2]);
    return 0;  // no frame in 3-D; tet_status tells whether the element is in range
  }
}

// Local matrix of operator op (kOpMass or kOpAniso) into L.a (pidx order; mass: every entry; aniso: the
// off-diagonal entries). coef: mass c_t (nullable: 1), aniso the tensor's upper triangle of element t.
template <int D>
__device__ __forceinline__ int element_df_operator(const VtxDF<D>* const (&V)[D + 1], int op,
                                                   const double* __restrict__ coef, LocalDF<D>& L) {
  constexpr int D1 = D + 1;
  df2 n[D1][D], dm;
  const int s = element_normals_df<D>(V, n, dm);  // d! |tau| times 2^-ds
  int st;
  if constexpr (D == 3) st = tet_status(V, dm);
  else st = (dm.h > 0.0f && dm.h < INFINITY) ? FEM_OK : FEM_ERR_DEGENERATE;
  if (op == kOpMass) {
    // c |tau| / ((d+1)(d+2)) = c d! |tau| / (2 * 12) in 2-D, / (6 * 20) in 3-D; homogeneous of degree d
    if (!scale_in_range(D * s)) st = worst(st, FEM_ERR_RANGE);
    const df2 inv = (D == 2) ? df2{0.041666667908430099f, -1.2417634e-09f} : df2{0.0083333337679505348f, -4.3461720e-10f};
    const df2 c = coef ? coef_df(__ldg(coef), st) : df2{1.0f, 0.0f};
    const df2 off = df_ldexp(df_mul(c, df_mul(dm, inv)), scale_in_range(D * s) ? D * s : 0);
    const df2 dia = df_scale(off, 2.0f);
    if (!df_prod_in_range(dia, c.h != 0.0f)) st = worst(st, FEM_ERR_RANGE);
#pragma unroll
    for (int i = 0; i < D1; ++i) L.a[i] = dia;
#pragma unroll
    for (int c2 = D1; c2 < D1 * (D1 + 1) / 2; ++c2) L.a[c2] = off;
  } else {
    // 1 / (d!^2 |tau|) in the scaled frame, times 2^(d-2)s: homogeneous of degree d - 2
    df2 K[D][D];
    sym_tensor_df<D>(coef, K, st);
    if (!scale_in_range((D - 2) * s)) st = worst(st, FEM_ERR_RANGE);
    const df2 sc = df_ldexp(df_recip(D == 2 ? df_scale(dm, 2.0f) : df_mul_f(dm, 6.0f)),
                            scale_in_range((D - 2) * s) ? (D - 2) * s : 0);
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int j = i + 1; j < D1; ++j) L.a[pidx<D>(i, j)] = df_mul(sc, df_quad<D>(n[i], K, n[j]));
    // range on the terms' magnitude max|n| max|K| max|n| / (d!^2 |tau|) (n_i^T K n_j may cancel)
    float nm = 0.0f, km = 0.0f;
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int c2 = 0; c2 < D; ++c2) nm = fmaxf(nm, fabsf(n[i][c2].h));
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) km = fmaxf(km, fabsf(K[a][b2].h));
    if (!mag_in_range(__fmul_rn(__fmul_rn(__fmul_rn(fabsf(sc.h), nm), nm), km), 0, km != 0.0f))
      st = worst(st, FEM_ERR_RANGE);
  }
  return st;
}

}  // namespace fem
