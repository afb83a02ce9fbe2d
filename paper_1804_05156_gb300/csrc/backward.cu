// Backward of the assembly: gradients of L = w . val + r . b with respect to the node coordinates and
// the per-element coefficients, in float-float arithmetic (dfloat.cuh).
//
// With g_i = grad lambda_i = n_i / (d! |tau|) (eq. (dlambda)), a^tau = k |tau| G G^T, the identities
// d|tau|/dx_m = |tau| g_m and dg_i/dx_m = -g_m g_i^T, W_ij = w[slot(t, i, j)] and P_ij = g_i . g_j:
//   dL/dk_t   = |tau| S,                           S = sum_ij W_ij P_ij
//   dL_A/dx_m = k |tau| (S g_m - sum_i Q_im g_i),  Q = (W + W^T) P
//   dL_b/dx_m = |tau| g_m sum_q w_q f_q rl_q + |tau| sum_q w_q lambda_m(q) grad f(x_q) rl_q,
//               rl_q = sum_i r_i lambda_i(q)
// One thread per element writes gk[t] and its (d+1) x d vertex contributions (float pairs); a second
// kernel sums each vertex's contributions over its incidence list in ascending element order
// (deterministic) and writes gnode. When the pattern has a tile plan the elements run in tile order with
// their vertices split once per tile in shared memory, and the contributions of element-row (t, m) go to
// the plan's packet slot of incidence (t, m), so each vertex reads its contributions contiguously;
// otherwise they run in the caller's order and go to the pattern's scratch. No FP64 arithmetic except
// the loss-weight pair sums and the final rounding of each output.
#include <cuda_runtime.h>

#include "common.cuh"
#include "element_df.cuh"
#include "packet.cuh"

namespace fem {

const float4* sincos_table_device();  // values_blocked.cu

namespace {

// sin and cos of pi x for the 3-D load adjoint's twelve points, as one out-of-line copy: the element
// adjoint's straight-line code is long enough that instruction fetch stalls it, and twelve inlined
// copies of this evaluation are a large part of it (measured: 1 % faster than inlined, the same bits)
__device__ __noinline__ void sincospi_point(df2 x, const float4* __restrict__ tab, df2& s, df2& c) {
  df_sincospi(x, tab, s, c);
}

// Adjoint of one element: out[m][c] = dL/dx_{m,c} contributions and gkv = dL/dk_t, from the staged
// coordinates V, the coefficient kt, the symmetrised loss weights Ws = W + W^T (with_w) and the
// load-vector weights rv of the element's vertices (with_r). Returns FEM_OK, FEM_ERR_DEGENERATE or
// FEM_ERR_RANGE (element_df.cuh).
// The geometry is that of the value kernels. 2-D: FP64 edges, the element scaled by 2^-s, so that g_i,
// |tau| and every product of them stay of order one; each term is scaled back by its degree of
// homogeneity in the coordinates: dL/dk and the stiffness part of dL/dx by 2^(d-2)s and 2^(d-3)s, the
// load part's |tau| g_m term by 2^(d-1)s and its |tau| grad f term by 2^ds. 3-D: exact split edges at
// the element's own scale (s = 0), within the 6 |tau| range tet_status checks.
// Stiffness part in the form that needs the fewest products: h_j = sum_i Ws_ij g_i, then
// S = (1/2) sum_j h_j . g_j and sum_i Q_im g_i = sum_j (g_j . g_m) h_j.
template <int D>
__device__ __forceinline__ int element_adjoint(const VtxDF<D>* const (&V)[D + 1], int t, df2 kt, bool with_w,
                                               const df2 (&Ws)[D + 1][D + 1], bool with_r, const df2 (&rv)[D + 1],
                                               int f_kind, const double* __restrict__ f_arg,
                                               const float4* __restrict__ tab, df2 (&out)[D + 1][D], df2& gkv) {
  constexpr int D1 = D + 1;
  // scaled inward normals n_i and the positive measure |tau| (d! |tau| = signed 2-D area x 2, 3-D vol x 6),
  // 2-D in the element's frame scaled by 2^-s, 3-D at the element's own scale (s = 0)
  df2 n[D1][D];
  df2 dmeas;  // d! |tau| times 2^-ds
  int s;
  if constexpr (D == 2) {
    df2 ev[3][2];
    s = tri_edges(V, ev, dmeas);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      n[i][0] = df_neg(ev[i][1]);
      n[i][1] = ev[i][0];
    }
  } else {
    df2 ed[3][3];
    tet_normals(V, ed, n);
    dmeas = df_dot<3>(n[3], ed[2]);
    s = 0;  // no frame in 3-D
  }
  int st;
  if constexpr (D == 3) st = tet_status(V, dmeas);
  else st = (dmeas.h > 0.0f && dmeas.h < INFINITY) ? FEM_OK : FEM_ERR_DEGENERATE;
  const int eA = (D - 3) * s, eK = (D - 2) * s, e1 = (D - 1) * s, e2 = D * s;
  if (!(scale_in_range(eA) && scale_in_range(e2))) st = worst(st, FEM_ERR_RANGE);
  // the exponent of the element's size: 3-D, from 6 |tau| (about |e|^3), for the range checks of terms of
  // other degrees; 2-D works in its frame, whose shifts s.. carry the size
  const int ge = (D == 3) ? (fexp(dmeas.h) + 300) / 3 - 100 : 0;
  const int sA = scale_in_range(eA) ? eA : 0, sK = scale_in_range(eK) ? eK : 0;
  const int s1 = scale_in_range(e1) ? e1 : 0, s2 = scale_in_range(e2) ? e2 : 0;
  const df2 inv = df_recip(dmeas);
  const df2 meas = (D == 2) ? df_scale(dmeas, 0.5f) : df_mul(dmeas, df2{0.1666666716337204f, -4.9670538793e-09f});
  df2 g[D1][D];
#pragma unroll
  for (int i = 0; i < D1; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) g[i][c] = df_mul(n[i][c], inv);
#pragma unroll
  for (int i = 0; i < D1; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) out[i][c] = df2{0.0f, 0.0f};
  gkv = df2{0.0f, 0.0f};
  if (with_w) {
    // range, on the magnitudes of the terms (their sums may cancel, dfloat.cuh), by exponents: |tau| W g g
    // for dL/dk (degree d - 2 in the coordinates) and k |tau| W g g g for dL/dx (degree d - 3)
    float wm = 0.0f;
#pragma unroll
    for (int i = 0; i < D1; ++i)
#pragma unroll
      for (int j = 0; j < D1; ++j) wm = fmaxf(wm, fabsf(Ws[i][j].h));
    if (wm != 0.0f && (!exp_in_range(fexp(wm) + sK + (D - 2) * ge) ||
                       (kt.h != 0.0f && !exp_in_range(fexp(kt.h) + fexp(wm) + sA + (D - 3) * ge))))
      st = worst(st, FEM_ERR_RANGE);
    // h_j = sum_i Ws_ij g_i, each component one fused float-float dot product
    df2 h[D1][D];
#pragma unroll
    for (int j = 0; j < D1; ++j)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        df2 A[D1], B[D1];
#pragma unroll
        for (int i = 0; i < D1; ++i) {
          A[i] = Ws[i][j];
          B[i] = g[i][c];
        }
        h[j][c] = df_dot<D1>(A, B);
      }
    df2 S2;  // sum_j h_j . g_j
    {
      df2 A[D1 * D], B[D1 * D];
#pragma unroll
      for (int j = 0; j < D1; ++j)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          A[j * D + c] = h[j][c];
          B[j * D + c] = g[j][c];
        }
      S2 = df_dot<D1 * D>(A, B);
    }
    const df2 S = df_scale(S2, 0.5f);
    gkv = df_ldexp(df_mul(meas, S), sK);
    const df2 km = df_mul(kt, meas);
    df2 P[D1][D1];  // g_j . g_m (symmetric)
#pragma unroll
    for (int j = 0; j < D1; ++j)
#pragma unroll
      for (int m = j; m < D1; ++m) {
        P[j][m] = df_dot<D>(g[j], g[m]);
        P[m][j] = P[j][m];
      }
#pragma unroll
    for (int m = 0; m < D1; ++m)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        // S g_m - sum_j P_jm h_j
        df2 A[D1 + 1], B[D1 + 1];
        A[0] = S;
        B[0] = g[m][c];
#pragma unroll
        for (int j = 0; j < D1; ++j) {
          A[j + 1] = df_neg(P[j][m]);
          B[j + 1] = h[j][c];
        }
        out[m][c] = df_ldexp(df_mul(km, df_dot<D1 + 1>(A, B)), sA);
      }
  }
  if (with_r) {
    // quadrature points: f, grad f; barycentric weights lambda_q(q) = lo + ld, lambda_i(q) = lo (i != q)
    // and the point weight wqd, as float-float constants (2-D: edge midpoints, 1/2 and 0, weight 1/3;
    // 3-D: (a, b, b, b) with a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, weight 1/4)
    df2 fq[D1], gf[D1][D];
    df2 lo, ld, wqd;
    if constexpr (D == 2) {
      lo = df2{0.5f, 0.0f};
      ld = df2{-0.5f, 0.0f};
      wqd = df2{0.3333333432674408f, -9.9341077586e-09f};
    } else {
      const df2 al = {0.58541017770767212f, 1.8917296174e-08f}, be = {0.13819660246372223f, -1.3387116971e-09f};
      lo = be;
      ld = df_sub(al, be);
      wqd = df2{0.25f, 0.0f};
    }
#pragma unroll
    for (int q = 0; q < D1; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) gf[q][c] = df2{0.0f, 0.0f};
    if (f_kind == FEM_F_SINPROD) {
      df2 sn[D1][D], cs[D1][D];  // sin(pi x_q,m), cos(pi x_q,m)
      if constexpr (D == 2) {
        SC sc[3][2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int m = 0; m < 2; ++m) sc[i][m] = sincospi_half(split3(V[i]->x[m]), tab);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int u = (q + 1) % 3, v = (q + 2) % 3;
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            sn[q][m] = sin_mid(sc[u][m], sc[v][m]);
            cs[q][m] = df_sub(df_mul(sc[u][m].c, sc[v][m].c), df_mul(sc[u][m].s, sc[v][m].s));
          }
        }
      } else {
        const df2 al = {0.58541017770767212f, 1.8917296174e-08f}, be = {0.13819660246372223f, -1.3387116971e-09f};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const float nn = rintf(V[0]->x[m].a);
          df2 y[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            y[i] = df_add(two_sum(V[i]->x[m].a, -nn), fast_two_sum(V[i]->x[m].b, V[i]->x[m].c));
          const df2 sy = df_add(df_add(y[0], y[1]), df_add(y[2], y[3]));
          const float sgn = int_parity(nn) ? -1.0f : 1.0f;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            sincospi_point(df_add(df_mul(be, sy), df_mul(df_sub(al, be), y[q])), tab, sn[q][m], cs[q][m]);
            sn[q][m] = df2{sn[q][m].h * sgn, sn[q][m].l * sgn};
            cs[q][m] = df2{cs[q][m].h * sgn, cs[q][m].l * sgn};
          }
        }
      }
      const df2 PI = {3.14159274101257324f, -8.74227765734758577e-8f};
#pragma unroll
      for (int q = 0; q < D1; ++q) {
        df2 f = sn[q][0];
#pragma unroll
        for (int m = 1; m < D; ++m) f = df_mul(f, sn[q][m]);
        fq[q] = f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          df2 gv = df_mul(PI, cs[q][c]);
#pragma unroll
          for (int m = 0; m < D; ++m)
            if (m != c) gv = df_mul(gv, sn[q][m]);
          gf[q][c] = gv;
        }
      }
    } else if (f_kind == FEM_F_QPVALUES) {
#pragma unroll
      for (int q = 0; q < D1; ++q) fq[q] = coef_df(__ldg(f_arg + (size_t)t * D1 + q), st);
    } else {
      const df2 c0 = f_arg ? coef_df(__ldg(f_arg), st) : df2{1.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < D1; ++q) fq[q] = c0;
    }
    // range, on the magnitudes of the terms, by exponents: |tau| g r f (degree d - 1) and, for the sine
    // product, |tau| r grad f (degree d)
    float rm = 0.0f, fm = 0.0f, dm = 0.0f;
#pragma unroll
    for (int q = 0; q < D1; ++q) {
      rm = fmaxf(rm, fabsf(rv[q].h));
      fm = fmaxf(fm, fabsf(fq[q].h));
#pragma unroll
      for (int c = 0; c < D; ++c) dm = fmaxf(dm, fabsf(gf[q][c].h));
    }
    if (rm != 0.0f && ((fm != 0.0f && !exp_in_range(fexp(rm) + fexp(fm) + s1 + (D - 1) * ge)) ||
                       (dm != 0.0f && !exp_in_range(fexp(rm) + fexp(dm) + s2 + D * ge))))
      st = worst(st, FEM_ERR_RANGE);
    // rl_q = sum_i r_i lambda_i(q) = lo sum_i r_i + ld r_q;  Rb = sum_q w_q f_q rl_q
    df2 rs = rv[0];
#pragma unroll
    for (int i = 1; i < D1; ++i) rs = df_add(rs, rv[i]);
    df2 rl[D1];
#pragma unroll
    for (int q = 0; q < D1; ++q) rl[q] = df_add(df_mul(rs, lo), df_mul(rv[q], ld));
    const df2 Rb = df_mul(wqd, df_dot<D1>(fq, rl));
    // sum_q w_q lambda_m(q) grad f(x_q) rl_q = w_q (lo sum_q gr_q + ld gr_m), gr_q = grad f(x_q) rl_q
    df2 gr[D1][D], gs[D];
    if (f_kind == FEM_F_SINPROD) {
#pragma unroll
      for (int q = 0; q < D1; ++q)
#pragma unroll
        for (int c = 0; c < D; ++c) gr[q][c] = df_mul(gf[q][c], rl[q]);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        df2 a = gr[0][c];
#pragma unroll
        for (int q = 1; q < D1; ++q) a = df_add(a, gr[q][c]);
        gs[c] = a;
      }
    }
#pragma unroll
    for (int m = 0; m < D1; ++m)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        // |tau| g_m Rb (degree d - 1) and |tau| sum_q w_q lambda_m(q) grad f(x_q) rl_q (degree d)
        df2 v = df_ldexp(df_mul(meas, df_mul(g[m][c], Rb)), s1);
        if (f_kind == FEM_F_SINPROD)
          v = df_add(v, df_ldexp(df_mul(meas, df_mul(wqd, df_add(df_mul(gs[c], lo), df_mul(gr[m][c], ld)))), s2));
        out[m][c] = df_add(out[m][c], v);
      }
  }
  // and no result overflows
  bool fin = fabsf(gkv.h) <= 0x1p120f;
#pragma unroll
  for (int m = 0; m < D1; ++m)
#pragma unroll
    for (int c = 0; c < D; ++c) fin = fin && fabsf(out[m][c].h) <= 0x1p120f;
  if (!fin) st = worst(st, FEM_ERR_RANGE);
  return st;
}

// Ws = W + W^T of element t from the loss weights on its slots (pairs summed in FP64, then split)
template <int D>
__device__ __forceinline__ void sym_weights(const int32_t* __restrict__ slot, int64_t NT, int t,
                                            const double* __restrict__ w, df2 (&Ws)[D + 1][D + 1], int& st) {
  constexpr int D1 = D + 1;
#pragma unroll
  for (int i = 0; i < D1; ++i)
#pragma unroll
    for (int j = i; j < D1; ++j) {
      const double wij = __ldg(w + __ldg(slot + (size_t)(i * D1 + j) * NT + t));
      const double wji = (i == j) ? wij : __ldg(w + __ldg(slot + (size_t)(j * D1 + i) * NT + t));
      const double ws = __dadd_rn(wij, wji);
      if (!input_in_range(ws)) st = worst(st, FEM_ERR_RANGE);
      Ws[i][j] = df_from_double_fast(ws);
      Ws[j][i] = Ws[i][j];
    }
}

// Element order of the caller, vertices read per element; contributions to scratch[(m*D+c)*NT + t].
template <int D>
__global__ void __launch_bounds__(128, 4) k_backward_df(const int32_t* __restrict__ elem, int NT,
                                                        const double* __restrict__ node, const double* __restrict__ k,
                                                        int f_kind, const double* __restrict__ f_arg,
                                                        const int32_t* __restrict__ slot, const double* __restrict__ w,
                                                        const double* __restrict__ r, double* __restrict__ gk,
                                                        float2* __restrict__ scratch, const float4* __restrict__ tab,
                                                        int* __restrict__ err) {
  constexpr int D1 = D + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  int e[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) e[i] = __ldg(elem + (size_t)t * D1 + i);
  VtxDF<D> X[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) stage_vertex<D>(X[i], node + (size_t)e[i] * D);
  df2 Ws[D1][D1], rv[D1];
  int st = FEM_OK;
  if (w) sym_weights<D>(slot, NT, t, w, Ws, st);
  if (r) {
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      const double ri = __ldg(r + e[i]);
      if (!input_in_range(ri)) st = worst(st, FEM_ERR_RANGE);
      rv[i] = df_from_double_fast(ri);
    }
  }
  const df2 kt = k ? coef_df(__ldg(k + t), st) : df2{1.0f, 0.0f};
  const VtxDF<D>* V[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) V[i] = &X[i];
  df2 out[D1][D], gkv;
  st = worst(st, element_adjoint<D>(reinterpret_cast<const VtxDF<D>* const(&)[D1]>(V), t, kt, w != nullptr, Ws,
                                    r != nullptr, rv, f_kind, f_arg, tab, out, gkv));
  if (st != FEM_OK) report(err, st);
  if (gk) gk[t] = df_to_double(gkv);
#pragma unroll
  for (int m = 0; m < D1; ++m)
#pragma unroll
    for (int c = 0; c < D; ++c) scratch[(size_t)(m * D + c) * NT + t] = make_float2(out[m][c].h, out[m][c].l);
}

// Tile order (the forward's tile plan): the tile's vertices are split once into shared memory; the
// contributions of element-row (t, m) go to packet ipos(t, m), so each vertex's packets are contiguous.
template <int D, int TE>
__global__ void __launch_bounds__(TE, 512 / TE) k_backward_tiles(
    int64_t NT, const int32_t* __restrict__ elist, const uint16_t* __restrict__ lelem, const int32_t* __restrict__ voff,
    const int32_t* __restrict__ vlist, const int32_t* __restrict__ ipos, const double* __restrict__ node,
    const double* __restrict__ k, int f_kind, const double* __restrict__ f_arg, const int32_t* __restrict__ slot,
    const double* __restrict__ w, const double* __restrict__ r, double* __restrict__ gk, float4* __restrict__ pk,
    const float4* __restrict__ tab, int* __restrict__ err) {
  constexpr int D1 = D + 1;
  extern __shared__ __align__(16) unsigned char sm[];
  VtxDF<D>* xs = reinterpret_cast<VtxDF<D>*>(sm);
  const int tile = blockIdx.x;
  const int v0 = __ldg(voff + tile), nv = __ldg(voff + tile + 1) - v0;
  const int64_t j = (int64_t)tile * TE + threadIdx.x;
  const bool act = j < NT;
  int t = 0, lv[D1], qi[D1];
  if (act) {
    t = __ldg(elist + j);
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      lv[i] = __ldg(lelem + (int64_t)i * NT + j);
      qi[i] = __ldg(ipos + (int64_t)i * NT + j);
    }
  }
  for (int v = threadIdx.x; v < nv; v += TE) {
    const int R = __ldg(vlist + v0 + v);
    VtxDF<D> x;
    stage_vertex<D>(x, node + (size_t)R * D);
    xs[v] = x;
  }
  __syncthreads();
  if (!act) return;
  df2 Ws[D1][D1], rv[D1];
  int st = FEM_OK;
  if (w) sym_weights<D>(slot, NT, t, w, Ws, st);
  if (r) {
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      const double ri = __ldg(r + __ldg(vlist + v0 + lv[i]));
      if (!input_in_range(ri)) st = worst(st, FEM_ERR_RANGE);
      rv[i] = df_from_double_fast(ri);
    }
  }
  const df2 kt = k ? coef_df(__ldg(k + t), st) : df2{1.0f, 0.0f};
  const VtxDF<D>* V[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) V[i] = &xs[lv[i]];
  df2 out[D1][D], gkv;
  st = worst(st, element_adjoint<D>(reinterpret_cast<const VtxDF<D>* const(&)[D1]>(V), t, kt, w != nullptr, Ws,
                                    r != nullptr, rv, f_kind, f_arg, tab, out, gkv));
  if (st != FEM_OK) report(err, st);
  if (gk) gk[t] = df_to_double(gkv);
#pragma unroll
  for (int m = 0; m < D1; ++m) {
    float4* dst = pk + 2 * (size_t)qi[m];
    const float4 p0 = make_float4(out[m][0].h, out[m][0].l, out[m][1].h, out[m][1].l);
    if constexpr (D == 3) store_packet32(dst, p0, make_float4(out[m][2].h, out[m][2].l, 0.0f, 0.0f));
    else dst[0] = p0;
  }
}

// per vertex: its packets are contiguous, in ascending element order
template <int D>
__global__ void __launch_bounds__(256) k_backward_gather_tiles(const int32_t* __restrict__ inc_ptr, int64_t N,
                                                               const float4* __restrict__ pk,
                                                               double* __restrict__ gnode) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  df2 acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = df2{0.0f, 0.0f};
  const int q1 = __ldg(inc_ptr + v + 1);
  for (int q = __ldg(inc_ptr + v); q < q1; ++q) {
    float4 a, b;
    if constexpr (D == 3) load_packet32<false>(pk + 2 * (size_t)q, a, b);
    else a = __ldg(pk + 2 * (size_t)q);
    acc[0] = df_acc(acc[0], df2{a.x, a.y});
    acc[1] = df_acc(acc[1], df2{a.z, a.w});
    if constexpr (D == 3) acc[2] = df_acc(acc[2], df2{b.x, b.y});
  }
#pragma unroll
  for (int c = 0; c < D; ++c) gnode[v * D + c] = df_to_double(acc[c]);
}

template <int D>
__global__ void __launch_bounds__(256) k_backward_gather_df(const int32_t* __restrict__ inc_ptr,
                                                            const int32_t* __restrict__ inc, int N, int NT,
                                                            const float2* __restrict__ scratch, double* __restrict__ gnode) {
  constexpr int D1 = D + 1;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  df2 acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = df2{0.0f, 0.0f};
  for (int q = inc_ptr[v]; q < inc_ptr[v + 1]; ++q) {
    const int p = inc[q];
    const int t = p / D1, m = p - t * D1;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float2 x = __ldg(scratch + (size_t)(m * D + c) * NT + t);
      acc[c] = df_acc(acc[c], df2{x.x, x.y});
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) gnode[(size_t)v * D + c] = df_to_double(acc[c]);
}

}  // namespace

int assemble_backward(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                         const double* w, const double* r, double* gnode, double* gk, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  if (!P->scratch) return set_error(FEM_ERR_STATE, "pattern has no scratch for the backward gather");
  const float4* tab = sincos_table_device();
  if (!tab) return set_error(FEM_ERR_CUDA, "sin/cos table unavailable");
  const int NT = (int)P->NT, N = (int)P->N;
  if (NT == 0) {
    if (gnode && N > 0) FEM_CUDA(cudaMemsetAsync(gnode, 0, sizeof(double) * N * P->d, s));
    return FEM_OK;
  }
  const TilePlan& T = P->tile;
  if (T.ok && T.pk && (T.TE == 128 || T.TE == 256) && (reinterpret_cast<uintptr_t>(T.pk) & 31) == 0) {
    const int smem = ((T.max_v * vtx_bytes(P->d)) + 15) / 16 * 16;
    const int g2 = (N + 255) / 256;
#define FEM_BWD_TILES(DD, TT)                                                                                      \
  FEM_LAUNCH((k_backward_tiles<DD, TT>), T.ntiles, TT, smem, s, P->NT, T.elist, T.lelem, T.voff, T.vlist, T.ipos, \
             node, k, f_kind, f_arg, P->slot, w, r, gk, T.pk, tab, err)
    if (P->d == 2) {
      if (T.TE == 128) FEM_BWD_TILES(2, 128);
      else FEM_BWD_TILES(2, 256);
      if (gnode) FEM_LAUNCH(k_backward_gather_tiles<2>, g2, 256, 0, s, P->inc_ptr, P->N, T.pk, gnode);
    } else {
      if (T.TE == 128) FEM_BWD_TILES(3, 128);
      else FEM_BWD_TILES(3, 256);
      if (gnode) FEM_LAUNCH(k_backward_gather_tiles<3>, g2, 256, 0, s, P->inc_ptr, P->N, T.pk, gnode);
    }
#undef FEM_BWD_TILES
    return FEM_OK;
  }
  float2* scr = reinterpret_cast<float2*>(P->scratch);
  const int g1 = (NT + 127) / 128, g2 = (N + 255) / 256;
  if (P->d == 2) {
    FEM_LAUNCH(k_backward_df<2>, g1, 128, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, w, r, gk, scr, tab, err);
    if (gnode) FEM_LAUNCH(k_backward_gather_df<2>, g2, 256, 0, s, P->inc_ptr, P->inc, N, NT, scr, gnode);
  } else {
    FEM_LAUNCH(k_backward_df<3>, g1, 128, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, w, r, gk, scr, tab, err);
    if (gnode) FEM_LAUNCH(k_backward_gather_df<3>, g2, 256, 0, s, P->inc_ptr, P->inc, N, NT, scr, gnode);
  }
  return FEM_OK;
}

}  // namespace fem
