/*
 * CPU oracle for P1 finite-element assembly of the Poisson problem (L. Chen, "Programming of Finite
 * Element Methods in MATLAB", arXiv:1804.05156).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously correct reference that the CUDA
 * library is checked against. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is IEEE double, compiled without floating-point contraction (-ffp-contract=off), in
 * plain loops, in the order the paper's definitions give. Indices are 0-based (the paper is 1-based).
 *
 *   ora_sparse        the `sparse(i,j,s,m,n)` operation of Sec. 2.2: COO triples in any order with
 *                     duplicates summed, returned as CSR (rows ascending, columns ascending). Summation
 *                     order: stable, i.e. the order the triples are given.
 *   ora_triples       the COO triples (ii, jj, sA) of the vectorised assembly of Sec. 3.1.3 (eq. for
 *                     a_ij^tau below eq. (dlambda); 2-D edge vectors and area; 3-D face normals and
 *                     signed volume), times a per-element coefficient k, in the element-by-element
 *                     order of `assemblingsparse` (Sec. 3.1.2): t ascending, then local i, then j.
 *                     A row mask keeps only triples whose row is selected (for sampled rows).
 *   ora_slots         position of each (elem[t,i], elem[t,j]) pair inside a CSR pattern (binary search).
 *   ora_measure       signed area/volume of every element (Sec. 3.1.3).
 *   ora_rhs           load vector of Sec. 3.2: 2-D three-edge-midpoint rule; 3-D four-point rule (see
 *                     its comment for the reading), accumulated per vertex as `accumarray` does.
 *   ora_boundary      Dirichlet node mask of Sec. 1.2/3.3 from bdFlag == 1, or, with no bdFlag, from
 *                     the sides that belong to exactly one element ("whole boundary").
 *   ora_dirichlet     Sec. 3.3: u = g_D on boundary nodes, b <- b - A*u, freeNode, and the equivalent
 *                     symmetric eliminated system (boundary rows -> identity rows, boundary columns of
 *                     free rows -> 0, b[bd] = g_D).
 *   ora_backward      gradients of L = sum_s w_s A_s + sum_i r_i b_i with respect to node coordinates
 *                     and element coefficients, by the closed-form adjoint derived from eq. (dlambda):
 *                     d|tau|/dx_m = |tau| g_m and dg_i/dx_m = -g_m g_i^T (g_i = grad lambda_i).
 *   ora_local_affine  Sec. 3.1.1 local stiffness by the affine map to the reference triangle
 *                     (a second, independent formula used only to pin the first).
 *   ora_boundary_terms  Neumann (bdFlag 2) and Robin (bdFlag 3) sides: the one-point side rule of the
 *                     paper's Neumann code (Sec. 3.3) for the load, and the side mass matrix for Robin.
 *   ora_side_points   the quadrature point (midpoint / centroid) of every side.
 *   ora_mean_shift    the pure-Neumann compatibility fix b - mean(b) (Sec. 3.3).
 *   ora_zero_average  u - c with c the area-weighted mean of u (Sec. 3.3), the zero-average constraint.
 *   ora_operator_triples  triples of the mass matrix and of the anisotropic operator div(K grad u) on
 *                     the same element loop (grad lambda from eq. (dlambda)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_ERR_ARG -1
#define ORA_ERR_INDEX -2
#define ORA_ERR_DEGENERATE -3
#define ORA_ERR_OOM -5

/* ------------------------------------------------------------------------------------------------
 * Element geometry, Sec. 3.1.3.
 *
 * 2-D: edge vectors ve_1 = x3 - x2, ve_2 = x1 - x3, ve_3 = x2 - x1 (edge i is opposite vertex i),
 *      area = |(-ve_3.x * ve_2.y + ve_3.y * ve_2.x)| / 2, and n_i . n_j = ve_i . ve_j because the
 *      scaled normal is the edge vector rotated by 90 degrees. With this orientation of ve_i the
 *      rotation v -> (-v.y, v.x) gives the inward normal, so grad lambda_i = (-ve_i.y, ve_i.x)/(2|tau|).
 * 3-D: face i opposite vertex i, with vertex lists [2 4 3], [1 3 4], [1 4 2], [1 2 3] (1-based);
 *      n_i = (x_f2 - x_f1) x (x_f3 - x_f1) is the inward normal with |n_i| = 2 |F_i|;
 *      volume = ((x2 - x1) x (x3 - x1)) . (x4 - x1) / 6, signed (positive for right-handed elements).
 * a_ij^tau = n_i . n_j / (d!^2 |tau|), eq. below (dlambda).
 * ------------------------------------------------------------------------------------------------ */

static void sub2(const double* a, const double* b, double* out) { out[0] = a[0] - b[0]; out[1] = a[1] - b[1]; }
static void sub3(const double* a, const double* b, double* out) {
  out[0] = a[0] - b[0]; out[1] = a[1] - b[1]; out[2] = a[2] - b[2];
}
static void cross3(const double* u, const double* v, double* out) {
  out[0] = u[1] * v[2] - u[2] * v[1];
  out[1] = u[2] * v[0] - u[0] * v[2];
  out[2] = u[0] * v[1] - u[1] * v[0];
}
static double dot(const double* u, const double* v, int d) {
  double s = 0.0;
  for (int m = 0; m < d; ++m) s = s + u[m] * v[m];
  return s;
}

static const int FACE3[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};  /* 0-based [2 4 3] ... */

/* Scaled normals n[i][*] (d components each) and the measure |tau| of element t.
 * 2-D returns the paper's abs() area; 3-D returns the signed volume. */
static double element_normals(int d, const double* node, const int32_t* e, double n[4][3]) {
  if (d == 2) {
    const double *x1 = node + 2 * (int64_t)e[0], *x2 = node + 2 * (int64_t)e[1], *x3 = node + 2 * (int64_t)e[2];
    double ve[3][2];
    sub2(x3, x2, ve[0]);
    sub2(x1, x3, ve[1]);
    sub2(x2, x1, ve[2]);
    for (int i = 0; i < 3; ++i) { n[i][0] = -ve[i][1]; n[i][1] = ve[i][0]; n[i][2] = 0.0; }
    return 0.5 * fabs(-ve[2][0] * ve[1][1] + ve[2][1] * ve[1][0]);
  } else {
    const double* x[4];
    for (int i = 0; i < 4; ++i) x[i] = node + 3 * (int64_t)e[i];
    for (int i = 0; i < 4; ++i) {
      double v12[3], v13[3];
      sub3(x[FACE3[i][1]], x[FACE3[i][0]], v12);
      sub3(x[FACE3[i][2]], x[FACE3[i][0]], v13);
      cross3(v12, v13, n[i]);
    }
    double v12[3], v13[3], v14[3], c[3];
    sub3(x[1], x[0], v12);
    sub3(x[2], x[0], v13);
    sub3(x[3], x[0], v14);
    cross3(v12, v13, c);
    return dot(c, v14, 3) / 6.0;
  }
}

/* a_ij^tau = k * (n_i . n_j / (d!^2 |tau|)) */
static double local_entry(int d, double n[4][3], double meas, double k, int i, int j) {
  double dd = (d == 2) ? 4.0 : 36.0;
  return k * (dot(n[i], n[j], d) / (dd * meas));
}

/* Magnitude bound of the rounding of that entry: k * sum_m |n|_im |n|_jm / (d!^2 |tau|), where |n|_im
 * is the magnitude of the terms that form n_im (2-D: |n_im| itself, an edge component; 3-D: the two
 * products of the cross product, |u_a v_b| + |u_b v_a|). For the diagonal the sum runs over
 * j != i, which also bounds the diagonal formed as minus the off-diagonal row sum (sum_j n_j = 0).
 * This is the scale the parity tolerance is relative to. */
static void normal_magnitudes(int d, const double* node, const int32_t* e, double nm[4][3]) {
  if (d == 2) {
    double n[4][3];
    element_normals(d, node, e, n);
    for (int i = 0; i < 3; ++i)
      for (int m = 0; m < 2; ++m) nm[i][m] = fabs(n[i][m]);
    return;
  }
  const double* x[4];
  for (int i = 0; i < 4; ++i) x[i] = node + 3 * (int64_t)e[i];
  for (int i = 0; i < 4; ++i) {
    double u[3], v[3];
    sub3(x[FACE3[i][1]], x[FACE3[i][0]], u);
    sub3(x[FACE3[i][2]], x[FACE3[i][0]], v);
    nm[i][0] = fabs(u[1] * v[2]) + fabs(u[2] * v[1]);
    nm[i][1] = fabs(u[2] * v[0]) + fabs(u[0] * v[2]);
    nm[i][2] = fabs(u[0] * v[1]) + fabs(u[1] * v[0]);
  }
}

static double local_scale(int d, double nm[4][3], double meas, double k, int i, int j) {
  double dd = (d == 2) ? 4.0 : 36.0, s = 0.0;
  if (i != j) {
    for (int m = 0; m < d; ++m) s = s + nm[i][m] * nm[j][m];
  } else {
    for (int q = 0; q <= d; ++q)
      if (q != i)
        for (int m = 0; m < d; ++m) s = s + nm[i][m] * nm[q][m];
  }
  return fabs(k) * (s / (dd * fabs(meas)));
}

int ora_measure(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, double* meas) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + (d + 1) * t;
    for (int i = 0; i <= d; ++i)
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
    double n[4][3];
    if (d == 2) {
      /* signed area, for the orientation check: (-ve3.x ve2.y + ve3.y ve2.x)/2 */
      const double *x1 = node + 2 * (int64_t)e[0], *x2 = node + 2 * (int64_t)e[1], *x3 = node + 2 * (int64_t)e[2];
      double ve2[2], ve3[2];
      sub2(x1, x3, ve2);
      sub2(x2, x1, ve3);
      meas[t] = 0.5 * (-ve3[0] * ve2[1] + ve3[1] * ve2[0]);
    } else {
      meas[t] = element_normals(d, node, e, n);
    }
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * sparse(i, j, s, m, n), Sec. 2.2: duplicates are summed; the result is stored as CSR. For a
 * symmetric matrix these arrays equal the CSC arrays MATLAB keeps internally (Sec. 2.1).
 * Entries whose sum is exactly zero are kept (structural pattern).
 * ------------------------------------------------------------------------------------------------ */
typedef struct { int64_t row, col, pos; } coo_key;

static int cmp_coo(const void* a, const void* b) {
  const coo_key *x = (const coo_key*)a, *y = (const coo_key*)b;
  if (x->row != y->row) return x->row < y->row ? -1 : 1;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;  /* stable: keep the given order */
  return 0;
}

/* Returns nnz (>= 0) or an error code. row_ptr has m+1 entries; col/val have room for ntrip.
 * s2 (optional, may be NULL) is a second value array summed the same way into val2. */
int64_t ora_sparse(int64_t m, int64_t n, int64_t ntrip, const int64_t* I, const int64_t* J, const double* S,
                   const double* S2, int64_t* row_ptr, int64_t* col, double* val, double* val2) {
  coo_key* k = (coo_key*)malloc(sizeof(coo_key) * (ntrip > 0 ? ntrip : 1));
  if (!k) return ORA_ERR_OOM;
  for (int64_t p = 0; p < ntrip; ++p) {
    if (I[p] < 0 || I[p] >= m || J[p] < 0 || J[p] >= n) { free(k); return ORA_ERR_INDEX; }
    k[p].row = I[p]; k[p].col = J[p]; k[p].pos = p;
  }
  qsort(k, (size_t)ntrip, sizeof(coo_key), cmp_coo);
  int64_t nnz = 0;
  for (int64_t r = 0; r <= m; ++r) row_ptr[r] = 0;
  for (int64_t p = 0; p < ntrip; ++p) {
    int fresh = (p == 0) || k[p].row != k[p - 1].row || k[p].col != k[p - 1].col;
    if (fresh) {
      col[nnz] = k[p].col;
      val[nnz] = 0.0;
      if (val2) val2[nnz] = 0.0;
      row_ptr[k[p].row + 1] += 1;
      nnz += 1;
    }
    val[nnz - 1] = val[nnz - 1] + S[k[p].pos];
    if (val2) val2[nnz - 1] = val2[nnz - 1] + S2[k[p].pos];
  }
  for (int64_t r = 0; r < m; ++r) row_ptr[r + 1] += row_ptr[r];
  free(k);
  return nnz;
}

/* ------------------------------------------------------------------------------------------------
 * COO triples of the stiffness matrix, Sec. 3.1: for t = 0..NT-1, i = 0..d, j = 0..d:
 *   ii = elem[t,i], jj = elem[t,j], sA = k_t * n_i.n_j / (d!^2 |tau|), sScale = magnitude bound.
 * row_mask (optional): keep only triples whose row has row_mask[row] != 0.
 * Returns the number of triples written, or an error code. Degenerate or inverted elements
 * (measure <= 0 in 3-D, area == 0 in 2-D) are an error, as orientation is assumed (Sec. 1.1).
 * ------------------------------------------------------------------------------------------------ */
int64_t ora_triples(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, const double* k,
                    const uint8_t* row_mask, int64_t* I, int64_t* J, double* S, double* Sscale) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  int64_t q = 0;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + (d + 1) * t;
    for (int i = 0; i <= d; ++i)
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
    int any = 1;
    if (row_mask) {
      any = 0;
      for (int i = 0; i <= d; ++i) any |= row_mask[e[i]] != 0;
    }
    if (!any) continue;
    double n[4][3];
    double meas = element_normals(d, node, e, n);
    if (!(meas > 0.0)) return ORA_ERR_DEGENERATE;
    double kt = k ? k[t] : 1.0;
    double nm[4][3];
    if (Sscale) normal_magnitudes(d, node, e, nm);
    for (int i = 0; i <= d; ++i) {
      if (row_mask && !row_mask[e[i]]) continue;
      for (int j = 0; j <= d; ++j) {
        I[q] = e[i];
        J[q] = e[j];
        S[q] = local_entry(d, n, meas, kt, i, j);
        if (Sscale) Sscale[q] = local_scale(d, nm, meas, kt, i, j);
        q += 1;
      }
    }
  }
  return q;
}

/* slot[t*(d+1)^2 + i*(d+1) + j] = position of (elem[t,i], elem[t,j]) in the CSR pattern. */
int ora_slots(int d, int64_t N, int64_t NT, const int32_t* elem, const int64_t* row_ptr, const int64_t* col,
              int64_t* slot) {
  int d1 = d + 1;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + d1 * t;
    for (int i = 0; i < d1; ++i) {
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
      for (int j = 0; j < d1; ++j) {
        int64_t lo = row_ptr[e[i]], hi = row_ptr[e[i] + 1] - 1, found = -1;
        while (lo <= hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (col[mid] == e[j]) { found = mid; break; }
          if (col[mid] < e[j]) lo = mid + 1; else hi = mid - 1;
        }
        if (found < 0) return ORA_ERR_INDEX;
        slot[(t * d1 + i) * d1 + j] = found;
      }
    }
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Right-hand side, Sec. 3.2 and Sec. 4.
 *
 * f kinds: 0 constant (farg[0], or 1 if farg is NULL); 1 product of sin(pi x_m) over the coordinates;
 * 2 caller values at the quadrature points, farg[t*nq + q].
 * sin(pi x) is evaluated as +-sin(pi r) with x = j + r, j = round(x), |r| <= 1/2 (x - j is exact), so
 * the rounding of pi*x near integers does not blow up the relative error.
 *
 * 2-D (Sec. 3.2): point q is the midpoint m_q of the edge opposite vertex q; the rule is
 *   b_i += |tau| * (f(m_{i+1}) + f(m_{i+2})) / 6   (cyclic), i.e. weights 1/3 and lambda_i(m_q) = 1/2
 *   for q != i, 0 for q == i; it is exact for quadratics (Sec. 4).
 * 3-D: the paper names a "4-points rule" without printing it. Reading: the symmetric degree-2 rule
 *   with barycentric points (a, b, b, b) and its permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20,
 *   weights 1/4; point q has the weight a on vertex q. b_i += |tau| * sum_q f(x_q) lambda_i(x_q) / 4.
 * ------------------------------------------------------------------------------------------------ */
static double sinpi_ref(double x) {
  double j = nearbyint(x);
  double r = x - j;
  double s = sin(M_PI * r);
  return (fmod(fabs(j), 2.0) == 1.0) ? -s : s;
}

/* sin(pi x_m) and cos(pi x_m) at the point x = sum_i lam[i] x_i of element e (coordinate m). The vertices
 * are first moved by the integer k nearest to the element's first vertex (exact differences), the point is
 * formed from the moved vertices, and sin(pi (y + k)) = (-1)^k sin(pi y): next to an integer the point keeps
 * its relative accuracy, which forming x first (a sum near the integer, rounded to the integer's ulp) would
 * lose. */
static void sincos_at(int d, const double* node, const int32_t* e, const double* lam, int m, double* s, double* c) {
  double k0 = nearbyint(node[d * (int64_t)e[0] + m]);
  double y = 0.0;
  for (int i = 0; i <= d; ++i) y = y + lam[i] * (node[d * (int64_t)e[i] + m] - k0);
  double j = nearbyint(y);
  double r = y - j;
  int odd = (fmod(fabs(k0), 2.0) == 1.0) != (fmod(fabs(j), 2.0) == 1.0);
  *s = odd ? -sin(M_PI * r) : sin(M_PI * r);
  *c = odd ? -cos(M_PI * r) : cos(M_PI * r);
}

/* f at quadrature point q of element t, barycentric weights lam (kind 1 through sincos_at) */
static double f_eval(int kind, int d, const double* node, const int32_t* e, const double* lam, const double* farg,
                     int64_t t, int q, int nq) {
  if (kind == 0) return farg ? farg[0] : 1.0;
  if (kind == 1) {
    double v = 1.0;
    for (int m = 0; m < d; ++m) {
      double sm, cm;
      sincos_at(d, node, e, lam, m, &sm, &cm);
      v = v * sm;
    }
    return v;
  }
  return farg[t * nq + q];
}

int ora_quad_points(int d, const double* node, const int32_t* e, double pts[4][3], double lam[4][4]) {
  if (d == 2) {
    for (int q = 0; q < 3; ++q) {
      const double* a = node + 2 * (int64_t)e[(q + 1) % 3];
      const double* b = node + 2 * (int64_t)e[(q + 2) % 3];
      for (int m = 0; m < 2; ++m) pts[q][m] = (a[m] + b[m]) / 2.0;
      for (int i = 0; i < 3; ++i) lam[q][i] = (i == q) ? 0.0 : 0.5;
    }
    return 3;
  }
  double s5 = sqrt(5.0);
  double alpha = (5.0 + 3.0 * s5) / 20.0, beta = (5.0 - s5) / 20.0;
  for (int q = 0; q < 4; ++q) {
    for (int i = 0; i < 4; ++i) lam[q][i] = (i == q) ? alpha : beta;
    for (int m = 0; m < 3; ++m) {
      double s = 0.0;
      for (int i = 0; i < 4; ++i) s = s + lam[q][i] * node[3 * (int64_t)e[i] + m];
      pts[q][m] = s;
    }
  }
  return 4;
}

int ora_rhs(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, int fkind, const double* farg,
            const uint8_t* row_mask, double* b) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  if (fkind == 2 && !farg) return ORA_ERR_ARG;
  for (int64_t r = 0; r < N; ++r) b[r] = 0.0;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + (d + 1) * t;
    for (int i = 0; i <= d; ++i)
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
    if (row_mask) {
      int any = 0;
      for (int i = 0; i <= d; ++i) any |= row_mask[e[i]] != 0;
      if (!any) continue;
    }
    double n[4][3];
    double meas = element_normals(d, node, e, n);
    if (!(meas > 0.0)) return ORA_ERR_DEGENERATE;
    double pts[4][3], lam[4][4];
    int nq = ora_quad_points(d, node, e, pts, lam);
    double fq[4];
    for (int q = 0; q < nq; ++q) fq[q] = f_eval(fkind, d, node, e, lam[q], farg, t, q, nq);
    for (int i = 0; i <= d; ++i) {
      double bt;
      if (d == 2) {
        bt = meas * (fq[(i + 1) % 3] + fq[(i + 2) % 3]) / 6.0;
      } else {
        double s = 0.0;
        for (int q = 0; q < 4; ++q) s = s + fq[q] * lam[q][i];
        bt = meas * s / 4.0;
      }
      b[e[i]] = b[e[i]] + bt;
    }
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Boundary nodes, Sec. 1.2 and Sec. 3.3. Side i of element t is opposite vertex i: 2-D side i is
 * elem(t, [i+1, i+2]) (cyclic, the `totalEdge` order of Sec. 1.2); 3-D side i is the face with the
 * vertex list of FACE3[i]. With bdFlag, a side is Dirichlet when bdFlag[t,i] == 1. Without it
 * (reading of "Dirichlet on the whole boundary"), a side is a boundary side when no other element
 * has the same vertex set. isBd[v] = 1 for every vertex of a Dirichlet side.
 * ------------------------------------------------------------------------------------------------ */
typedef struct { int32_t v[3]; int64_t id; } side_key;

static int cmp_side(const void* a, const void* b) {
  const side_key *x = (const side_key*)a, *y = (const side_key*)b;
  for (int m = 0; m < 3; ++m)
    if (x->v[m] != y->v[m]) return x->v[m] < y->v[m] ? -1 : 1;
  return 0;
}

static void side_vertices(int d, const int32_t* e, int i, int32_t out[3]) {
  if (d == 2) {
    out[0] = e[(i + 1) % 3]; out[1] = e[(i + 2) % 3]; out[2] = -1;
  } else {
    for (int m = 0; m < 3; ++m) out[m] = e[FACE3[i][m]];
  }
}

int ora_boundary(int d, int64_t N, int64_t NT, const int32_t* elem, const int8_t* bdflag, uint8_t* is_bd) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  int d1 = d + 1, nv = d;
  for (int64_t v = 0; v < N; ++v) is_bd[v] = 0;
  for (int64_t p = 0; p < NT * d1; ++p)
    if (elem[p] < 0 || elem[p] >= N) return ORA_ERR_INDEX;
  if (bdflag) {
    for (int64_t t = 0; t < NT; ++t)
      for (int i = 0; i < d1; ++i)
        if (bdflag[t * d1 + i] == 1) {
          int32_t sv[3];
          side_vertices(d, elem + d1 * t, i, sv);
          for (int m = 0; m < nv; ++m) is_bd[sv[m]] = 1;
        }
    return ORA_OK;
  }
  int64_t ns = NT * d1;
  side_key* s = (side_key*)malloc(sizeof(side_key) * (ns > 0 ? ns : 1));
  if (!s) return ORA_ERR_OOM;
  for (int64_t t = 0; t < NT; ++t)
    for (int i = 0; i < d1; ++i) {
      side_key* k = s + t * d1 + i;
      side_vertices(d, elem + d1 * t, i, k->v);
      /* sort the vertex list so the key does not depend on orientation */
      for (int a = 0; a < nv; ++a)
        for (int b2 = a + 1; b2 < nv; ++b2)
          if (k->v[b2] < k->v[a]) { int32_t tmp = k->v[a]; k->v[a] = k->v[b2]; k->v[b2] = tmp; }
      k->id = t * d1 + i;
    }
  qsort(s, (size_t)ns, sizeof(side_key), cmp_side);
  for (int64_t p = 0; p < ns;) {
    int64_t q = p + 1;
    while (q < ns && cmp_side(s + p, s + q) == 0) ++q;
    if (q - p == 1)
      for (int m = 0; m < nv; ++m) is_bd[s[p].v[m]] = 1;
    p = q;
  }
  free(s);
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Dirichlet boundary condition, Sec. 3.3.
 *   u = g_D on boundary nodes (0 when gD is NULL), 0 elsewhere;
 *   b <- b - A*u, where (A*u)_r is summed over the row's entries in ascending column order,
 *        s = s + val*u[col] starting from s = 0 (no fused multiply-add);
 *   freeNode = free nodes in ascending order (returned count in *n_free);
 *   eliminated system: boundary rows become identity rows, boundary columns of free rows become 0,
 *   b[bd] = g_D[bd].
 * ------------------------------------------------------------------------------------------------ */
int ora_dirichlet(int64_t N, const int64_t* row_ptr, const int64_t* col, const uint8_t* is_bd, const double* gD,
                  double* val, double* b, int64_t* free_node, int64_t* n_free) {
  double* u = (double*)malloc(sizeof(double) * (N > 0 ? N : 1));
  if (!u) return ORA_ERR_OOM;
  for (int64_t v = 0; v < N; ++v) u[v] = is_bd[v] ? (gD ? gD[v] : 0.0) : 0.0;
  for (int64_t r = 0; r < N; ++r) {
    double s = 0.0;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) s = s + val[p] * u[col[p]];
    b[r] = b[r] - s;
  }
  int64_t nf = 0;
  for (int64_t r = 0; r < N; ++r) {
    if (!is_bd[r]) free_node[nf++] = r;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      if (is_bd[r]) val[p] = (col[p] == r) ? 1.0 : 0.0;
      else if (is_bd[col[p]]) val[p] = 0.0;
    }
    if (is_bd[r]) b[r] = u[r];
  }
  *n_free = nf;
  free(u);
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Backward. L = sum_s w[s] A[s] + sum_i r[i] b[i].
 * Per element, g_i = grad lambda_i = n_i / (d! |tau|) (eq. (dlambda)), a^tau = k |tau| G G^T, and with
 * W_ij = w[slot(t,i,j)]:
 *   dL/dk_t    = |tau| sum_ij W_ij g_i.g_j
 *   dL_A/dx_m  = k |tau| [ S g_m - sum_ij W_ij ((g_m.g_j) g_i + (g_m.g_i) g_j) ],  S = sum_ij W_ij g_i.g_j
 *   dL_b/dx_m  = |tau| g_m sum_i r_i sum_q w_q f(x_q) lambda_i(q)
 *                + |tau| sum_i r_i sum_q w_q lambda_i(q) lambda_m(q) grad f(x_q)
 * where (w_q, lambda(q)) is the element's rule (2-D midpoints: w_q = 1/3; 3-D: w_q = 1/4).
 * grad f is available for kinds 0 (zero) and 1 (product of sin(pi x_m)); kind 2 has no coordinate
 * gradient through f (f values are inputs).
 * Node gradients are summed over incident elements in element order.
 * ------------------------------------------------------------------------------------------------ */
static void f_grad(int kind, int d, const double* node, const int32_t* e, const double* lam, double* g) {
  for (int m = 0; m < d; ++m) g[m] = 0.0;
  if (kind != 1) return;
  double sv[3], cv[3];
  for (int m = 0; m < d; ++m) sincos_at(d, node, e, lam, m, &sv[m], &cv[m]);
  for (int m = 0; m < d; ++m) {
    double v = 1.0;
    for (int q = 0; q < d; ++q) v = v * ((q == m) ? M_PI * cv[q] : sv[q]);
    g[m] = v;
  }
}

int ora_backward(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, const double* k,
                 int fkind, const double* farg, const int64_t* slot, const double* w, const double* r,
                 double* gnode, double* gk, double* gnode_mag, double* gk_mag) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  int d1 = d + 1;
  for (int64_t p = 0; p < N * d; ++p) gnode[p] = 0.0;
  if (gnode_mag)
    for (int64_t p = 0; p < N * d; ++p) gnode_mag[p] = 0.0;
  double dfact = (d == 2) ? 2.0 : 6.0;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + d1 * t;
    double n[4][3];
    double meas = element_normals(d, node, e, n);
    if (!(meas > 0.0)) return ORA_ERR_DEGENERATE;
    double g[4][3];
    for (int i = 0; i < d1; ++i)
      for (int m = 0; m < d; ++m) g[i][m] = n[i][m] / (dfact * meas);
    double kt = k ? k[t] : 1.0;
    double W[4][4];
    for (int i = 0; i < d1; ++i)
      for (int j = 0; j < d1; ++j) W[i][j] = w ? w[slot[(t * d1 + i) * d1 + j]] : 0.0;
    double S = 0.0;
    for (int i = 0; i < d1; ++i)
      for (int j = 0; j < d1; ++j) S = S + W[i][j] * dot(g[i], g[j], d);
    if (gk) gk[t] = meas * S;
    /* magnitudes: the same expressions with every term replaced by its absolute value and every basis
       gradient component by the magnitude of the terms that form it (normal_magnitudes) */
    double nm[4][3], ga[4][3], Sa = 0.0;
    normal_magnitudes(d, node, e, nm);
    for (int i = 0; i < d1; ++i)
      for (int m = 0; m < d; ++m) ga[i][m] = nm[i][m] / (dfact * meas);
    for (int i = 0; i < d1; ++i)
      for (int j = 0; j < d1; ++j) Sa = Sa + fabs(W[i][j]) * dot(ga[i], ga[j], d);
    if (gk_mag) gk_mag[t] = meas * Sa;
    /* rhs part */
    double pts[4][3], lam[4][4], fq[4], gf[4][3];
    int nq = ora_quad_points(d, node, e, pts, lam);
    double wq = (d == 2) ? 1.0 / 3.0 : 1.0 / 4.0;
    for (int q = 0; q < nq; ++q) {
      fq[q] = f_eval(fkind, d, node, e, lam[q], farg, t, q, nq);
      f_grad(fkind, d, node, e, lam[q], gf[q]);
    }
    double Rb = 0.0, Rba = 0.0;  /* sum_i r_i sum_q w_q f_q lambda_i(q), and its magnitude */
    if (r)
      for (int i = 0; i < d1; ++i) {
        double s = 0.0, sa = 0.0;
        for (int q = 0; q < nq; ++q) {
          s = s + wq * fq[q] * lam[q][i];
          sa = sa + wq * fabs(fq[q]) * lam[q][i];
        }
        Rb = Rb + r[e[i]] * s;
        Rba = Rba + fabs(r[e[i]]) * sa;
      }
    for (int mm = 0; mm < d1; ++mm) {
      double out[3], outa[3];
      for (int c = 0; c < d; ++c) {
        double acc = S * g[mm][c], acca = Sa * ga[mm][c];
        for (int i = 0; i < d1; ++i)
          for (int j = 0; j < d1; ++j) {
            acc = acc - W[i][j] * (dot(g[mm], g[j], d) * g[i][c] + dot(g[mm], g[i], d) * g[j][c]);
            acca = acca + fabs(W[i][j]) * (dot(ga[mm], ga[j], d) * ga[i][c] + dot(ga[mm], ga[i], d) * ga[j][c]);
          }
        out[c] = kt * meas * acc;
        outa[c] = fabs(kt) * meas * acca;
      }
      if (r) {
        for (int c = 0; c < d; ++c) {
          double s2 = 0.0, s2a = 0.0;
          for (int i = 0; i < d1; ++i)
            for (int q = 0; q < nq; ++q) {
              s2 = s2 + r[e[i]] * wq * lam[q][i] * lam[q][mm] * gf[q][c];
              s2a = s2a + fabs(r[e[i]]) * wq * lam[q][i] * lam[q][mm] * fabs(gf[q][c]);
            }
          out[c] = out[c] + meas * g[mm][c] * Rb + meas * s2;
          outa[c] = outa[c] + meas * ga[mm][c] * Rba + meas * s2a;
        }
      }
      for (int c = 0; c < d; ++c) gnode[(int64_t)e[mm] * d + c] = gnode[(int64_t)e[mm] * d + c] + out[c];
      if (gnode_mag)
        for (int c = 0; c < d; ++c)
          gnode_mag[(int64_t)e[mm] * d + c] = gnode_mag[(int64_t)e[mm] * d + c] + outa[c];
    }
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Sec. 3.1.1: local stiffness by the affine map F(x^) = B^T x^ + c of the reference triangle
 * (1,0), (0,1), (0,0): B = [x1 - x3; x2 - x3], reference gradients G = [(1,0), (0,1), (-1,-1)],
 * area = |det B|/2, At(i,j) = area * (B^{-1} G_i) . (B^{-1} G_j). Independent of the normal formula.
 * ------------------------------------------------------------------------------------------------ */
int ora_local_affine(const double* p /* 3x2 row-major */, double* At /* 3x3 */) {
  double B[2][2] = {{p[0] - p[4], p[1] - p[5]}, {p[2] - p[4], p[3] - p[5]}};
  double det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
  if (det == 0.0) return ORA_ERR_DEGENERATE;
  double area = 0.5 * fabs(det);
  double G[3][2] = {{1.0, 0.0}, {0.0, 1.0}, {-1.0, -1.0}};
  double y[3][2];
  for (int i = 0; i < 3; ++i) {
    /* solve B y = G_i by Cramer's rule */
    y[i][0] = (G[i][0] * B[1][1] - B[0][1] * G[i][1]) / det;
    y[i][1] = (B[0][0] * G[i][1] - G[i][0] * B[1][0]) / det;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) At[3 * i + j] = area * (y[i][0] * y[j][0] + y[i][1] * y[j][1]);
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Neumann and Robin sides ("Boundary conditions" and Sec. 3.3), and the pure-Neumann fixes.
 *
 * bdFlag(t, j) = 2 marks the side opposite vertex j of element t as Neumann, 3 as Robin
 * (du/dn + alpha u = g_R). The side's vertices are the element's other d vertices, taken in
 * ascending local index. Its measure |s|: 2-D the edge length sqrt(dx^2 + dy^2); 3-D the triangle
 * area |(p1 - p0) x (p2 - p0)| / 2.
 *   Neumann and Robin load: b[v] += (|s| * g) / d for each vertex v of the side, g the side's value
 *   (g_side[t][j], or g_const when g_side is NULL) at its midpoint (2-D, the paper's rule) or centroid
 *   (3-D reading: the same one-point rule on a triangle).
 *   Robin matrix: alpha * integral over the side of lambda_a lambda_b = alpha |s| (1 + delta_ab) / (d (d+1))
 *   added to the CSR entry (a, b) for every pair of the side's vertices (a 1-D or 2-D mass matrix).
 * Contributions are added element by element (t ascending), side by side (j ascending), vertex by
 * vertex (ascending local index), each as ((alpha * |s|) * w) / (d (d+1)) and (|s| * g) / d in that
 * order, without contraction.
 * ------------------------------------------------------------------------------------------------ */
static double side_measure(int d, const double* node, const int32_t* e, int j) {
  int32_t v[3];
  int c = 0;
  for (int k = 0; k <= d; ++k)
    if (k != j) v[c++] = e[k];
  if (d == 2) {
    const double dx = node[2 * v[1]] - node[2 * v[0]], dy = node[2 * v[1] + 1] - node[2 * v[0] + 1];
    return sqrt(dx * dx + dy * dy);
  }
  double u[3], w[3], x[3];
  for (int m = 0; m < 3; ++m) {
    u[m] = node[3 * v[1] + m] - node[3 * v[0] + m];
    w[m] = node[3 * v[2] + m] - node[3 * v[0] + m];
  }
  x[0] = u[1] * w[2] - u[2] * w[1];
  x[1] = u[2] * w[0] - u[0] * w[2];
  x[2] = u[0] * w[1] - u[1] * w[0];
  return sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) * 0.5;
}

static int64_t find_col(const int64_t* row_ptr, const int64_t* col, int64_t r, int64_t c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (col[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return (lo < row_ptr[r + 1] && col[lo] == c) ? lo : -1;
}

int ora_boundary_terms(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, const int8_t* bdflag,
                       const double* g_side, double g_const, double alpha, const int64_t* row_ptr,
                       const int64_t* col, double* val, double* b) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  const int d1 = d + 1;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + t * d1;
    for (int j = 0; j < d1; ++j) {
      const int flag = bdflag[t * d1 + j];
      if (flag != 2 && flag != 3) continue;
      const double m = side_measure(d, node, e, j);
      const double g = g_side ? g_side[t * d1 + j] : g_const;
      for (int a = 0; a < d1; ++a) {
        if (a == j) continue;
        if (e[a] < 0 || e[a] >= N) return ORA_ERR_INDEX;
        if (b) b[e[a]] = b[e[a]] + (m * g) / (double)d;
        if (flag == 3 && val) {
          for (int c = 0; c < d1; ++c) {
            if (c == j) continue;
            const int64_t pos = find_col(row_ptr, col, e[a], e[c]);
            if (pos < 0) return ORA_ERR_INDEX;
            const double wgt = (a == c) ? 2.0 : 1.0;
            val[pos] = val[pos] + ((alpha * m) * wgt) / (double)(d * d1);
          }
        }
      }
    }
  }
  return ORA_OK;
}

/* quadrature point of every side: the midpoint (2-D) or centroid (3-D) of its vertices, [NT][d+1][d] */
int ora_side_points(int d, int64_t NT, const double* node, const int32_t* elem, double* pts) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  const int d1 = d + 1;
  for (int64_t t = 0; t < NT; ++t)
    for (int j = 0; j < d1; ++j)
      for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int k = 0; k < d1; ++k)
          if (k != j) s = s + node[(int64_t)elem[t * d1 + k] * d + m];
        pts[(t * d1 + j) * d + m] = s / (double)d;
      }
  return ORA_OK;
}

/* pure Neumann: b <- b - mean(b), the mean summed in index order */
int ora_mean_shift(int64_t N, double* b) {
  if (N <= 0) return ORA_OK;
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) s = s + b[i];
  const double mean = s / (double)N;
  for (int64_t i = 0; i < N; ++i) b[i] = b[i] - mean;
  return ORA_OK;
}

/* zero average: c = sum_t mean(u(elem_t)) |tau_t| / sum_t |tau_t| (2-D |area|, 3-D signed volume), u <- u - c */
int ora_zero_average(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, double* u,
                     double* c_out) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  const int d1 = d + 1;
  double* meas = (double*)malloc(sizeof(double) * (NT > 0 ? NT : 1));
  if (!meas) return ORA_ERR_OOM;
  int rc = ora_measure(d, N, NT, node, elem, meas);
  if (rc) {
    free(meas);
    return rc;
  }
  double num = 0.0, den = 0.0;
  for (int64_t t = 0; t < NT; ++t) {
    double s = 0.0;
    for (int i = 0; i < d1; ++i) s = s + u[elem[t * d1 + i]];
    const double area = d == 2 ? fabs(meas[t]) : meas[t];
    num = num + (s / (double)d1) * area;
    den = den + area;
  }
  free(meas);
  const double c = den > 0.0 ? num / den : 0.0;
  for (int64_t v = 0; v < N; ++v) u[v] = u[v] - c;
  if (c_out) *c_out = c;
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------
 * Other second-order operators on the same element loop (the same triples order as ora_triples):
 *   op 1, mass:        m_ij^tau = c_t |tau| (1 + delta_ij) / ((d+1)(d+2)),  the exact integral of
 *                      c lambda_i lambda_j over tau (c_t = coef[t], 1 when coef is NULL);
 *   op 2, anisotropic: a_ij^tau = n_i^T K_t n_j / (d!^2 |tau|) = |tau| grad lambda_i^T K_t grad lambda_j
 *                      (eq. (dlambda)), K_t symmetric, given by its upper triangle in coef[t]:
 *                      2-D (xx, xy, yy), 3-D (xx, xy, xz, yy, yz, zz).
 * Sscale: the magnitude bound of each entry's rounding: |m_ij| for the mass matrix; for the anisotropic
 * matrix sum_ab |n|_ia |K_ab| |n|_jb / (d!^2 |tau|) with the normal magnitudes of normal_magnitudes (for
 * the diagonal summed over the other vertices q != i, which bounds minus the off-diagonal row sum too).
 * ------------------------------------------------------------------------------------------------ */
static void sym_tensor(int d, const double* c, double K[3][3]) {
  if (d == 2) {
    K[0][0] = c[0]; K[0][1] = c[1]; K[1][0] = c[1]; K[1][1] = c[2];
  } else {
    K[0][0] = c[0]; K[0][1] = c[1]; K[0][2] = c[2];
    K[1][0] = c[1]; K[1][1] = c[3]; K[1][2] = c[4];
    K[2][0] = c[2]; K[2][1] = c[4]; K[2][2] = c[5];
  }
}

static double quad_form(int d, const double* u, double K[3][3], const double* v) {
  double s = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) s = s + u[a] * (K[a][b] * v[b]);
  return s;
}

int64_t ora_operator_triples(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, int op,
                             const double* coef, int64_t* I, int64_t* J, double* S, double* Sscale) {
  if ((d != 2 && d != 3) || (op != 1 && op != 2) || (op == 2 && !coef)) return ORA_ERR_ARG;
  const int d1 = d + 1, nk = d * (d + 1) / 2;
  const double dd = (d == 2) ? 4.0 : 36.0;
  int64_t q = 0;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + d1 * t;
    for (int i = 0; i < d1; ++i)
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
    double n[4][3], nm[4][3], K[3][3], Ka[3][3];
    const double meas = element_normals(d, node, e, n);
    if (!(meas > 0.0)) return ORA_ERR_DEGENERATE;
    if (op == 2) {
      sym_tensor(d, coef + nk * t, K);
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Ka[a][b] = fabs(K[a][b]);
      normal_magnitudes(d, node, e, nm);
    }
    const double c = (op == 1 && coef) ? coef[t] : 1.0;
    for (int i = 0; i < d1; ++i)
      for (int j = 0; j < d1; ++j) {
        double v, sc;
        if (op == 1) {
          v = c * (meas * ((i == j ? 2.0 : 1.0) / (double)(d1 * (d + 2))));
          sc = fabs(v);
        } else {
          v = quad_form(d, n[i], K, n[j]) / (dd * meas);
          sc = 0.0;
          for (int qq = 0; qq < d1; ++qq) {
            if (i == j ? qq == i : qq != j) continue;
            sc = sc + quad_form(d, nm[i], Ka, nm[qq]);
          }
          sc = sc / (dd * meas);
        }
        I[q] = e[i];
        J[q] = e[j];
        S[q] = v;
        if (Sscale) Sscale[q] = sc;
        q += 1;
      }
  }
  return q;
}

/* ------------------------------------------------------------------------------------------------
 * Load vector with a given rule ("Numerical Quadrature"): b_i += |tau| sum_q w_q f(p_q) lambda_i(p_q),
 * p_q = sum_i bary[q][i] x_i, the rule's weights summing to 1. f kinds as ora_rhs (2: values
 * farg[t * nq + q]). The rule itself is built by the Python layer of the oracle.
 * ------------------------------------------------------------------------------------------------ */
int ora_rhs_rule(int d, int64_t N, int64_t NT, const double* node, const int32_t* elem, int nq, const double* bary,
                 const double* w, int fkind, const double* farg, double* b) {
  if (d != 2 && d != 3) return ORA_ERR_ARG;
  if (fkind == 2 && !farg) return ORA_ERR_ARG;
  const int d1 = d + 1;
  for (int64_t r = 0; r < N; ++r) b[r] = 0.0;
  for (int64_t t = 0; t < NT; ++t) {
    const int32_t* e = elem + d1 * t;
    for (int i = 0; i < d1; ++i)
      if (e[i] < 0 || e[i] >= N) return ORA_ERR_INDEX;
    double n[4][3];
    const double meas = element_normals(d, node, e, n);
    if (!(meas > 0.0)) return ORA_ERR_DEGENERATE;
    /* the points relative to an integer near the element (exact differences), so that sin(pi x) keeps
       its relative accuracy next to the integers: sin(pi (z + k)) = (-1)^k sin(pi z) */
    double k0[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < d; ++m) k0[m] = floor(node[(int64_t)e[0] * d + m] + 0.5);
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nq; ++q) {
      double p[3] = {0.0, 0.0, 0.0}, z[3] = {0.0, 0.0, 0.0};
      for (int m = 0; m < d; ++m)
        for (int i = 0; i < d1; ++i) {
          p[m] = p[m] + bary[q * d1 + i] * node[(int64_t)e[i] * d + m];
          z[m] = z[m] + bary[q * d1 + i] * (node[(int64_t)e[i] * d + m] - k0[m]);
        }
      double f;
      if (fkind == 1) {
        f = 1.0;
        for (int m = 0; m < d; ++m) f = f * (fmod(k0[m], 2.0) != 0.0 ? -1.0 : 1.0) * sinpi_ref(z[m]);
      } else {
        f = f_eval(fkind, d, node, e, bary + q * d1, farg, t, q, nq);
      }
      for (int i = 0; i < d1; ++i) c[i] = c[i] + (w[q] * f) * bary[q * d1 + i];
    }
    for (int i = 0; i < d1; ++i) b[e[i]] = b[e[i]] + meas * c[i];
  }
  return ORA_OK;
}
