// Load vector with quadrature rules of any order ("Numerical Quadrature": I_n(f) = sum_i f(p_i) w_i |tau|).
//
// Rules are conical products built here from their definitions: the simplex is the image of the unit
// square / cube under the collapsed map x = u (1 - v), y = v (2-D) and x = u (1 - v)(1 - w), y = v (1 - w),
// z = w (3-D), whose Jacobian (1 - v) (1 - w)^2 is absorbed into Gauss-Jacobi rules in v and w (weights
// (1 - v)^1, (1 - w)^2) next to a Gauss-Legendre rule in u. n points per direction give n^d points, exact
// for polynomials of total degree 2n - 1. Nodes are found by Newton's method on the three-term
// recurrence of the Jacobi polynomials, with deflation by the roots already found; weights follow from
// the derivative at the node and are normalised to the weight function's integral.
//
// Per element (one thread each, the caller's order): the points in float-float from the exact coordinate
// splits, f there (constant, the sine product, or the caller's values), the d+1 contributions
// |tau| sum_q w_q f(x_q) lambda_i(x_q) into the pattern's scratch; then each vertex sums its
// contributions over its incidence list in ascending element order (deterministic) and rounds once.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "element_df.cuh"

namespace fem {

const float4* sincos_table_device();  // values_blocked.cu

namespace {

// P_n^{(a,0)}(t) and its derivative, by the three-term recurrence
void jacobi(int n, double a, double t, double* p, double* dp) {
  double p0 = 1.0, p1 = 0.5 * (a + (a + 2.0) * t);
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double c = 2.0 * k + a;
    const double a1 = 2.0 * k * (k + a) * (c - 2.0);
    const double a2 = (c - 1.0) * (c * (c - 2.0) * t + a * a);
    const double a3 = 2.0 * (k + a - 1.0) * (k - 1.0) * c;
    const double p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  // (2n + a)(1 - t^2) P_n' = n (a - (2n + a) t) P_n + 2 (n + a) n P_{n-1}
  const double c = 2.0 * n + a;
  *dp = (n * (a - c * t) * p1 + 2.0 * (n + a) * n * p0) / (c * (1.0 - t * t));
}

// Gauss-Jacobi rule on [0, 1] for the weight (1 - v)^a: nodes and weights summing to 1 / (a + 1)
void gauss_jacobi01(int n, int a, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> t(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));  // a start near the i-th root
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      jacobi(n, a, z, &p, &dp);
      double s = 0.0;  // deflation by the roots already found
      for (int j = 0; j < i; ++j) s += 1.0 / (z - t[j]);
      const double dz = p / (dp - s * p);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    t[i] = z;
  }
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  double sum = 0.0;
  for (int i = 0; i < n; ++i) {
    double p, dp;
    jacobi(n, a, t[i], &p, &dp);
    w[i] = 1.0 / ((1.0 - t[i] * t[i]) * dp * dp);
    x[i] = 0.5 * (1.0 + t[i]);
    sum += w[i];
  }
  for (int i = 0; i < n; ++i) w[i] *= (1.0 / (a + 1.0)) / sum;
}

struct Rule {
  std::vector<double> bary, w;  // [nq][d+1], [nq]; weights sum to 1
};

std::mutex g_rule_mu;
std::map<int, Rule> g_rules;  // key d * 64 + n

const Rule& rule_for(int d, int n) {
  std::lock_guard<std::mutex> lk(g_rule_mu);
  auto it = g_rules.find(d * 64 + n);
  if (it != g_rules.end()) return it->second;
  std::vector<double> xu, wu, xv, wv, xw, ww;
  gauss_jacobi01(n, 0, xu, wu);
  gauss_jacobi01(n, 1, xv, wv);
  Rule r;
  if (d == 2) {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        const double x = xu[a] * (1.0 - xv[b]), y = xv[b];
        r.bary.insert(r.bary.end(), {1.0 - x - y, x, y});
        r.w.push_back(2.0 * wu[a] * wv[b]);  // the reference triangle's area is 1/2
      }
  } else {
    gauss_jacobi01(n, 2, xw, ww);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c) {
          const double x = xu[a] * (1.0 - xv[b]) * (1.0 - xw[c]), y = xv[b] * (1.0 - xw[c]), z = xw[c];
          r.bary.insert(r.bary.end(), {1.0 - x - y - z, x, y, z});
          r.w.push_back(6.0 * wu[a] * wv[b] * ww[c]);  // the reference tetrahedron's volume is 1/6
        }
  }
  return g_rules.emplace(d * 64 + n, std::move(r)).first->second;
}

template <int D>
__global__ void __launch_bounds__(128) k_rhs_rule(int64_t NT, const int32_t* __restrict__ elem,
                                                  const double* __restrict__ node, int nq,
                                                  const double* __restrict__ rule, int f_kind,
                                                  const double* __restrict__ f_arg, const float4* __restrict__ tab,
                                                  float2* __restrict__ contrib, int* __restrict__ err) {
  constexpr int D1 = D + 1;
  extern __shared__ __align__(16) unsigned char sm[];
  df2* lam = reinterpret_cast<df2*>(sm);  // [nq][D1] barycentric coordinates, then [nq] weights
  df2* wq = lam + nq * D1;
  for (int x = threadIdx.x; x < nq * (D1 + 1); x += blockDim.x) lam[x] = df_from_double(rule[x]);
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NT) return;
  VtxDF<D> X[D1];
  const VtxDF<D>* V[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) {
    stage_vertex<D>(X[i], node + (size_t)__ldg(elem + t * D1 + i) * D);
    V[i] = &X[i];
  }
  df2 n[D1][D], dm;
  const int s = element_normals_df<D>(reinterpret_cast<const VtxDF<D>* const(&)[D1]>(V), n, dm);  // d! |tau| 2^-ds
  int st;
  if constexpr (D == 3) st = tet_status(reinterpret_cast<const VtxDF<3>* const(&)[4]>(V), dm);
  else st = (dm.h > 0.0f && dm.h < INFINITY) ? FEM_OK : FEM_ERR_DEGENERATE;
  if (!scale_in_range(D * s)) st = worst(st, FEM_ERR_RANGE);
  const df2 meas = df_ldexp((D == 2) ? df_scale(dm, 0.5f) : df_mul(dm, df2{0.1666666716337204f, -4.9670538793e-09f}),
                            scale_in_range(D * s) ? D * s : 0);
  // coordinates shifted by an integer near the element (one FP64 subtraction each), so that sin(pi x)
  // keeps its relative accuracy next to integers
  df2 y[D1][D];
  float sgn = 1.0f;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    if constexpr (D == 2) {
      const float nn = rintf(lead_float(X[0].x[m]));
      if (int_parity(nn)) sgn = -sgn;
      const double nd = f2d_bits(nn);
#pragma unroll
      for (int i = 0; i < D1; ++i) y[i][m] = df_from_double_shift(__dsub_rn(X[i].x[m], nd), 0);
    } else {
      const float nn = rintf(X[0].x[m].a);
      if (int_parity(nn)) sgn = -sgn;
#pragma unroll
      for (int i = 0; i < D1; ++i)
        y[i][m] = df_add(two_sum(X[i].x[m].a, -nn), fast_two_sum(X[i].x[m].b, X[i].x[m].c));
    }
  }
  const df2 fc = (f_kind == FEM_F_CONST && f_arg) ? coef_df(__ldg(f_arg), st) : df2{1.0f, 0.0f};
  df2 c[D1];
#pragma unroll
  for (int i = 0; i < D1; ++i) c[i] = df2{0.0f, 0.0f};
  float wfm = 0.0f;  // the largest |w_q f_q|
  for (int q = 0; q < nq; ++q) {
    const df2* lq = lam + q * D1;
    df2 f;
    if (f_kind == FEM_F_SINPROD) {
      f = df2{sgn, 0.0f};
#pragma unroll
      for (int m = 0; m < D; ++m) {
        df2 xm = df_mul(lq[0], y[0][m]);
#pragma unroll
        for (int i = 1; i < D1; ++i) xm = df_add(xm, df_mul(lq[i], y[i][m]));
        f = df_mul(f, df_sinpi(xm, tab));
      }
    } else if (f_kind == FEM_F_QPVALUES) {
      f = coef_df(__ldg(f_arg + t * nq + q), st);
    } else {
      f = fc;
    }
    const df2 wf = df_mul(wq[q], f);
    wfm = fmaxf(wfm, fabsf(wf.h));
#pragma unroll
    for (int i = 0; i < D1; ++i) c[i] = df_add(c[i], df_mul(wf, lq[i]));
  }
  // range on the terms' magnitude |tau| max_q |w_q f_q| (the sums over the points may cancel)
  if (!mag_in_range(__fmul_rn(fabsf(meas.h), wfm), 0, meas.h != 0.0f && wfm != 0.0f)) st = worst(st, FEM_ERR_RANGE);
#pragma unroll
  for (int i = 0; i < D1; ++i) {
    const df2 v = df_mul(meas, c[i]);
    contrib[t * D1 + i] = make_float2(v.h, v.l);
  }
  if (st != FEM_OK) report(err, st);
}

__global__ void __launch_bounds__(256) k_rhs_gather(int64_t N, const int32_t* __restrict__ inc_ptr,
                                                    const int32_t* __restrict__ inc, const float2* __restrict__ contrib,
                                                    double* __restrict__ b) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  df2 acc = {0.0f, 0.0f};
  const int q1 = __ldg(inc_ptr + v + 1);
  for (int q = __ldg(inc_ptr + v); q < q1; ++q) {
    const float2 x = __ldg(contrib + __ldg(inc + q));
    acc = df_acc(acc, df2{x.x, x.y});
  }
  b[v] = df_to_double(acc);
}

template <int D>
__global__ void k_rule_points(int64_t NT, const int32_t* __restrict__ elem, const double* __restrict__ node, int nq,
                              const double* __restrict__ rule, double* __restrict__ pts) {
  constexpr int D1 = D + 1;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < NT * nq; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = s / nq;
    const int q = (int)(s - t * nq);
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double x = 0.0;
#pragma unroll
      for (int i = 0; i < D1; ++i)
        x = __dadd_rn(x, __dmul_rn(rule[q * D1 + i], __ldg(node + (size_t)__ldg(elem + t * D1 + i) * D + m)));
      pts[s * D + m] = x;
    }
  }
}

// the rule (bary then weights) on the device, per (device, d, n); never freed
const double* device_rule(int d, int n) {
  static std::mutex mu;
  static std::map<long long, double*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  const long long key = ((long long)dev << 16) | (d * 64 + n);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const Rule& r = rule_for(d, n);
  std::vector<double> h(r.bary);
  h.insert(h.end(), r.w.begin(), r.w.end());
  double* p = nullptr;
  if (cudaMalloc((void**)&p, sizeof(double) * h.size()) != cudaSuccess) return nullptr;
  if (cudaMemcpy(p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(p);
    return nullptr;
  }
  cache[key] = p;
  return p;
}

}  // namespace

int quad_rule(int d, int n, double* bary, double* w, int* nq) {
  const Rule& r = rule_for(d, n);
  const int m = (int)r.w.size();
  if (nq) *nq = m;
  if (bary) std::copy(r.bary.begin(), r.bary.end(), bary);
  if (w) std::copy(r.w.begin(), r.w.end(), w);
  return FEM_OK;
}

int rhs_rule(const Pattern* P, const double* node, int n, int f_kind, const double* f_arg, double* b, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  const float4* tab = sincos_table_device();
  if (!tab) return set_error(FEM_ERR_CUDA, "sin/cos table unavailable");
  const double* rule = device_rule(P->d, n);
  if (!rule) return set_error(FEM_ERR_CUDA, "quadrature rule upload failed");
  if (P->N == 0) return FEM_OK;
  if (P->NT == 0) {
    FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * P->N, s));
    return FEM_OK;
  }
  const int nq = P->d == 2 ? n * n : n * n * n;
  float2* contrib = reinterpret_cast<float2*>(P->scratch);  // d+1 float pairs per element
  const int smem = nq * (P->d1 + 1) * (int)sizeof(df2);
  const int g1 = (int)((P->NT + 127) / 128);
  if (P->d == 2)
    FEM_LAUNCH(k_rhs_rule<2>, g1, 128, smem, s, P->NT, P->elem, node, nq, rule, f_kind, f_arg, tab, contrib, err);
  else
    FEM_LAUNCH(k_rhs_rule<3>, g1, 128, smem, s, P->NT, P->elem, node, nq, rule, f_kind, f_arg, tab, contrib, err);
  FEM_LAUNCH(k_rhs_gather, (int)((P->N + 255) / 256), 256, 0, s, P->N, P->inc_ptr, P->inc, contrib, b);
  return FEM_OK;
}

int rule_points(const Pattern* P, const double* node, int n, double* pts, cudaStream_t s) {
  const double* rule = device_rule(P->d, n);
  if (!rule) return set_error(FEM_ERR_CUDA, "quadrature rule upload failed");
  const int nq = P->d == 2 ? n * n : n * n * n;
  const int64_t total = P->NT * nq;
  if (P->d == 2) FEM_LAUNCH(k_rule_points<2>, grid_for(total, 256), 256, 0, s, P->NT, P->elem, node, nq, rule, pts);
  else FEM_LAUNCH(k_rule_points<3>, grid_for(total, 256), 256, 0, s, P->NT, P->elem, node, nq, rule, pts);
  return FEM_OK;
}

}  // namespace fem
