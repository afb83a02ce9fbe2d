// Value kernels (FP64 reference path): local stiffness, load vector, and their reduction into the CSR
// values through the slot map.
//
// Sec. 3.1.3: grad lambda_i = n_i / (d! |tau|) (eq. (dlambda)) and a_ij^tau = n_i . n_j / (d!^2 |tau|),
// with n_i the scaled inward normal of the side opposite vertex i; only the off-diagonal entries are
// formed from dot products and the diagonal is minus the off-diagonal row sum (sum_i n_i = 0), which
// halves the dot products (the symmetry remark of Sec. 3.1.3 taken one step further).
// Sec. 3.2: 2-D three-edge-midpoint rule; 3-D four-point degree-2 rule.
#include <cuda_runtime.h>

#include "common.cuh"
#include "element.cuh"

namespace fem {

namespace {

// ---- atomic variant: one thread per element, FP64 atomicAdd into val and b ------------------------
template <int D>
__global__ void __launch_bounds__(256) k_assemble_atomic(const int32_t* __restrict__ elem, int64_t NT,
                                                         const double* __restrict__ node, const double* __restrict__ k,
                                                         int f_kind, const double* __restrict__ f_arg,
                                                         const int32_t* __restrict__ slot, double* __restrict__ val,
                                                         double* __restrict__ b, int* __restrict__ err) {
  constexpr int D1 = D + 1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    int e[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) e[i] = elem[t * D1 + i];
    double x[D1][D];
    load_coords<D>(node, e, x);
    Local<D> L;
    if (!element_local<D>(x, k ? k[t] : 1.0, val != nullptr, b != nullptr, f_kind, f_arg, t, L)) report(err, FEM_ERR_DEGENERATE);
    if (val) {
#pragma unroll
      for (int i = 0; i < D1; ++i)
#pragma unroll
        for (int j = 0; j < D1; ++j) atomicAdd(val + slot[(int64_t)(i * D1 + j) * NT + t], L.a[pidx<D>(i, j)]);
    }
    if (b) {
#pragma unroll
      for (int i = 0; i < D1; ++i) atomicAdd(b + e[i], L.bt[i]);
    }
  }
}

// ---- deterministic variant, pass 1: per-element values to scratch (SoA) ----------------------------
template <int D>
__global__ void __launch_bounds__(256) k_element_values(const int32_t* __restrict__ elem, int64_t NT,
                                                        const double* __restrict__ node, const double* __restrict__ k,
                                                        int f_kind, const double* __restrict__ f_arg, bool want_a,
                                                        bool want_b, double* __restrict__ scratch, int* __restrict__ err) {
  constexpr int D1 = D + 1, U = D1 * (D1 + 1) / 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    int e[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) e[i] = elem[t * D1 + i];
    double x[D1][D];
    load_coords<D>(node, e, x);
    Local<D> L;
    if (!element_local<D>(x, k ? k[t] : 1.0, want_a, want_b, f_kind, f_arg, t, L)) report(err, FEM_ERR_DEGENERATE);
    if (want_a) {
#pragma unroll
      for (int c = 0; c < U; ++c) scratch[(int64_t)c * NT + t] = L.a[c];
    }
    if (want_b) {
#pragma unroll
      for (int i = 0; i < D1; ++i) scratch[(int64_t)(U + i) * NT + t] = L.bt[i];
    }
  }
}

// ---- deterministic variant, pass 2: one thread per row sums its incidences in element order ----------
template <int D>
__global__ void __launch_bounds__(256) k_row_reduce(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc,
                                                    const int32_t* __restrict__ slot, int64_t N, int64_t NT,
                                                    const double* __restrict__ scratch, double* __restrict__ val,
                                                    double* __restrict__ b) {
  constexpr int D1 = D + 1, U = D1 * (D1 + 1) / 2;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int q0 = inc_ptr[r], q1 = inc_ptr[r + 1];
    double bacc = 0.0;
    for (int q = q0; q < q1; ++q) {
      const int p = inc[q];
      const int64_t t = p / D1;
      const int i = p - (int)t * D1;
      if (val) {
        for (int j = 0; j < D1; ++j) {
          const int s = slot[(int64_t)(i * D1 + j) * NT + t];
          val[s] = val[s] + scratch[(int64_t)pidx_rt<D>(i, j) * NT + t];
        }
      }
      if (b) bacc = bacc + scratch[(int64_t)(U + i) * NT + t];
    }
    if (b) b[r] = bacc;
  }
}

}  // namespace

int assemble_values(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                    double* val, double* b, int variant, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  const int64_t NT = P->NT, N = P->N;
  if (val && P->nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P->nnz, s));
  if (b && N > 0) FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * N, s));
  if (NT == 0) return FEM_OK;
  const int grid = grid_for(NT, 256, 152 * 16);
  if (variant == FEM_ATOMIC) {
    if (P->d == 2)
      FEM_LAUNCH(k_assemble_atomic<2>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, val, b, err);
    else
      FEM_LAUNCH(k_assemble_atomic<3>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, P->slot, val, b, err);
    return FEM_OK;
  }
  if (!P->scratch) return set_error(FEM_ERR_STATE, "pattern has no scratch for the deterministic reduction");
  if (P->d == 2) {
    FEM_LAUNCH(k_element_values<2>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, val != nullptr, b != nullptr,
               P->scratch, err);
    FEM_LAUNCH(k_row_reduce<2>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, P->slot, N, NT, P->scratch, val, b);
  } else {
    FEM_LAUNCH(k_element_values<3>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, val != nullptr, b != nullptr,
               P->scratch, err);
    FEM_LAUNCH(k_row_reduce<3>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, P->slot, N, NT, P->scratch, val, b);
  }
  return FEM_OK;
}

int assemble_values_two_pass(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                              double* val, double* b, double* scratch, int* err, cudaStream_t s) {
  const int64_t NT = P->NT, N = P->N;
  if (val && P->nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P->nnz, s));
  if (b && N > 0) FEM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * N, s));
  if (NT == 0) return FEM_OK;
  const int grid = grid_for(NT, 256, 152 * 16);
  if (P->d == 2) {
    FEM_LAUNCH_UNTIMED(k_element_values<2>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, val != nullptr, b != nullptr,
               scratch, err);
    FEM_LAUNCH_UNTIMED(k_row_reduce<2>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, P->slot, N, NT, scratch, val, b);
  } else {
    FEM_LAUNCH_UNTIMED(k_element_values<3>, grid, 256, 0, s, P->elem, NT, node, k, f_kind, f_arg, val != nullptr, b != nullptr,
               scratch, err);
    FEM_LAUNCH_UNTIMED(k_row_reduce<3>, grid_for(N, 256), 256, 0, s, P->inc_ptr, P->inc, P->slot, N, NT, scratch, val, b);
  }
  return FEM_OK;
}

}  // namespace fem
