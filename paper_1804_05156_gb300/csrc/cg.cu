// Conjugate gradients on the Dirichlet-eliminated system, driven by the matrix-free operator
// (fem_cg_solve) or by the assembled CSR matrix (fem_cg_solve_csr, with the product fem_csr_spmv).
//
// Sec. 3.3 ends the method with the reduced solve u(freeNode) = A(freeNode, freeNode) \ b(freeNode), after
// the boundary values are lifted out: b <- b - A u_D. Here the stiffness matrix is never formed. The lift
// uses the full operator y = A u_D, and every iteration applies the eliminated operator of
// fem_apply_stiffness (boundary vertices contribute nothing to free rows, boundary rows give y = u), on
// the full-length vectors. Starting from u = u_D with r = 0 on the boundary rows, the boundary entries of
// r and p stay 0, so the iteration is plain CG on the free rows: A(free, free) is symmetric positive
// definite when every connected piece of the mesh has a boundary vertex.
//
// Every dot product is a fixed-shape FP64 reduction: a fixed number of blocks (a function of N only),
// each summing a fixed contiguous chunk in a fixed order, then each consumer sums the block partials
// with the same fixed tree. The iteration is therefore bitwise reproducible, on any GPU. Scalars
// (alpha, beta) are formed on the device, redundantly in every block from the partials, so the host
// synchronises only to test convergence every few iterations. Once converged a device flag freezes u,
// r and p: the reported iteration count and result do not depend on when the host looks.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "common.cuh"

extern "C" int fem_apply_stiffness(fem_pattern_t p, const double* node, const double* k, const double* u,
                                   const uint8_t* is_bd, double* y, fem_stream_t stream);

namespace fem {
namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxRedBlocks = 1024;
constexpr int kCheckEvery = 8;  // iterations between host convergence tests

// scalar slots of the workspace
enum { kDone = 0, kIters = 1 };          // int slots
enum { kRR0 = 0, kRRLast = 1 };          // double slots

int red_blocks(int64_t N) { return (int)std::min<int64_t>(kMaxRedBlocks, std::max<int64_t>(1, (N + 4095) / 4096)); }

// Sum of one value per thread over the block, fixed order: shuffle tree in each warp, then warp 0 adds
// the warp sums with the same tree. The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Sum of the nb block partials, fixed order (lane-strided, then a shuffle tree), broadcast to the block.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int nb, double* sh) {
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) v += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sh[32] = v;
  }
  __syncthreads();
  const double s = sh[32];
  __syncthreads();
  return s;
}

// The done flag, read once per block (every thread of the block takes the same branch even when another
// block writes the flag during this kernel).
__device__ __forceinline__ bool block_done(const int* isc) {
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = isc[kDone];
  __syncthreads();
  const bool d = s_done != 0;
  __syncthreads();
  return d;
}

// [lo, hi) of block b when N entries are cut into nb equal chunks
__device__ __forceinline__ void chunk(int64_t N, int nb, int b, int64_t& lo, int64_t& hi) {
  const int64_t c = (N + nb - 1) / nb;
  lo = (int64_t)b * c;
  hi = lo + c < N ? lo + c : N;
}

// u_D: the boundary values on boundary vertices, 0 elsewhere
__global__ void k_cg_lift(int64_t N, const uint8_t* __restrict__ isbd, const double* __restrict__ gD,
                          double* __restrict__ ud) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    ud[i] = (isbd[i] && gD) ? gD[i] : 0.0;
}

// u = u_D, r = b - A u_D on free rows (0 on boundary rows), p = r; partial sums of r.r
__global__ void __launch_bounds__(kRedThreads) k_cg_init(int64_t N, const uint8_t* __restrict__ isbd,
                                                         const double* __restrict__ b, const double* __restrict__ gD,
                                                         const double* __restrict__ Aud, double* __restrict__ u,
                                                         double* __restrict__ r, double* __restrict__ p,
                                                         double* __restrict__ part) {
  __shared__ double sh[33];
  int64_t lo, hi;
  chunk(N, gridDim.x, blockIdx.x, lo, hi);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const bool bd = isbd[i] != 0;
    const double ri = bd ? 0.0 : b[i] - Aud[i];
    u[i] = bd ? (gD ? gD[i] : 0.0) : 0.0;
    r[i] = ri;
    p[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// rr0 = r.r; done at once when it is 0 (u_D already solves the system)
__global__ void k_cg_start(const double* __restrict__ part, int nb, double* __restrict__ dsc, int* __restrict__ isc) {
  __shared__ double sh[33];
  const double rr = sum_partials(part, nb, sh);
  if (threadIdx.x == 0) {
    dsc[kRR0] = rr;
    dsc[kRRLast] = rr;
    isc[kIters] = 0;
    isc[kDone] = (rr == 0.0) ? 1 : 0;
  }
}

// partial sums of p.q
__global__ void __launch_bounds__(kRedThreads) k_cg_pq(int64_t N, const double* __restrict__ p,
                                                       const double* __restrict__ q, double* __restrict__ part,
                                                       const int* __restrict__ isc) {
  __shared__ double sh[33];
  if (block_done(isc)) return;
  int64_t lo, hi;
  chunk(N, gridDim.x, blockIdx.x, lo, hi);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += p[i] * q[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = (r.r) / (p.q); u += alpha p; r -= alpha q; partial sums of the new r.r
__global__ void __launch_bounds__(kRedThreads) k_cg_update(int64_t N, const double* __restrict__ p,
                                                           const double* __restrict__ q, double* __restrict__ u,
                                                           double* __restrict__ r, const double* __restrict__ part_rr,
                                                           const double* __restrict__ part_pq,
                                                           double* __restrict__ part_rr_new, int* __restrict__ isc) {
  __shared__ double sh[33];
  if (block_done(isc)) return;
  const int nb = gridDim.x;
  const double rr = sum_partials(part_rr, nb, sh);
  const double pq = sum_partials(part_pq, nb, sh);
  if (!(pq > 0.0)) {  // breakdown: A not positive definite on the free rows (or a NaN)
    if (blockIdx.x == 0 && threadIdx.x == 0) isc[kDone] = 2;
    return;
  }
  const double alpha = rr / pq;
  int64_t lo, hi;
  chunk(N, nb, blockIdx.x, lo, hi);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    u[i] = u[i] + alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part_rr_new[blockIdx.x] = s;
}

// beta = (r.r)_new / (r.r)_old; p = r + beta p; one more iteration counted; done when
// (r.r)_new <= tol2 * rr0
__global__ void __launch_bounds__(kRedThreads) k_cg_direction(int64_t N, const double* __restrict__ r,
                                                              double* __restrict__ p,
                                                              const double* __restrict__ part_rr,
                                                              const double* __restrict__ part_rr_new, double tol2,
                                                              double* __restrict__ dsc, int* __restrict__ isc) {
  __shared__ double sh[33];
  if (block_done(isc)) return;
  const int nb = gridDim.x;
  const double rr = sum_partials(part_rr, nb, sh);
  const double rn = sum_partials(part_rr_new, nb, sh);
  const double beta = rn / rr;
  int64_t lo, hi;
  chunk(N, nb, blockIdx.x, lo, hi);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = r[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dsc[kRRLast] = rn;
    isc[kIters] = isc[kIters] + 1;
    if (rn <= tol2 * dsc[kRR0]) isc[kDone] = 1;
  }
}

// y = A x for the assembled CSR values, one thread per row: the row's entries in order, four at a time
// (their column indices and values, then the four x values, then four FP64 multiply-adds), so that
// several independent loads are in flight per thread; the sum order is fixed, so the result is bitwise
// reproducible. (A group of lanes per row with a shuffle tree was 3.5x slower: its dependent chain of
// row_ptr, col, x loads per row left too few rows in flight.) With is_bd, the Dirichlet-eliminated
// operator: a row of an eliminated vertex gives y_i = x_i and the columns of eliminated vertices are
// skipped.
__global__ void __launch_bounds__(256) k_csr_spmv(int64_t N, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ x, const uint8_t* __restrict__ isbd,
                                                  double* __restrict__ y) {
  for (int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; R < N; R += (int64_t)gridDim.x * blockDim.x) {
    if (isbd && isbd[R]) {
      y[R] = x[R];
      continue;
    }
    const int a = __ldg(row_ptr + R), e = __ldg(row_ptr + R + 1);
    double sum = 0.0;
    int q = a;
    for (; q + 4 <= e; q += 4) {
      int c[4];
      double v[4], xv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        c[j] = __ldg(col + q + j);
        v[j] = __ldg(val + q + j);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) xv[j] = (!isbd || !__ldg(isbd + c[j])) ? __ldg(x + c[j]) : 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) sum = __fma_rn(v[j], xv[j], sum);
    }
    for (; q < e; ++q) {
      const int c = __ldg(col + q);
      if (!isbd || !__ldg(isbd + c)) sum = __fma_rn(__ldg(val + q), __ldg(x + c), sum);
    }
    y[R] = sum;
  }
}

}  // namespace
}  // namespace fem

using fem::set_error;

namespace {

int launch_spmv(const fem::Pattern& P, const double* val, const double* x, const uint8_t* is_bd, double* y,
                cudaStream_t s) {
  using namespace fem;
  k_csr_spmv<<<grid_for(P.N, 256), 256, 0, s>>>(P.N, P.row_ptr, P.col_idx, val, x, is_bd, y);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEM_OK : cuda_error(e, "k_csr_spmv");
}

// The CG iteration of both entry points; apply(x, is_bd, y) is the operator (is_bd null: the full one).
template <class Apply>
int cg_run(const fem::Pattern& P, Apply apply, const uint8_t* is_bd, const double* b, const double* gD, double* u,
           int max_iter, double rtol, int* iters, double* relres, cudaStream_t s) {
  using namespace fem;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  const int64_t N = P.N;
  if (N == 0) return FEM_OK;
  const int nb = red_blocks(N);
  // workspace: r, p, q [N]; partials rr (two, alternating), pq [nb]; doubles then ints
  const size_t nd = 3 * (size_t)N + 3 * (size_t)nb + 2;
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, sizeof(double) * nd + 2 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (CG workspace)");
  double* r = static_cast<double*>(ws);
  double* pv = r + N;
  double* q = pv + N;
  double* part_rr[2] = {q + N, q + N + nb};
  double* part_pq = q + N + 2 * nb;
  double* dsc = part_pq + nb;
  int* isc = reinterpret_cast<int*>(dsc + 2);
  int rc = FEM_OK;
  int hs[2] = {0, 0};
  double hd[2] = {0.0, 0.0};
  int it = 0;
  const double tol2 = rtol * rtol;
#define CG_TRY(x)                      \
  do {                                 \
    rc = (x);                          \
    if (rc != FEM_OK) goto done_label; \
  } while (0)
#define CG_CUDA(x)                          \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) {                \
      rc = cuda_error(e_, #x);              \
      goto done_label;                      \
    }                                       \
  } while (0)
#define CG_LAUNCH(kernel, grid, block, ...)                     \
  do {                                                          \
    kernel<<<(grid), (block), 0, s>>>(__VA_ARGS__);             \
    g_launches.fetch_add(1, std::memory_order_relaxed);         \
    CG_CUDA(cudaGetLastError());                                \
  } while (0)
  // lift: r = b - A u_D on free rows
  CG_LAUNCH(k_cg_lift, grid_for(N, 256), 256, N, is_bd, gD, pv);
  CG_TRY(apply(pv, nullptr, q));
  CG_LAUNCH(k_cg_init, nb, kRedThreads, N, is_bd, b, gD, q, u, r, pv, part_rr[0]);
  CG_LAUNCH(k_cg_start, 1, 32, part_rr[0], nb, dsc, isc);
  for (it = 0; it < max_iter; ++it) {
    const int par = it & 1;
    CG_TRY(apply(pv, is_bd, q));
    CG_LAUNCH(k_cg_pq, nb, kRedThreads, N, pv, q, part_pq, isc);
    CG_LAUNCH(k_cg_update, nb, kRedThreads, N, pv, q, u, r, part_rr[par], part_pq, part_rr[1 - par], isc);
    CG_LAUNCH(k_cg_direction, nb, kRedThreads, N, r, pv, part_rr[par], part_rr[1 - par], tol2, dsc, isc);
    if ((it + 1) % kCheckEvery == 0 || it + 1 == max_iter) {
      CG_CUDA(cudaMemcpyAsync(hs, isc, sizeof(hs), cudaMemcpyDeviceToHost, s));
      CG_CUDA(cudaStreamSynchronize(s));
      if (hs[kDone]) break;
    }
  }
  CG_CUDA(cudaMemcpyAsync(hs, isc, sizeof(hs), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaMemcpyAsync(hd, dsc, sizeof(hd), cudaMemcpyDeviceToHost, s));
  CG_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = hs[kIters];
  if (relres) *relres = hd[kRR0] > 0.0 ? sqrt(hd[kRRLast] / hd[kRR0]) : 0.0;
  if (hs[kDone] == 2) rc = set_error(FEM_ERR_STATE, "CG breakdown: p.Ap <= 0 (the operator is not positive definite "
                                                    "on the free vertices)");
done_label:
#undef CG_TRY
#undef CG_CUDA
#undef CG_LAUNCH
  cudaFreeAsync(ws, s);
  return rc;
}

bool aligned8(const void* q) { return ((uintptr_t)q % 8) == 0; }

}  // namespace

extern "C" int fem_cg_solve(fem_pattern_t p, const double* node, const double* k, const uint8_t* is_bd,
                            const double* b, const double* gD, double* u, int max_iter, double rtol, int* iters,
                            double* relres, fem_stream_t stream) {
  using namespace fem;
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  const Pattern& P = p->P;
  if (max_iter < 0 || !(rtol >= 0.0)) return set_error(FEM_ERR_ARG, "max_iter must be >= 0 and rtol >= 0");
  if (P.N > 0 && (!node || !is_bd || !b || !u)) return set_error(FEM_ERR_ARG, "node, is_bd, b and u are required");
  if (!aligned8(node) || !aligned8(k) || !aligned8(b) || !aligned8(gD) || !aligned8(u))
    return set_error(FEM_ERR_ARG, "misaligned double array");
  if (u == b || u == gD) return set_error(FEM_ERR_ARG, "u must not alias b or gD");
  auto apply = [&](const double* x, const uint8_t* bd, double* y) {
    return fem_apply_stiffness(p, node, k, x, bd, y, stream);
  };
  return cg_run(P, apply, is_bd, b, gD, u, max_iter, rtol, iters, relres, (cudaStream_t)stream);
}

extern "C" int fem_csr_spmv(fem_pattern_t p, const double* val, const double* x, const uint8_t* is_bd, double* y,
                            fem_stream_t stream) {
  using namespace fem;
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  const Pattern& P = p->P;
  if (P.N == 0) return FEM_OK;
  if (!val || !x || !y) return set_error(FEM_ERR_ARG, "val, x and y are required");
  if (!aligned8(val) || !aligned8(x) || !aligned8(y)) return set_error(FEM_ERR_ARG, "misaligned double array");
  if (x == y) return set_error(FEM_ERR_ARG, "x and y must be distinct");
  return launch_spmv(P, val, x, is_bd, y, (cudaStream_t)stream);
}

extern "C" int fem_cg_solve_csr(fem_pattern_t p, const double* val, const uint8_t* is_bd, const double* b,
                                const double* gD, double* u, int max_iter, double rtol, int* iters, double* relres,
                                fem_stream_t stream) {
  using namespace fem;
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  const Pattern& P = p->P;
  if (max_iter < 0 || !(rtol >= 0.0)) return set_error(FEM_ERR_ARG, "max_iter must be >= 0 and rtol >= 0");
  if (P.N > 0 && (!val || !is_bd || !b || !u)) return set_error(FEM_ERR_ARG, "val, is_bd, b and u are required");
  if (!aligned8(val) || !aligned8(b) || !aligned8(gD) || !aligned8(u))
    return set_error(FEM_ERR_ARG, "misaligned double array");
  if (u == b || u == gD || u == val) return set_error(FEM_ERR_ARG, "u must not alias val, b or gD");
  const cudaStream_t s = (cudaStream_t)stream;
  auto apply = [&](const double* x, const uint8_t* bd, double* y) { return launch_spmv(P, val, x, bd, y, s); };
  return cg_run(P, apply, is_bd, b, gD, u, max_iter, rtol, iters, relres, s);
}
