// C ABI entry points (include/femasm.h): argument checks, handle lifetime, dispatch to the kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

namespace fem {

std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_timing{false};

namespace {
struct TimingRec {
  const char* name;
  cudaEvent_t b, e;
};
std::mutex g_tm_mu;
std::vector<TimingRec> g_tm_recs;
cudaEvent_t g_tm_pending = nullptr;
}  // namespace

void timing_mark(const char* name, cudaStream_t s, bool begin) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_tm_mu);
  cudaEvent_t ev = nullptr;
  if (cudaEventCreate(&ev) != cudaSuccess) return;
  cudaEventRecord(ev, s);
  if (begin) {
    if (g_tm_pending) cudaEventDestroy(g_tm_pending);
    g_tm_pending = ev;
  } else if (g_tm_pending) {
    g_tm_recs.push_back({name, g_tm_pending, ev});
    g_tm_pending = nullptr;
  } else {
    cudaEventDestroy(ev);
  }
}

namespace {
thread_local char g_msg[512] = "no error";
std::mutex g_err_mu;
int* g_err_word[64] = {nullptr};
}  // namespace

const char* g_msg_ptr() { return g_msg; }

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();
  return set_error(e == cudaErrorMemoryAllocation ? FEM_ERR_OOM : FEM_ERR_CUDA, "%s failed: %s", what,
                   cudaGetErrorString(e));
}

int* device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_word[dev]) {
    int* p = nullptr;
    if (cudaMalloc((void**)&p, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
    g_err_word[dev] = p;
  }
  return g_err_word[dev];
}

int* device_error_word_if_ready() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err_word[dev];
}

}  // namespace fem

using fem::Pattern;
using fem::set_error;

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

void free_pattern(Pattern& P) {
  fem::free_host_exec(P);
  fem::free_block_plan(P.blk);
  fem::free_tile_plan(P.tile);
  cudaFree(P.elem);
  cudaFree(P.row_ptr);
  cudaFree(P.col_idx);
  cudaFree(P.slot);
  cudaFree(P.inc_ptr);
  cudaFree(P.inc);
  cudaFree(P.scratch);
  cudaFree(P.work_counter);
  cudaFree(P.bd_whole);
  P = Pattern();
}

int check_values_args(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                      int variant) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (p->P.NT > 0 && !node) return set_error(FEM_ERR_ARG, "null node array");
  if (!aligned(node, 8) || !aligned(k, 8) || !aligned(f_arg, 8)) return set_error(FEM_ERR_ARG, "misaligned double array");
  if (f_kind != FEM_F_CONST && f_kind != FEM_F_SINPROD && f_kind != FEM_F_QPVALUES)
    return set_error(FEM_ERR_ARG, "unknown f_kind %d", f_kind);
  if (f_kind == FEM_F_QPVALUES && !f_arg && p->P.NT > 0) return set_error(FEM_ERR_ARG, "FEM_F_QPVALUES needs f_arg");
  if (variant != FEM_DETERMINISTIC && variant != FEM_ATOMIC) return set_error(FEM_ERR_ARG, "unknown variant %d", variant);
  return FEM_OK;
}

}  // namespace

extern "C" {

int fem_mesh_build_pattern(int d, int64_t N, int64_t NT, const int32_t* elem, fem_pattern_t* out, fem_stream_t stream) {
  if (!out) return set_error(FEM_ERR_ARG, "null output handle");
  *out = nullptr;
  if (d != 2 && d != 3) return set_error(FEM_ERR_ARG, "d must be 2 or 3 (got %d)", d);
  if (N < 0 || NT < 0 || N >= ((int64_t)1 << 31)) return set_error(FEM_ERR_ARG, "bad sizes N=%lld NT=%lld", (long long)N, (long long)NT);
  const int64_t d1 = d + 1;
  if (NT * d1 * d1 >= ((int64_t)1 << 31)) return set_error(FEM_ERR_ARG, "NT=%lld too large for int32 slot indexing", (long long)NT);
  if (NT > 0 && !elem) return set_error(FEM_ERR_ARG, "null elem array");
  if (!aligned(elem, 4)) return set_error(FEM_ERR_ARG, "misaligned elem array");
  fem_pattern_s* h = new (std::nothrow) fem_pattern_s();
  if (!h) return set_error(FEM_ERR_OOM, "host allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  Pattern& P = h->P;
  P.d = d;
  P.d1 = d + 1;
  P.N = N;
  P.NT = NT;
  cudaGetDevice(&P.device);
  if (!fem::device_error_word()) {
    delete h;
    return set_error(FEM_ERR_OOM, "cannot allocate the device error word");
  }
  int rc = fem::build_pattern(&P, elem, s);
  if (rc == FEM_OK && cudaMalloc((void**)&P.work_counter, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    P.work_counter = nullptr;
    rc = set_error(FEM_ERR_OOM, "work counter allocation failed");
  }
  if (rc == FEM_OK && NT > 0) {
    P.scratch_elems = fem::scratch_per_elem(d) * NT;
    if (cudaMallocAsync((void**)&P.scratch, sizeof(double) * (size_t)P.scratch_elems, s) != cudaSuccess) {
      cudaGetLastError();
      P.scratch = nullptr;
      rc = set_error(FEM_ERR_OOM, "scratch allocation failed");
    }
  }
  if (rc == FEM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = fem::cuda_error(cudaGetLastError(), "pattern build");
  if (rc == FEM_OK) rc = fem::rebuild_block_plan(&P, nullptr, nullptr, s);
  if (rc != FEM_OK) {
    cudaStreamSynchronize(s);
    free_pattern(P);
    delete h;
    return rc;
  }
  *out = h;
  return FEM_OK;
}

int fem_pattern_set_locality(fem_pattern_t p, const double* node, const int32_t* group, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!aligned(node, 8) || !aligned(group, 4)) return set_error(FEM_ERR_ARG, "misaligned array");
  return fem::rebuild_block_plan(&p->P, node, group, (cudaStream_t)stream);
}

int fem_pattern_launch_shape(fem_pattern_t p, int* rows_per_block, int* threads, int* ctas_per_sm, int* persistent,
                             float* tuned_ms) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  const fem::BlockPlan& B = p->P.blk;
  if (rows_per_block) *rows_per_block = B.ok ? B.V : 0;
  if (threads) *threads = B.ok ? B.threads : 0;
  if (ctas_per_sm) *ctas_per_sm = B.ok ? B.minb : 0;
  if (tuned_ms) *tuned_ms = B.tuned_ms;
  if (persistent) *persistent = B.ok && B.persistent ? 1 : 0;
  return FEM_OK;
}

int fem_pattern_force_launch(fem_pattern_t p, int threads, int ctas_per_sm, int persistent) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  fem::BlockPlan& B = p->P.blk;
  if (!B.ok) return set_error(FEM_ERR_STATE, "this mesh has no blocked plan");
  const bool ok2 = (threads == 512 && ctas_per_sm == 2) || (threads == 256 && (ctas_per_sm == 4 || ctas_per_sm == 2));
  const bool ok3 = (threads == 512 && ctas_per_sm == 1) || (threads == 256 && (ctas_per_sm == 2 || ctas_per_sm == 1));
  if (!(p->P.d == 2 ? ok2 : ok3)) return set_error(FEM_ERR_ARG, "unsupported launch shape %d x %d", threads, ctas_per_sm);
  if (fem::blocked_smem_need(B, p->P.d, p->P.d == 2) > fem::blocked_smem_budget(ctas_per_sm))
    return set_error(FEM_ERR_ARG, "launch shape %d x %d does not fit this plan in shared memory", threads, ctas_per_sm);
  B.threads = threads;
  B.minb = ctas_per_sm;
  B.persistent = persistent != 0;
  B.tuned_ms = 0.0f;
  p->P.use_tiles = false;
  return FEM_OK;
}

int fem_pattern_value_path(fem_pattern_t p, int* path, int* tile_elems, float* tuned_ms) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  const Pattern& P = p->P;
  const int pth = P.use_tiles ? (P.tile.fused ? FEM_PATH_TILES_FUSED : FEM_PATH_TILES)
                              : (P.blk.ok ? FEM_PATH_BLOCKED : FEM_PATH_TWO_PASS);
  if (path) *path = pth;
  if (tile_elems) *tile_elems = P.use_tiles ? P.tile.TE : 0;
  if (tuned_ms) {
    *tuned_ms = 0.0f;
    if ((pth == FEM_PATH_TILES || pth == FEM_PATH_TILES_FUSED) && P.tile.tuned_ms < 1e29f) *tuned_ms = P.tile.tuned_ms;
    if (pth == FEM_PATH_BLOCKED) *tuned_ms = P.blk.tuned_ms;
  }
  return FEM_OK;
}

int fem_pattern_barrier_fault(fem_pattern_t p, int extra_arrivals, int max_polls) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (extra_arrivals < 0 || max_polls < 0) return set_error(FEM_ERR_ARG, "negative fault-injection setting");
  p->P.bar_extra = extra_arrivals;
  p->P.bar_polls = max_polls;
  return FEM_OK;
}

int fem_pattern_force_path(fem_pattern_t p, int path, int tile_elems, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  Pattern& P = p->P;
  if (path == FEM_PATH_TWO_PASS) {
    fem::free_block_plan(P.blk);
    fem::free_tile_plan(P.tile);
    P.use_tiles = false;
    return FEM_OK;
  }
  if (path == FEM_PATH_BLOCKED) {
    if (!P.blk.ok) return set_error(FEM_ERR_STATE, "this mesh has no blocked plan");
    P.use_tiles = false;
    return FEM_OK;
  }
  if (path != FEM_PATH_TILES && path != FEM_PATH_TILES_FUSED) return set_error(FEM_ERR_ARG, "unknown value path %d", path);
  if (tile_elems != 128 && tile_elems != 256) return set_error(FEM_ERR_ARG, "tile size must be 128 or 256");
  if (!(P.tile.ok && P.tile.TE == tile_elems)) {
    fem::TilePlan T;
    int rc = fem::build_tile_plan(&P, P.blk.order, tile_elems, &T, (cudaStream_t)stream);
    if (rc) return rc;
    if (!T.ok) {
      fem::free_tile_plan(T);
      return set_error(FEM_ERR_STATE, "this mesh has no tile plan (a row longer than 256 entries)");
    }
    fem::free_tile_plan(P.tile);
    P.tile = T;
  }
  const bool fused = path == FEM_PATH_TILES_FUSED;
  if (fused && fem::tile_fused_smem(P.tile, P.d) == 0)
    return set_error(FEM_ERR_STATE, "the fused tile launch does not fit this mesh in shared memory");
  P.tile.fused = fused;
  P.use_tiles = true;
  return FEM_OK;
}

int fem_pattern_info(fem_pattern_t p, int* d, int64_t* N, int64_t* NT, int64_t* nnz, const int32_t** row_ptr,
                     const int32_t** col_idx, const int32_t** slot) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (d) *d = p->P.d;
  if (N) *N = p->P.N;
  if (NT) *NT = p->P.NT;
  if (nnz) *nnz = p->P.nnz;
  if (row_ptr) *row_ptr = p->P.row_ptr;
  if (col_idx) *col_idx = p->P.col_idx;
  if (slot) *slot = p->P.slot;
  return FEM_OK;
}

void fem_pattern_destroy(fem_pattern_t p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->P.device);
  cudaDeviceSynchronize();
  free_pattern(p->P);
  cudaSetDevice(cur);
  delete p;
}

int fem_assemble(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg, double* val,
                 double* b, int variant, fem_stream_t stream) {
  int rc = check_values_args(p, node, k, f_kind, f_arg, variant);
  if (rc) return rc;
  if (!aligned(val, 8) || !aligned(b, 8)) return set_error(FEM_ERR_ARG, "misaligned output array");
  if (!val && !b) return FEM_OK;
  if (variant == FEM_DETERMINISTIC && p->P.use_tiles)
    return fem::assemble_tiles(&p->P, node, k, f_kind, f_arg, val, b, (cudaStream_t)stream);
  if (variant == FEM_DETERMINISTIC && p->P.blk.ok)
    return fem::assemble_blocked(&p->P, node, k, f_kind, f_arg, val, b, (cudaStream_t)stream);
  return fem::assemble_values(&p->P, node, k, f_kind, f_arg, val, b, variant, (cudaStream_t)stream);
}

int fem_assemble_stiffness(fem_pattern_t p, const double* node, const double* k, double* val, int variant,
                           fem_stream_t stream) {
  if (!val) return set_error(FEM_ERR_ARG, "null val");
  return fem_assemble(p, node, k, FEM_F_CONST, nullptr, val, nullptr, variant, stream);
}

int fem_assemble_rhs(fem_pattern_t p, const double* node, int f_kind, const double* f_arg, double* b, int variant,
                     fem_stream_t stream) {
  if (!b) return set_error(FEM_ERR_ARG, "null b");
  return fem_assemble(p, node, nullptr, f_kind, f_arg, nullptr, b, variant, stream);
}

int fem_boundary_nodes(fem_pattern_t p, const int8_t* bdflag, uint8_t* is_bd, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (p->P.N > 0 && !is_bd) return set_error(FEM_ERR_ARG, "null is_bd");
  return fem::boundary_nodes(&p->P, bdflag, is_bd, (cudaStream_t)stream);
}

int fem_apply_dirichlet(fem_pattern_t p, const uint8_t* is_bd, const double* gD, double* val, double* b,
                        int32_t* free_node, int64_t* n_free, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (p->P.N > 0 && (!is_bd || !val)) return set_error(FEM_ERR_ARG, "null is_bd or val");
  if (!aligned(gD, 8) || !aligned(val, 8) || !aligned(b, 8) || !aligned(free_node, 4))
    return set_error(FEM_ERR_ARG, "misaligned array");
  return fem::apply_dirichlet(&p->P, is_bd, gD, val, b, free_node, n_free, (cudaStream_t)stream);
}

static int ensure_tile_plan(Pattern& P, cudaStream_t s);

int fem_assemble_operator(fem_pattern_t p, const double* node, int op, const double* coef, double* val,
                          fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!node || !val) return set_error(FEM_ERR_ARG, "node and val are required");
  if (!aligned(node, 8) || !aligned(coef, 8) || !aligned(val, 8)) return set_error(FEM_ERR_ARG, "misaligned array");
  if (op == FEM_OP_STIFFNESS)
    return fem_assemble(p, node, coef, FEM_F_CONST, nullptr, val, nullptr, FEM_DETERMINISTIC, stream);
  if (op != FEM_OP_MASS && op != FEM_OP_ANISO) return set_error(FEM_ERR_ARG, "unknown operator %d", op);
  if (op == FEM_OP_ANISO && !coef) return set_error(FEM_ERR_ARG, "the anisotropic operator needs its tensors");
  Pattern& P = p->P;
  if (P.NT == 0 || P.nnz == 0) {
    if (P.nnz > 0) FEM_CUDA(cudaMemsetAsync(val, 0, sizeof(double) * P.nnz, (cudaStream_t)stream));
    return FEM_OK;
  }
  int rc = ensure_tile_plan(P, (cudaStream_t)stream);
  if (rc) return rc;
  return fem::assemble_tiles(&P, node, nullptr, FEM_F_CONST, nullptr, val, nullptr, (cudaStream_t)stream, op, coef);
}

static int ensure_tile_plan(Pattern& P, cudaStream_t s) {
  if (P.tile.ok) return FEM_OK;
  fem::TilePlan T;
  int rc = fem::build_tile_plan(&P, P.blk.order, 128, &T, s);
  if (rc) return rc;
  if (!T.ok) {
    fem::free_tile_plan(T);
    return set_error(FEM_ERR_STATE, "this mesh has no tile plan (a row longer than 256 entries)");
  }
  P.tile = T;
  return FEM_OK;
}

int fem_apply_stiffness(fem_pattern_t p, const double* node, const double* k, const double* u, const uint8_t* is_bd,
                        double* y, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!node || !u || !y) return set_error(FEM_ERR_ARG, "node, u and y are required");
  if (u == y) return set_error(FEM_ERR_ARG, "u and y must be distinct");
  if (!aligned(node, 8) || !aligned(k, 8) || !aligned(u, 8) || !aligned(y, 8)) return set_error(FEM_ERR_ARG, "misaligned array");
  Pattern& P = p->P;
  if (P.N == 0) return FEM_OK;
  if (P.NT == 0) {
    FEM_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * P.N, (cudaStream_t)stream));
    return FEM_OK;
  }
  int rc = ensure_tile_plan(P, (cudaStream_t)stream);
  if (rc) return rc;
  return fem::assemble_tiles(&P, node, k, FEM_F_CONST, nullptr, nullptr, nullptr, (cudaStream_t)stream, 3, nullptr, u,
                             is_bd, y);
}

int fem_quad_rule(int d, int n, double* bary, double* w, int* nq) {
  if (d != 2 && d != 3) return set_error(FEM_ERR_ARG, "d must be 2 or 3");
  if (n < 1 || n > FEM_RULE_MAX_N) return set_error(FEM_ERR_ARG, "n must be in [1, %d]", FEM_RULE_MAX_N);
  return fem::quad_rule(d, n, bary, w, nq);
}

int fem_rule_points(fem_pattern_t p, const double* node, int n, double* pts, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (n < 1 || n > FEM_RULE_MAX_N) return set_error(FEM_ERR_ARG, "n must be in [1, %d]", FEM_RULE_MAX_N);
  if (!node || !pts || !aligned(node, 8) || !aligned(pts, 8)) return set_error(FEM_ERR_ARG, "bad node or pts");
  return fem::rule_points(&p->P, node, n, pts, (cudaStream_t)stream);
}

int fem_assemble_rhs_rule(fem_pattern_t p, const double* node, int n, int f_kind, const double* f_arg, double* b,
                          fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (n < 1 || n > FEM_RULE_MAX_N) return set_error(FEM_ERR_ARG, "n must be in [1, %d]", FEM_RULE_MAX_N);
  if (!node || !b || !aligned(node, 8) || !aligned(b, 8) || !aligned(f_arg, 8))
    return set_error(FEM_ERR_ARG, "bad node, b or f_arg");
  if (f_kind != FEM_F_CONST && f_kind != FEM_F_SINPROD && f_kind != FEM_F_QPVALUES)
    return set_error(FEM_ERR_ARG, "unknown f_kind %d", f_kind);
  if (f_kind == FEM_F_QPVALUES && !f_arg) return set_error(FEM_ERR_ARG, "FEM_F_QPVALUES needs f_arg");
  if (p->P.NT > 0 && !p->P.scratch) return set_error(FEM_ERR_STATE, "pattern has no scratch");
  return fem::rhs_rule(&p->P, node, n, f_kind, f_arg, b, (cudaStream_t)stream);
}

int fem_boundary_terms(fem_pattern_t p, const double* node, const int8_t* bdflag, const double* g_side, double g_const,
                       double alpha, double* val, double* b, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!node || !bdflag) return set_error(FEM_ERR_ARG, "node and bdflag are required");
  if (!aligned(node, 8) || !aligned(g_side, 8) || !aligned(val, 8) || !aligned(b, 8))
    return set_error(FEM_ERR_ARG, "misaligned array");
  if (!val && !b) return FEM_OK;
  return fem::boundary_terms(&p->P, node, bdflag, g_side, g_const, alpha, val, b, (cudaStream_t)stream);
}

int fem_side_points(fem_pattern_t p, const double* node, double* pts, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!node || !pts) return set_error(FEM_ERR_ARG, "node and pts are required");
  if (!aligned(node, 8) || !aligned(pts, 8)) return set_error(FEM_ERR_ARG, "misaligned array");
  return fem::side_points(&p->P, node, pts, (cudaStream_t)stream);
}

int fem_mean_shift(double* x, int64_t n, fem_stream_t stream) {
  if (n < 0) return set_error(FEM_ERR_ARG, "n must be >= 0");
  if (n > 0 && !x) return set_error(FEM_ERR_ARG, "null array");
  if (!aligned(x, 8)) return set_error(FEM_ERR_ARG, "misaligned array");
  return fem::mean_shift(x, n, (cudaStream_t)stream);
}

int fem_zero_average(fem_pattern_t p, const double* node, double* u, double* c_out, fem_stream_t stream) {
  if (!p) return set_error(FEM_ERR_ARG, "null pattern");
  if (!node || !u) return set_error(FEM_ERR_ARG, "node and u are required");
  if (!aligned(node, 8) || !aligned(u, 8) || !aligned(c_out, 8)) return set_error(FEM_ERR_ARG, "misaligned array");
  return fem::zero_average(&p->P, node, u, c_out, (cudaStream_t)stream);
}

int fem_assemble_backward(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                          const double* w, const double* r, double* gnode, double* gk, fem_stream_t stream) {
  int rc = check_values_args(p, node, k, f_kind, f_arg, FEM_DETERMINISTIC);
  if (rc) return rc;
  if (!aligned(w, 8) || !aligned(r, 8) || !aligned(gnode, 8) || !aligned(gk, 8))
    return set_error(FEM_ERR_ARG, "misaligned array");
  if (!gnode && !gk) return FEM_OK;
  return fem::assemble_backward(&p->P, node, k, f_kind, f_arg, w, r, gnode, gk, (cudaStream_t)stream);
}

int fem_get_error(fem_stream_t stream) {
  int* w = fem::device_error_word();
  if (!w) return set_error(FEM_ERR_CUDA, "no device error word");
  cudaStream_t s = (cudaStream_t)stream;
  int code = 0;
  if (cudaMemcpyAsync(&code, w, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fem::cuda_error(cudaGetLastError(), "reading the device error word");
  if (code != 0) {
    cudaMemsetAsync(w, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return set_error(code, "a kernel reported error %d (%s)", code,
                     code == FEM_ERR_DEGENERATE ? "degenerate or inverted element"
                     : code == FEM_ERR_INDEX    ? "index out of range"
                     : code == FEM_ERR_TIMEOUT  ? "device wait timed out"
                                                : "see femasm.h");
  }
  return FEM_OK;
}

const char* fem_last_error_string(void) { return fem::g_msg_ptr(); }

int64_t fem_launch_count(void) { return fem::g_launches.load(); }

int fem_timing_enable(int on) {
  fem::g_timing.store(on != 0);
  return FEM_OK;
}

int fem_timing_report(char* buf, int64_t buflen) {
  std::lock_guard<std::mutex> lk(fem::g_tm_mu);
  struct Acc {
    const char* name;
    int64_t n;
    double ms;
  };
  std::vector<Acc> acc;
  int rc = FEM_OK;
  for (auto& r : fem::g_tm_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.e) != cudaSuccess || cudaEventElapsedTime(&ms, r.b, r.e) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(FEM_ERR_CUDA, "timing event failed");
    }
    cudaEventDestroy(r.b);
    cudaEventDestroy(r.e);
    size_t i = 0;
    while (i < acc.size() && strcmp(acc[i].name, r.name) != 0) ++i;
    if (i == acc.size()) acc.push_back({r.name, 0, 0.0});
    acc[i].n += 1;
    acc[i].ms += ms;
  }
  fem::g_tm_recs.clear();
  if (buf && buflen > 0) {
    int64_t off = 0;
    buf[0] = 0;
    for (auto& x : acc) {
      int w = snprintf(buf + off, (size_t)(buflen - off), "%s %lld %.6f\n", x.name, (long long)x.n, x.ms);
      if (w < 0 || off + w >= buflen) break;
      off += w;
    }
  }
  return rc;
}

}  // extern "C"
