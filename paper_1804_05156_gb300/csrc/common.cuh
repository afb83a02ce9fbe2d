// Shared internals of the femasm CUDA library (sm_103a). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "femasm.h"

namespace fem {

// ---- error word --------------------------------------------------------------------------------
// One int per device, allocated on first use: the first non-zero code a kernel reports wins;
// fem_get_error reads and clears it. Kernels receive its address as an argument.
__device__ __forceinline__ void report(int* err, int code) { atomicCAS(err, 0, code); }
int* device_error_word();  // for the current device; nullptr on allocation failure

// ---- host-side bookkeeping -----------------------------------------------------------------------
extern std::atomic<int64_t> g_launches;
int set_error(int code, const char* fmt, ...);
const char* g_msg_ptr();
int cuda_error(cudaError_t e, const char* what);

#define FEM_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::fem::cuda_error(e_, #call); \
  } while (0)

// Per-kernel timing (off by default): CUDA events recorded on the launching stream around each
// launch, summed per kernel name by fem_timing_report.
extern std::atomic<bool> g_timing;
void timing_mark(const char* name, cudaStream_t s, bool begin);

// Launch helper: counts every kernel launch, optionally times it, and checks the launch error.
#define FEM_LAUNCH(kernel, grid, block, smem, stream, ...)                        \
  do {                                                                            \
    if ((grid) > 0) {                                                             \
      const bool tm_ = ::fem::g_timing.load(std::memory_order_relaxed);           \
      if (tm_) ::fem::timing_mark(#kernel, (stream), true);                       \
      kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                 \
      ::fem::g_launches.fetch_add(1, std::memory_order_relaxed);                  \
      cudaError_t e_ = cudaGetLastError();                                        \
      if (e_ != cudaSuccess) return ::fem::cuda_error(e_, #kernel);              \
      if (tm_) ::fem::timing_mark(#kernel, (stream), false);                      \
    }                                                                             \
  } while (0)

// Same, without the optional timing events (for paths that must not create any CUDA objects).
#define FEM_LAUNCH_UNTIMED(kernel, grid, block, smem, stream, ...)                \
  do {                                                                            \
    if ((grid) > 0) {                                                             \
      kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                 \
      ::fem::g_launches.fetch_add(1, std::memory_order_relaxed);                  \
      cudaError_t e_ = cudaGetLastError();                                        \
      if (e_ != cudaSuccess) return ::fem::cuda_error(e_, #kernel);              \
    }                                                                             \
  } while (0)

inline int grid_for(int64_t n, int block, int max_blocks = 152 * 32) {
  int64_t g = (n + block - 1) / block;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// ---- locality plan (owner-computes blocks), see blockplan.cu -----------------------------------------
struct BlockPlan {
  int V = 0, nblocks = 0;
  int64_t E = 0, VT = 0;                  // listed elements / listed vertices over all blocks
  int max_e = 0, max_v = 0, max_acc = 0;  // per-block maxima (shared-memory sizing)
  int max_rec = 0;                        // most records in one block
  int threads = 512, minb = 1;            // launch shape: threads per CTA, CTAs per SM
  bool persistent = false;                // one resident wave drawing blocks from a counter
  float tuned_ms = 0.0f;                  // the tuner's time for the chosen shape (0 if not tuned)
  bool ok = false;                        // the packed record limits hold for this mesh
  int32_t* order = nullptr;               // [N] vertices in locality order; block b owns [b*V, b*V+V)
  int32_t* rec_off = nullptr;             // [N+1] record offsets of the owned rows, locality order
  uint16_t* own_local = nullptr;          // [N] local vertex id of each owned row in its block
  int32_t* rowp = nullptr;                // [N] row_ptr of each owned row, locality order
  uint16_t* rldp = nullptr;               // [N] row length | in-row position of the diagonal << 8
  int32_t* eoff = nullptr;                // [nblocks+1] element-list offsets
  int32_t* voff = nullptr;                // [nblocks+1] vertex-list offsets
  int32_t* elist = nullptr;               // [E] caller element ids, ascending within a block
  uint16_t* lelem = nullptr;              // [(d+1)][E] local vertex ids of the listed elements
  int32_t* vlist = nullptr;               // [VT] global vertex ids, ascending within a block
  uint32_t* rec = nullptr;                // [NT*(d+1)] packed incidence records
};
void free_block_plan(BlockPlan& B);
int build_block_plan(const struct Pattern* P, const double* node_hint, const int32_t* group, int V, BlockPlan* out,
                     cudaStream_t s);

// ---- tile plan of the two-phase value path, see tileplan.cu -----------------------------------------
struct TilePlan {
  int TE = 0, ntiles = 0;      // elements per tile, tiles
  int64_t VT = 0;              // listed vertices over all tiles
  int max_v = 0, max_row = 0;  // most vertices of one tile; longest row
  bool ok = false;             // local ids fit 16 bits and rows have <= 256 entries
  float tuned_ms = 1e30f;      // the tuner's time for this plan (1e30 if not timed)
  bool fused = false;          // both phases in one cooperative launch (k_tiles_fused)
  int32_t* elist = nullptr;    // [NT] caller element ids in tile order
  uint16_t* lelem = nullptr;   // [(d+1)][NT] local vertex ids, tile order
  int32_t* voff = nullptr;     // [ntiles+1] vertex-list offsets
  int32_t* vlist = nullptr;    // [VT] global vertex ids, ascending within a tile
  int32_t* ipos = nullptr;     // [(d+1)][NT] packet (incidence) index of (elist[j], i)
  void* pw = nullptr;          // [NT*(d+1)] per incidence: other columns' in-row positions (uint16 2-D, uint32 3-D)
  uint8_t* rdp = nullptr;      // [N] in-row position of the diagonal
  float4* pk = nullptr;        // packets, 32 bytes per incidence: 3-D and fused 2-D [NT*(d+1)][2] float4;
                               // two-launch 2-D a pair array [NT*3] float4 then a load array [NT*3] float2
};
void free_tile_plan(TilePlan& T);
int build_tile_plan(const struct Pattern* P, const int32_t* order, int TE, TilePlan* out, cudaStream_t s);

// ---- pattern object --------------------------------------------------------------------------------
struct Pattern {
  int d = 0, d1 = 0;
  int64_t N = 0, NT = 0, nnz = 0;
  int device = 0;
  int32_t* elem = nullptr;     // [NT][d+1], copy of the caller's topology
  int32_t* row_ptr = nullptr;  // [N+1]
  int32_t* col_idx = nullptr;  // [nnz]
  int32_t* slot = nullptr;     // [(d+1)^2][NT]
  int32_t* inc_ptr = nullptr;  // [N+1] vertex -> incidence list offsets
  int32_t* inc = nullptr;      // [NT*(d+1)] entries t*(d+1)+i, ascending within a vertex
  double* scratch = nullptr;   // per-element values for the deterministic reduction
  int64_t scratch_elems = 0;   // doubles in scratch
  BlockPlan blk;               // owner-computes locality plan (blk.ok == false: two-pass path only)
  TilePlan tile;               // two-phase plan (tile.ok == false: not available)
  bool use_tiles = false;      // the deterministic value path runs the two-phase kernels
  bool one_launch = false;     // plans must run in a single launch (batched assembly under a graph)
  int* work_counter = nullptr; // [4] device counters: [0] blocked persistent launch, [1..3] fused tile launch
  uint8_t* bd_whole = nullptr;  // [N] whole-boundary vertex mask, computed on first request
  struct HostExec* hx = nullptr;  // streams and device buffers of fem_assemble_host, made on first use
  int bar_extra = 0;           // fault injection: arrivals the fused grid barrier waits for beyond the grid
  int bar_polls = 0;           // fault injection: poll limit of the fused grid barrier (0: the default)
};
void free_host_exec(Pattern& P);
// (Re)build P->blk, halving the block size until the packed limits hold (blk.ok false if they never do).
int rebuild_block_plan(Pattern* P, const double* node_hint, const int32_t* group, cudaStream_t s);
// For a pattern that must run in one launch: switch the tile plan to its fused form, or fall back to the
// persistent blocked launch.
void enforce_one_launch(Pattern* P);
int blocked_smem_budget(int ctas_per_sm);
int blocked_smem_need(const BlockPlan& B, int d, bool sinprod);
int assemble_blocked(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                     double* val, double* b, cudaStream_t s);
// op: 0 stiffness (+ load vector), 1 mass, 2 anisotropic (values only; opk: their coefficients)
// op 3: y = A u matrix-free (the stiffness matrix with coefficient k; isbd: eliminated rows give u)
int assemble_tiles(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg, double* val,
                   double* b, cudaStream_t s, int op = 0, const double* opk = nullptr, const double* u = nullptr,
                   const uint8_t* isbd = nullptr, double* y = nullptr);
int tile_fused_smem(const TilePlan& T, int d);  // 0: the fused launch does not fit

// scratch doubles per element: stiffness unique entries + rhs entries (+ gradient entries)
inline int64_t scratch_per_elem(int d) { return d == 2 ? 9 : 14; }

// ---- device-wide exclusive scan of int32 counts -> int32 offsets (n+1 entries), total on host ----
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int64_t* total_host, cudaStream_t s);

// ---- kernels entry points (host launchers) ----------------------------------------------------------
int build_pattern(Pattern* P, const int32_t* elem_in, cudaStream_t s);
int assemble_values(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                    double* val, double* b, int variant, cudaStream_t s);
// Deterministic two-pass value path with caller-provided per-element scratch (scratch_per_elem(d) * NT
// doubles) and error word; allocates nothing.
int assemble_values_two_pass(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                              double* val, double* b, double* scratch, int* err, cudaStream_t s);
int* device_error_word_if_ready();  // the current device's error word, or nullptr if never allocated
int boundary_nodes(Pattern* P, const int8_t* bdflag, uint8_t* is_bd, cudaStream_t s);
int apply_dirichlet(const Pattern* P, const uint8_t* is_bd, const double* gD, double* val, double* b,
                    int32_t* free_node, int64_t* n_free, cudaStream_t s);
int boundary_terms(const Pattern* P, const double* node, const int8_t* bdflag, const double* g_side, double g_const,
                   double alpha, double* val, double* b, cudaStream_t s);
int side_points(const Pattern* P, const double* node, double* pts, cudaStream_t s);
int mean_shift(double* x, int64_t n, cudaStream_t s);
int zero_average(const Pattern* P, const double* node, double* u, double* c_out, cudaStream_t s);
int quad_rule(int d, int n, double* bary, double* w, int* nq);
int rhs_rule(const Pattern* P, const double* node, int n, int f_kind, const double* f_arg, double* b, cudaStream_t s);
int rule_points(const Pattern* P, const double* node, int n, double* pts, cudaStream_t s);
struct BatchPlan;
int assemble_backward(const Pattern* P, const double* node, const double* k, int f_kind, const double* f_arg,
                      const double* w, const double* r, double* gnode, double* gk, cudaStream_t s);

}  // namespace fem

struct fem_pattern_s {
  fem::Pattern P;
};
