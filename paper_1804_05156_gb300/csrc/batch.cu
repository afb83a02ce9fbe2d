// Batched assembly of many independent meshes: one block-diagonal pattern for all meshes, one value
// pass over all their elements, and a CUDA graph that replays it.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "common.cuh"

struct fem_batch_s {
  int d = 0, B = 0, device = 0;
  std::vector<int64_t> node_off, elem_off, nnz_off;
  fem_pattern_t pat = nullptr;
  // captured graph and the arguments it was captured with
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  const void* gargs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int gkind = -1, gvariant = -1;
  int64_t graph_kernels = 0;  // kernels per replay (counted at capture)
};

namespace {

using fem::set_error;

// vertex ids of mesh m's elements become global: add node_off[m] (m found by binary search)
__global__ void k_offset_elem(const int32_t* __restrict__ in, int32_t* __restrict__ out, int d1,
                              const int64_t* __restrict__ elem_off, const int64_t* __restrict__ node_off, int B,
                              int64_t NT) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < NT; t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (elem_off[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const int64_t off = node_off[lo];
    for (int i = 0; i < d1; ++i) out[t * d1 + i] = (int32_t)(in[t * d1 + i] + off);
  }
}

// group id of every vertex: the mesh it belongs to (binary search over the vertex offsets)
__global__ void k_vertex_group(const int64_t* __restrict__ node_off, int B, int64_t N, int32_t* __restrict__ group) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (node_off[mid] <= v) lo = mid;
      else hi = mid - 1;
    }
    group[v] = lo;
  }
}

}  // namespace

extern "C" {

int fem_batch_set_locality(fem_batch_t bt, const double* node_cat, fem_stream_t stream) {
  if (!bt) return set_error(FEM_ERR_ARG, "null batch");
  if (((uintptr_t)node_cat) % 8 != 0) return set_error(FEM_ERR_ARG, "misaligned node_cat");
  const int64_t N = bt->node_off[bt->B];
  if (N == 0) return FEM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* doff = nullptr;
  int32_t* group = nullptr;
  if (cudaMallocAsync((void**)&doff, sizeof(int64_t) * (bt->B + 1), s) != cudaSuccess ||
      cudaMallocAsync((void**)&group, sizeof(int32_t) * N, s) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FEM_ERR_OOM, "batch locality allocation failed");
  }
  cudaMemcpyAsync(doff, bt->node_off.data(), sizeof(int64_t) * (bt->B + 1), cudaMemcpyHostToDevice, s);
  k_vertex_group<<<fem::grid_for(N, 256), 256, 0, s>>>(doff, bt->B, N, group);
  fem::g_launches.fetch_add(1);
  int rc = fem_pattern_set_locality(bt->pat, node_cat, group, stream);
  cudaStreamSynchronize(s);
  cudaFree(doff);
  cudaFree(group);
  // a re-planned batch invalidates any captured graph
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->exec = nullptr;
  bt->graph = nullptr;
  return rc;
}


int fem_batch_plan(int d, int B, const int64_t* N, const int64_t* NT, const int32_t* elem_cat, fem_batch_t* out,
                   fem_stream_t stream) {
  if (!out) return set_error(FEM_ERR_ARG, "null output handle");
  *out = nullptr;
  if ((d != 2 && d != 3) || B <= 0 || !N || !NT) return set_error(FEM_ERR_ARG, "bad batch arguments");
  fem_batch_s* h = new (std::nothrow) fem_batch_s();
  if (!h) return set_error(FEM_ERR_OOM, "host allocation failed");
  h->d = d;
  h->B = B;
  cudaGetDevice(&h->device);
  h->node_off.assign(B + 1, 0);
  h->elem_off.assign(B + 1, 0);
  for (int m = 0; m < B; ++m) {
    if (N[m] < 0 || NT[m] < 0) {
      delete h;
      return set_error(FEM_ERR_ARG, "negative size in mesh %d", m);
    }
    h->node_off[m + 1] = h->node_off[m] + N[m];
    h->elem_off[m + 1] = h->elem_off[m] + NT[m];
  }
  const int64_t Ntot = h->node_off[B], NTtot = h->elem_off[B];
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* eg = nullptr;
  int64_t* doff = nullptr;
  int rc = FEM_OK;
  if (NTtot > 0) {
    if (!elem_cat) {
      delete h;
      return set_error(FEM_ERR_ARG, "null elem_cat");
    }
    if (cudaMalloc((void**)&eg, sizeof(int32_t) * (size_t)NTtot * (d + 1)) != cudaSuccess ||
        cudaMalloc((void**)&doff, sizeof(int64_t) * (size_t)(2 * (B + 1))) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(eg);
      delete h;
      return set_error(FEM_ERR_OOM, "batch plan allocation failed");
    }
    cudaMemcpyAsync(doff, h->elem_off.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(doff + B + 1, h->node_off.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s);
    k_offset_elem<<<fem::grid_for(NTtot, 256), 256, 0, s>>>(elem_cat, eg, d + 1, doff, doff + B + 1, B, NTtot);
    fem::g_launches.fetch_add(1);
    if (cudaGetLastError() != cudaSuccess) rc = set_error(FEM_ERR_CUDA, "offset kernel launch failed");
  }
  if (rc == FEM_OK) rc = fem_mesh_build_pattern(d, Ntot, NTtot, eg, &h->pat, stream);
  cudaStreamSynchronize(s);
  cudaFree(eg);
  cudaFree(doff);
  if (rc != FEM_OK) {
    delete h;
    return rc;
  }
  // the batch runs in one launch (the fused tile form or the persistent blocked form)
  h->pat->P.one_launch = true;
  fem::enforce_one_launch(&h->pat->P);
  // nnz offsets: row_ptr at the mesh boundaries
  h->nnz_off.assign(B + 1, 0);
  std::vector<int32_t> rp((size_t)Ntot + 1);
  if (cudaMemcpy(rp.data(), h->pat->P.row_ptr, sizeof(int32_t) * (Ntot + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
    fem_pattern_destroy(h->pat);
    delete h;
    return set_error(FEM_ERR_CUDA, "row_ptr copy failed");
  }
  for (int m = 0; m <= B; ++m) h->nnz_off[m] = rp[h->node_off[m]];
  *out = h;
  return FEM_OK;
}

int fem_batch_info(fem_batch_t bt, int* B, const int64_t** node_off, const int64_t** elem_off, const int64_t** nnz_off,
                   fem_pattern_t* pattern) {
  if (!bt) return set_error(FEM_ERR_ARG, "null batch");
  if (B) *B = bt->B;
  if (node_off) *node_off = bt->node_off.data();
  if (elem_off) *elem_off = bt->elem_off.data();
  if (nnz_off) *nnz_off = bt->nnz_off.data();
  if (pattern) *pattern = bt->pat;
  return FEM_OK;
}

int fem_batch_assemble(fem_batch_t bt, const double* node_cat, const double* k_cat, int f_kind, const double* f_arg,
                       double* val_cat, double* b_cat, int variant, fem_stream_t stream) {
  if (!bt) return set_error(FEM_ERR_ARG, "null batch");
  return fem_assemble(bt->pat, node_cat, k_cat, f_kind, f_arg, val_cat, b_cat, variant, stream);
}

int fem_batch_assemble_graph(fem_batch_t bt, const double* node_cat, const double* k_cat, int f_kind,
                             const double* f_arg, double* val_cat, double* b_cat, int variant, fem_stream_t stream) {
  if (!bt) return set_error(FEM_ERR_ARG, "null batch");
  const void* args[6] = {node_cat, k_cat, f_arg, val_cat, b_cat, nullptr};
  bool same = bt->exec && bt->gkind == f_kind && bt->gvariant == variant;
  for (int i = 0; i < 5 && same; ++i) same = args[i] == bt->gargs[i];
  if (!same) {
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    bt->exec = nullptr;
    bt->graph = nullptr;
    if (!bt->cap_stream && cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fem::cuda_error(cudaGetLastError(), "capture stream");
    // the capture stream must see the caller's prior work; order it after the caller's stream
    cudaStreamSynchronize((cudaStream_t)stream);
    if (cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fem::cuda_error(cudaGetLastError(), "begin capture");
    const int64_t before = fem::g_launches.load();
    int rc = fem_assemble(bt->pat, node_cat, k_cat, f_kind, f_arg, val_cat, b_cat, variant, bt->cap_stream);
    bt->graph_kernels = fem::g_launches.load() - before;
    fem::g_launches.fetch_sub(bt->graph_kernels);  // counted when replayed
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(bt->cap_stream, &g);
    if (rc != FEM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fem::cuda_error(e, "end capture");
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return fem::cuda_error(e, "graph instantiate");
    }
    bt->graph = g;
    for (int i = 0; i < 5; ++i) bt->gargs[i] = args[i];
    bt->gkind = f_kind;
    bt->gvariant = variant;
  }
  cudaError_t e = cudaGraphLaunch(bt->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fem::cuda_error(e, "graph launch");
  fem::g_launches.fetch_add(bt->graph_kernels);
  return FEM_OK;
}

void fem_batch_destroy(fem_batch_t bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
  fem_pattern_destroy(bt->pat);
  delete bt;
}

}  // extern "C"
