// Assembly from and to host memory: a sequence of assemblies of one pattern, pipelined over three
// streams.
//
// Step i uses device buffer set x = i mod 2 (node, k, val, b):
//   input stream:  wait until step i-2 has finished computing from set x; copy node_h[i], k_h[i] in;
//   caller stream: wait for those copies and for the output copies of step i-2 from set x; assemble
//                  (fem_assemble, deterministic path) into set x;
//   output stream: wait for the assembly; copy val and b out to val_h[i], b_h[i].
// So the input copies of step i+1 and the output copies of step i-1 run while step i computes, and
// the two copy directions run at once. The call returns when every output is in host memory; later
// work on the caller's stream is ordered after it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace fem {

struct HostExec {
  int device = -1;
  int64_t N = 0, NT = 0, nnz = 0;
  int d = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t entry = nullptr, join = nullptr;
  cudaEvent_t in_ready[2] = {}, computed[2] = {}, out_done[2] = {};
  double* node[2] = {};
  double* k[2] = {};
  double* val[2] = {};
  double* b[2] = {};
};

void free_host_exec(Pattern& P) {
  HostExec* h = P.hx;
  if (!h) return;
  if (h->s_in) cudaStreamSynchronize(h->s_in);
  if (h->s_out) cudaStreamSynchronize(h->s_out);
  for (int x = 0; x < 2; ++x) {
    cudaFree(h->node[x]);
    cudaFree(h->k[x]);
    cudaFree(h->val[x]);
    cudaFree(h->b[x]);
    if (h->in_ready[x]) cudaEventDestroy(h->in_ready[x]);
    if (h->computed[x]) cudaEventDestroy(h->computed[x]);
    if (h->out_done[x]) cudaEventDestroy(h->out_done[x]);
  }
  if (h->entry) cudaEventDestroy(h->entry);
  if (h->join) cudaEventDestroy(h->join);
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  delete h;
  P.hx = nullptr;
}

namespace {

bool aligned8(const void* q) { return ((uintptr_t)q % 8) == 0; }

// The pattern's host-step resources, made on first use: two streams, the events, and two sets of
// device buffers (2 x (N d + NT + nnz + N) doubles).
int ensure_host_exec(Pattern& P, HostExec** out) {
  if (P.hx) {
    *out = P.hx;
    return FEM_OK;
  }
  HostExec* h = new HostExec();
  h->device = P.device;
  h->N = P.N;
  h->NT = P.NT;
  h->nnz = P.nnz;
  h->d = P.d;
  P.hx = h;
  cudaError_t e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->entry, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
  for (int x = 0; x < 2 && e == cudaSuccess; ++x) {
    e = cudaEventCreateWithFlags(&h->in_ready[x], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->computed[x], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->out_done[x], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_host_exec(P);
    return cuda_error(e, "host step streams and events");
  }
  for (int x = 0; x < 2 && e == cudaSuccess; ++x) {
    e = cudaMalloc((void**)&h->node[x], sizeof(double) * (size_t)(P.N * P.d > 0 ? P.N * P.d : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->k[x], sizeof(double) * (size_t)(P.NT > 0 ? P.NT : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->val[x], sizeof(double) * (size_t)(P.nnz > 0 ? P.nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->b[x], sizeof(double) * (size_t)(P.N > 0 ? P.N : 1));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_host_exec(P);
    return set_error(FEM_ERR_OOM, "cannot allocate the host-step device buffers");
  }
  *out = h;
  return FEM_OK;
}

}  // namespace
}  // namespace fem

using fem::HostExec;

extern "C" int fem_assemble_host(fem_pattern_t p, int steps, const double* const* node_h, const double* const* k_h,
                                 int f_kind, const double* f_arg, double* const* val_h, double* const* b_h,
                                 fem_stream_t stream) {
  if (!p) return fem::set_error(FEM_ERR_ARG, "null pattern");
  if (steps < 0) return fem::set_error(FEM_ERR_ARG, "negative step count");
  if (steps == 0) return FEM_OK;
  fem::Pattern& P = p->P;
  if (!node_h) return fem::set_error(FEM_ERR_ARG, "null node_h");
  for (int i = 0; i < steps; ++i) {
    if (!node_h[i] && P.NT > 0) return fem::set_error(FEM_ERR_ARG, "null node_h[%d]", i);
    if (!fem::aligned8(node_h[i]) || (k_h && !fem::aligned8(k_h[i])) || (val_h && !fem::aligned8(val_h[i])) ||
        (b_h && !fem::aligned8(b_h[i])))
      return fem::set_error(FEM_ERR_ARG, "misaligned host array in step %d", i);
  }
  HostExec* h = nullptr;
  int rc = fem::ensure_host_exec(P, &h);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = sizeof(double) * (size_t)(P.N * P.d), kb = sizeof(double) * (size_t)P.NT;
  const size_t vb = sizeof(double) * (size_t)P.nnz, bb = sizeof(double) * (size_t)P.N;
  cudaError_t e = cudaEventRecord(h->entry, s);  // earlier work on the caller's stream comes first
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_in, h->entry, 0);
  for (int i = 0; i < steps && e == cudaSuccess && rc == FEM_OK; ++i) {
    const int x = i & 1;
    const bool hk = k_h && k_h[i];
    const bool wv = val_h && val_h[i], wb = b_h && b_h[i];
    // inputs of step i (set x is free once step i-2 has computed)
    e = cudaStreamWaitEvent(h->s_in, h->computed[x], 0);
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(h->node[x], node_h[i], nb, cudaMemcpyHostToDevice, h->s_in);
    if (e == cudaSuccess && hk && kb) e = cudaMemcpyAsync(h->k[x], k_h[i], kb, cudaMemcpyHostToDevice, h->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->in_ready[x], h->s_in);
    // the assembly (its outputs in set x are free once step i-2's copies out are done)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->in_ready[x], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->out_done[x], 0);
    if (e != cudaSuccess) break;
    rc = fem_assemble(p, h->node[x], hk ? h->k[x] : nullptr, f_kind, f_arg, wv ? h->val[x] : nullptr,
                      wb ? h->b[x] : nullptr, FEM_DETERMINISTIC, stream);
    if (rc) break;
    e = cudaEventRecord(h->computed[x], s);
    // outputs of step i
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->computed[x], 0);
    if (e == cudaSuccess && wv && vb) e = cudaMemcpyAsync(val_h[i], h->val[x], vb, cudaMemcpyDeviceToHost, h->s_out);
    if (e == cudaSuccess && wb && bb) e = cudaMemcpyAsync(b_h[i], h->b[x], bb, cudaMemcpyDeviceToHost, h->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(h->out_done[x], h->s_out);
  }
  // join: later work on the caller's stream follows the last copies out; wait for them here
  cudaError_t j = cudaEventRecord(h->join, h->s_out);
  if (j == cudaSuccess) j = cudaStreamWaitEvent(s, h->join, 0);
  const cudaError_t si = cudaStreamSynchronize(h->s_in);
  const cudaError_t so = cudaStreamSynchronize(h->s_out);
  if (rc) return rc;
  if (e != cudaSuccess) return fem::cuda_error(e, "host step copies");
  if (j != cudaSuccess) return fem::cuda_error(j, "host step join");
  if (si != cudaSuccess) return fem::cuda_error(si, "host step input stream");
  if (so != cudaSuccess) return fem::cuda_error(so, "host step output stream");
  return FEM_OK;
}
