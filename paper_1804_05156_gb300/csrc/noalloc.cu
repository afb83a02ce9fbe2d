// Allocation-free assembly entry point (fem_assemble_noalloc).
//
// Some callers of this library cannot call cudaMalloc while they assemble. One example is an
// application that hands all device memory to its own pool at start-up. Another is a solver loop
// with a fixed latency budget, where an allocation's implicit device synchronisation is not
// acceptable. For them this entry point runs the deterministic two-pass value path (per-element
// values, then a fixed-order per-row sum) with its per-element scratch in a fixed device array
// compiled into the library, instead of scratch the library would allocate.
//
// The array below is a file-scope __device__ symbol. Every GPU that loads the library holds it
// (FEM_NOALLOC_SCRATCH_DOUBLES doubles = 16 MiB) until the process exits. Host code cannot use the
// symbol's name as a device address. Its address is taken with cudaGetSymbolAddress, once per
// device, the first time the entry point runs with that device current, and cached.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kScratchDoubles = FEM_NOALLOC_SCRATCH_DOUBLES;  // 16 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_na_mu;
double* g_na_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up on first use).
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fem::cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fem::set_error(FEM_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fem::cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return FEM_OK;
}

}  // namespace

extern "C" {

int fem_assemble_noalloc(fem_pattern_t p, const double* node, const double* k, int f_kind, const double* f_arg,
                         double* val, double* b, fem_stream_t stream) {
  if (!p) return fem::set_error(FEM_ERR_ARG, "null pattern");
  const fem::Pattern& P = p->P;
  if (P.NT > 0 && !node) return fem::set_error(FEM_ERR_ARG, "null node array");
  if (((uintptr_t)node | (uintptr_t)k | (uintptr_t)f_arg | (uintptr_t)val | (uintptr_t)b) % 8 != 0)
    return fem::set_error(FEM_ERR_ARG, "misaligned double array");
  if (f_kind != FEM_F_CONST && f_kind != FEM_F_SINPROD && f_kind != FEM_F_QPVALUES)
    return fem::set_error(FEM_ERR_ARG, "unknown f_kind %d", f_kind);
  if (f_kind == FEM_F_QPVALUES && !f_arg && P.NT > 0) return fem::set_error(FEM_ERR_ARG, "FEM_F_QPVALUES needs f_arg");
  const int64_t need = fem::scratch_per_elem(P.d) * P.NT;
  if (need > kScratchDoubles)
    return fem::set_error(FEM_ERR_ARG,
                          "mesh too large for the allocation-free path: %lld elements, at most %lld for d = %d",
                          (long long)P.NT, (long long)(kScratchDoubles / fem::scratch_per_elem(P.d)), P.d);
  if (!val && !b) return FEM_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P.device)
    return fem::set_error(FEM_ERR_STATE, "the pattern was built on device %d, not the current device", P.device);
  int* err = fem::device_error_word_if_ready();
  if (!err) return fem::set_error(FEM_ERR_STATE, "no pattern was built on the current device");
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  return fem::assemble_values_two_pass(&P, node, k, f_kind, f_arg, val, b, scratch, err, (cudaStream_t)stream);
}

}  // extern "C"
