// 32-byte packets in one 256-bit global access (PTX ld/st .v8.f32; the address must be 32-byte aligned,
// which the callers' packet buffers are, and the launchers check).
//
// The value and backward kernels exchange per-incidence packets through global memory: the element
// phase writes one packet per element-row at a scattered slot, and a per-row pass reads a row's packets
// in order. Both sides are limited by the L1 data path's work for these scattered accesses, which is
// one request per access: a single 256-bit access per packet instead of two 128-bit halves halves it.
#pragma once

#include <cuda_runtime.h>

namespace fem {

// FRESH: the packet was written earlier in the same launch, so read it through L2 (.cg); otherwise
// through the read-only path (.nc), without allocating it in L1: every 32-byte packet is read once, so
// an L1 copy is never used again and only costs the L1 the allocation
template <bool FRESH>
__device__ __forceinline__ void load_packet32(const float4* p, float4& a, float4& b) {
  if constexpr (FRESH)
    asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
  else
    asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

__device__ __forceinline__ void store_packet32(float4* p, const float4& a, const float4& b) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
               "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}

}  // namespace fem
