// Tensor Memory Accelerator (TMA) building blocks for sm_103a, as inline PTX: tiled bulk-tensor copies between
// global and shared memory described by a CUtensorMap (a kernel parameter declared __grid_constant__), completion
// of loads on an mbarrier with an expected transaction byte count, and bulk-group completion of stores.
// The copies bypass the load/store units: staging a kernel's streamed operands this way takes them off the L1
// data pipe that the shared-memory taps of the semi-Lagrangian gathers already load.
#pragma once
#include <cuda.h>

#include <cstdint>

namespace claire {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// one arrival on the barrier that also announces `bytes` of transactions still to come
__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// tiled loads: the box at the given element coordinates (innermost first) lands densely at dst; out-of-range
// elements are filled with zeros
__device__ __forceinline__ void load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                      uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void load5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                      uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// tiled store of a dense shared-memory box (elements outside the tensor are not written); the coordinates are
// never negative here
__device__ __forceinline__ void store4(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
               : "memory");
}
__device__ __forceinline__ void store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the committed stores have read their shared-memory source (the CTA may then exit or reuse it)
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// make this thread's ordinary shared-memory writes visible to the bulk copies (the async proxy)
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tma
}  // namespace claire
