// tma.cuh -- tensor-memory-accelerator (TMA) tile loads with mbarrier
// completion, for the persistent strided passes (sm_103a inline PTX).
//
// A strided pass reads a tile of W adjacent pencils: L rows of W complex
// values (64 bytes) at a fixed row pitch.  Seen as a 2D tensor (inner axis =
// the contiguous index, outer axis = the pencil axis), the tile is one box of
// W x L elements of 8 bytes, fetched by cp.async.bulk.tensor in boxes of at
// most 256 rows into a dense [L][W] staging buffer.  Completion is tracked
// by one mbarrier per CTA (arrive.expect_tx by the issuing thread, complete_tx
// by the copy engine).  Every wait is bounded in time: past the limit the
// kernel records an error for the host and stops.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace ffcz {

// Device error codes written to the plan's error word.
enum DevErr : int { DERR_NONE = 0, DERR_TMA_TIMEOUT = 1, DERR_TMA_ALIGN = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also raises the expected transaction bytes of the phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Poll the phase of the given parity until it completes or `limit` SM
// cycles have passed (each poll may suspend the thread for a short,
// system-dependent time, so the bound is on elapsed cycles, not polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (copy engine) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Box load of the 2D tensor `map` at element coordinates (x, y) into dst
// (128-byte aligned shared memory), completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Contiguous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// SM cycles before a wait gives up (about 2 s at 2 GHz): far longer than any
// tile load, short enough to return promptly.
constexpr long long kTmaPollLimit = 4000000000LL;

}  // namespace ffcz
