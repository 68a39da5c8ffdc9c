// pospop_bulk.cuh -- one-dimensional bulk copies (cp.async.bulk, the
// non-tensor form of TMA) from global to shared memory with mbarrier
// completion, used by the staged kernels (the roofline read and the
// selected count).  Every wait is bounded.
#pragma once

#include <cstdint>

#include "pospop_internal.h"

namespace pospop {

constexpr uint32_t kBulkChunk = 8192;                  // bytes per chunk = 512 granules

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// This thread's arrival on the barrier's current phase, which then also
// waits for `bytes` bytes of bulk copies.
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Copy `bytes` from global to shared memory, completing them on the barrier
// (whose phase must expect them).  dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_copy_tx(uint32_t dst, const void *src, uint32_t bytes,
                                             uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// One copy that alone completes the barrier's current phase.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  mbar_expect(bar, bytes);
  bulk_copy_tx(dst, src, bytes, bar);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the barrier phase with the given parity to complete; false if it
// has not within `limit` SM clock cycles.  The clock is checked before each
// try, so a limit of 0 gives up without waiting at all (the kernels take
// their time-out exit on a healthy copy: that is how the exit is tested).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kBulkWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 >= limit) return false;
    if (mbar_try(bar, parity)) return true;
  }
}

}  // namespace pospop
