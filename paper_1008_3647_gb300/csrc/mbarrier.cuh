// Shared-memory addresses and mbarriers (PTX wrappers of the TMA-staged kernels).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ufg {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of bar for at most `limit` try_wait rounds.  When the rounds run out it
// raises *err (when given) and returns false: the caller then goes on with whatever shared memory
// holds, and the host reports the raised flag as UFG_TIMEOUT for the whole call.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit,
                                                  int* err) {
  for (uint32_t n = 0; !mbar_try_wait(bar, parity);) {
    if (++n > limit) {
      if (err != nullptr) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

// Test hook behind ufg_test_expire_waits: one bounded wait that is made to run out.  A second
// mbarrier expects 16 bytes that no copy will ever deliver, so its phase cannot complete; the
// wait gives up after `limit` rounds and raises the flag exactly as a real timeout would.  The
// slice's own copies complete on their own barrier, so nothing is left in flight.  Thread 0 only.
__device__ __forceinline__ void mbar_expire_one_wait(uint64_t* bar2, uint32_t limit, int* err) {
  mbar_init(bar2, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_expect_tx(bar2, 16u);
  mbar_wait_bounded(bar2, 0u, limit, err);
}

}  // namespace ufg
