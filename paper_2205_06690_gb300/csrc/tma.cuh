// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with mbarrier completion, and a
// wall-clock-bounded wait. A wait that runs out reports false; the caller sets its error flag and
// waits (again bounded) for the copies it still has in flight before the block exits.
#pragma once
#include <stdint.h>

namespace sbse {

__device__ __forceinline__ uint32_t tma_smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_bar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tma_smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of transaction for the current phase
__device__ __forceinline__ void tma_bar_expect(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tma_smem_addr(bar)), "r"(bytes)
               : "memory");
}

// global -> shared bulk copy; dst, src and bytes must be multiples of 16
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tma_smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(tma_smem_addr(bar))
      : "memory");
}

// order earlier generic-proxy accesses of shared memory before later async-proxy (bulk copy) ones
__device__ __forceinline__ void tma_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t tma_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool tma_bar_test(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(tma_smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the completion of the phase with the given parity; false after `limit_ns` (default 1 s)
__device__ __forceinline__ bool tma_bar_wait(uint64_t *bar, unsigned parity,
                                             uint64_t limit_ns = 1000000000ull) {
  if (tma_bar_test(bar, parity)) return true;
  const uint64_t t0 = tma_now_ns();
  while (!tma_bar_test(bar, parity))
    if (tma_now_ns() - t0 > limit_ns) return false;
  return true;
}

}  // namespace sbse
