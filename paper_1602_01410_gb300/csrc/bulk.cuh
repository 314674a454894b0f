// Bulk asynchronous copies from global to shared memory (the TMA engine's
// untiled form, cp.async.bulk), completed on a shared-memory mbarrier, and a
// bounded wait on that barrier.
//
// Use: one thread initialises the barrier (one expected arrival), a CTA
// barrier makes the initialisation visible, the same thread announces the
// byte count (arrive.expect_tx) and issues the copies; the consumers wait on
// phase 0.  Every address is 16-byte aligned and every size a multiple of
// 16 bytes (checked by the callers at compile time or on the host).
#pragma once

#include <cstdint>

namespace dcv {

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bound of the wait for copies still in flight after a wait ran out (they
// complete in microseconds), independent of the caller's limit so that a
// block never leaves while a copy into its shared memory is pending.
constexpr long long kDrainNs = 1000000000LL;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Barrier with one expected arrival per phase (the issuing thread's).
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The issuing thread's arrival, announcing `bytes` of copies that complete
// the phase (at most 2^20 - 1 bytes per phase).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// `bytes` (a multiple of 16) from 16-byte aligned global `src` to 16-byte
// aligned shared `dst`; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Prefetch into L2 (a hint with no completion to wait for) of the 16-byte
// granules covering [src, src + bytes): the span is widened to 16-byte
// boundaries, as the bulk prefetch requires, so the caller's buffer must
// own the granules around its ends (the plan's buffers start on 256-byte
// boundaries and are padded to them).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
  const uintptr_t e = (reinterpret_cast<uintptr_t>(src) + bytes + 15) & ~uintptr_t(15);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// True once the phase of the given parity has completed.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity; false when limit_ns nanoseconds
// passed first (the clock is read before the barrier, so a limit of 0 never
// waits).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if ((long long)(global_ns() - t0) >= limit_ns) return false;
    if (mbar_test(bar, parity)) return true;
  }
}

}  // namespace dcv
