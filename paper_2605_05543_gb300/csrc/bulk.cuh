// Bulk copies of contiguous global runs into shared memory by the TMA engine (cp.async.bulk), completed
// on an mbarrier with a transaction count, and a bounded wait on that barrier.
//
// Rules the callers keep: source and destination 16-byte aligned and the size a multiple of 16 bytes;
// one arrive.expect_tx of exactly the bytes of the copies that complete on the barrier, issued before
// them; the barrier initialised by one thread and made visible to the async proxy (fence_mbar_init)
// before the block synchronises and the first copy is issued. The copies read this GPU's own memory and
// target the issuing block's shared memory only (no cluster, no multicast).
#pragma once

#include <stdint.h>

namespace emppp {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(arrivals) : "memory");
}

// makes mbarrier initialisations of this thread visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// the one arrival of the phase, announcing `bytes` of copies that will complete on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// suspend-time hint of one probe (ns): the longest a probe keeps the thread waiting for the phase
constexpr uint32_t kProbeNs = 1000;

// one probe of the phase with the given parity; true once that phase has completed
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kProbeNs)
      : "memory");
  return ok != 0;
}

// at most `limit` probes of at most kProbeNs each; false if the phase has not completed by then
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace emppp
