// Bulk asynchronous copies (cp.async.bulk, sm_90 and later) from global to
// shared memory, their completion counted in bytes on an mbarrier: one
// thread announces the bytes a phase expects (arrive.expect_tx) and issues
// the copies; every thread that reads the data waits for the phase.
// Source and destination addresses and sizes are multiples of 16 bytes.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace kkt {
namespace bulk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// an mbarrier expecting one arrival per phase (the expect_tx below)
__device__ __forceinline__ void init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
// make the initialised barriers (and, after a barrier that ordered every
// thread's reads of a buffer, those reads) ordered before later copies
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// arrive on `bar` and add `bytes` to the transaction count of its phase
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` bytes, counted on `bar`
__device__ __forceinline__ void g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Wait for the phase of `bar` with parity `parity`; gives up after `limit`
// clock cycles and returns false then.
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

}  // namespace bulk
}  // namespace kkt
