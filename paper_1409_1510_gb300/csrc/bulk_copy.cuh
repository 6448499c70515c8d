// Shared-memory staging with the bulk-copy engine (cp.async.bulk) and mbarriers, in inline PTX.
//
// One thread of a block issues 1-D bulk copies global -> shared that signal an mbarrier with
// the bytes they deliver; the block's threads wait on the barrier's phase.  Every wait is
// bounded: after `limit` polls it gives up and returns false (the caller records the failure
// and skips the work that depended on the copy), so a lost transfer can never hang the GPU.
// Addresses and sizes of a bulk copy are multiples of 16 bytes.
#pragma once
#include <stdint.h>

namespace hisq {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
}

// make the initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` more bytes to be delivered in the current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned) completing on bar
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// wait for the phase with the given parity to complete; false after `limit` unsuccessful polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long limit) {
    const uint32_t a = smem_addr(bar);
    for (long i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace hisq
