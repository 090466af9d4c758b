// gp_async.cuh -- mbarrier and bulk-copy helpers shared by the kernels that
// stage global memory in shared memory through the tensor memory accelerator
// (the TMA z sweep, the bulk-copy observables reduction of real fields, the
// bounded-wait self-test).  Hand-written inline PTX of the documented instruction forms.
#pragma once

#include <stdint.h>

namespace gpcn {

// Bound of every mbarrier wait: about a second of SM clock cycles.
constexpr long long kSpinCycles = 1LL << 31;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of `bar` with the given parity, for at most `cycles`
// clock cycles (none at all once `ok` is false).  Returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, bool ok,
                                                  long long cycles = kSpinCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    if (!ok) return false;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// One untiled bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) from global memory into this CTA's shared memory,
// completing on the transaction count of mbarrier `bar`.
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace gpcn
