// kx_ptx.cuh -- inline-PTX helpers shared by the contraction kernels: shared
// memory addresses, mbarriers with bounded waits and bulk (TMA) copies.
#pragma once

#include <stdint.h>

#define KX_WAIT_CYCLES (4ll << 30)  // bounded mbarrier wait, about 2 s

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while its predecessor in the stream still runs:
// kx_pdl_wait blocks until the predecessor grid has completed and its memory
// operations are visible (it returns at once for an ordinary launch), and
// kx_pdl_trigger allows the successor's blocks to be scheduled.  Work before
// the wait may read only data that no earlier kernel of the sequence writes.
__device__ __forceinline__ void kx_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void kx_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t kx_smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void kx_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void kx_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool kx_mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity; gives up after `limit` SM clock
// cycles (KX_WAIT_CYCLES unless a caller asks for less) and returns false.
__device__ __forceinline__ bool kx_mbar_wait(uint32_t bar, uint32_t parity,
                                             long long limit = KX_WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!kx_mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void kx_bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void kx_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Makes mbarrier initialisation visible to the async proxy.
__device__ __forceinline__ void kx_fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
