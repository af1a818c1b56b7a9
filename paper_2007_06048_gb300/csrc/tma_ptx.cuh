// Inline PTX of the TMA-pipelined kernels: shared-memory mbarriers with
// transaction counts, bounded waits on them, tiled bulk-tensor loads
// (cp.async.bulk.tensor) and the acquire / release and proxy fences of the
// persistent kernel.  Every wait is bounded: it gives up after kWaitNs of
// %globaltimer, records the failure and lets the kernel return.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace mmod {
namespace {

constexpr unsigned long long kWaitNs = 100000000ull;   // a wait gives up after 100 ms

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's view of global memory (generic proxy) before its
// later bulk-tensor copies (async proxy).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase for at most kWaitNs of wall-clock time (try_wait suspends
// the thread in hardware between polls).  The slow path gives up at once if
// another CTA already reported a failure.  On give-up it records the failure
// and returns false.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity, int *abort_flag, int *err) {
    const unsigned long long t0 = global_ns();
    while (!(err && *(volatile int *)err) && global_ns() - t0 < kWaitNs)
        if (mbar_try_wait(bar, parity)) return true;
    *abort_flag = 1;
    if (err) atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *abort_flag, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, abort_flag, err);
}

// Bounded drain wait used after a give-up: no error reporting.
__device__ __noinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < kWaitNs)
        if (mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace
}  // namespace mmod
