// mbarrier and TMA (cp.async.bulk.tensor) wrappers for sm_103a, with bounded waits.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace dwt {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Invalidate a barrier whose phases have all completed, before it is
// initialised again for another work item.
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Data another thread wrote with ordinary stores and published through an
// acquired flag: order that acquire before this thread's later TMA reads of
// global memory.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Wait until *flag >= target (acquire, GPU scope); give up after `budget`
// clock cycles.  Spins with a short sleep between reads.  The comparison is
// modulo 2^32 (counters that grow over many calls may wrap).
__device__ __forceinline__ bool wait_counter_bounded(const int* flag, int target, long long budget) {
    const long long t0 = clock64();
    for (;;) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if ((int)((unsigned)v - (unsigned)target) >= 0) return true;
        if (clock64() - t0 > budget) return false;
        __nanosleep(256);
    }
}

// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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

// Wait for phase `parity` of the barrier; give up after `budget` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long budget) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// 2-D tiled TMA load of a box at element coordinates (x, y) into shared
// memory; completion is signalled on the barrier as transferred bytes.
// x * element size must be a multiple of 16 bytes; out-of-range elements
// (negative or past the tensor) are filled with zeros.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// A tensor map written to global memory by the host (a copy before the
// launch) is read by the TMA unit through the tensor-map proxy: acquire it
// there before the first copy that uses it.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// Programmatic dependent launch.  A grid launched with programmatic stream
// serialization may become resident while the kernel before it in the stream
// is still draining; griddepcontrol.wait blocks the calling thread until every
// prerequisite grid has completed and its memory is visible (it returns at
// once for a grid launched without the attribute).  launch_dependents lets the
// next such grid be scheduled once every CTA of this one has issued it or
// exited.  Both are issued by every thread before its first global access.
__device__ __forceinline__ void grid_dependency_sync() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The two halves, for kernels that set up their registers (from parameters
// only) between them: launch_dependents first, wait before the first global
// access.
__device__ __forceinline__ void grid_dependents_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// About one second at GB300 clocks.
constexpr long long kWaitBudget = 2000000000LL;

}  // namespace dwt
