// Inverse transform over many images: the batched kernel (one launch per
// level group, fusion depth and storage type) and the persistent queue kernel
// (one launch per storage type), with 2 or 4 quadruple columns per lane.  See
// the forward batch kernels for the table and the queue.
#include "dwt_inv_body.cuh"

namespace dwt {

// arguments in registers (not the constant bank): 12 warps per SM
template <class S, int SCH, int NL, int Q1>
__global__ void __launch_bounds__(kInvWarps * 32, 12 / kInvWarps)
    inv_batched_kernel(const BatchEntry* __restrict__ table, int n) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    grid_dependency_sync();
    const int gw = blockIdx.x * kInvWarps + (threadIdx.x >> 5);
    const BatchEntry& e = table[find_entry(table, n, gw)];
    const int wid = gw - e.first_warp;
    const FusedArgs a = e.args;  // registers: the body's stores cannot alias it
    if (wid < 0 || wid >= a.nstrips * a.nsegs) return;
    fence_tensormap_acquire(&e.m[0]);
    fence_tensormap_acquire(&e.m[1]);
    fence_tensormap_acquire(&e.m[2]);
    inv_body<S, SCH, NL, Q1>(&e.m[0], &e.m[1], &e.m[2], a, wid, smem_raw);
}

// Persistent form over a queue of work items; items are ordered by level
// group, so the bounded wait for the group an item depends on always ends
// unless a warp failed, and then the status word already says so.
template <class S, int SCH, int Q1>
__global__ void __launch_bounds__(kInvWarps * 32, inv_queue_resident(Q1) / kInvWarps)
    inv_queue_kernel(const BatchEntry* __restrict__ table, int n, int total, int* head, int* done,
                     int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    grid_dependency_sync();
    const int lane = threadIdx.x & 31;
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(head, 1);
        g = __shfl_sync(kFull, g, 0);
        if (g >= total) break;
        const BatchEntry& e = table[find_entry(table, n, g)];
        const FusedArgs a = e.args;
        const int wid = g - e.first_warp;
        bool ok = true;
        if (e.dep >= 0) {
            if (lane == 0) {
                ok = wait_counter_bounded(done + e.dep, e.dep_items, kWaitBudget);
                if (ok) fence_proxy_async_global();
                else atomicExch(err, -6);
            }
            ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
        }
        if (ok) {
            fence_tensormap_acquire(&e.m[0]);
            fence_tensormap_acquire(&e.m[1]);
            fence_tensormap_acquire(&e.m[2]);
            ok = e.nl == 2 ? inv_body<S, SCH, 2, Q1>(&e.m[0], &e.m[1], &e.m[2], a, wid, smem_raw)
                           : inv_body<S, SCH, 1, Q1>(&e.m[0], &e.m[1], &e.m[2], a, wid, smem_raw);
        }
        __syncwarp();
        if (!ok) break;  // copies may still be in flight: stop using the ring
        if (lane == 0) {
            __threadfence();  // this item's stores before its count
            atomicAdd(done + e.self, 1);
        }
    }
}

// The ring of the larger of the two fusion depths.
static size_t inv_queue_smem(int elem_bytes, int q1) {
    const size_t a = inv_tma_smem_bytes(elem_bytes, 1, q1), b = inv_tma_smem_bytes(elem_bytes, 2, q1);
    return a > b ? a : b;
}

template <class S, int SCH, int Q1>
static cudaError_t inv_queue_one(const BatchEntry* table, int n, int total, int* head, int* done,
                                 int* err, int grid, cudaStream_t st) {
    auto k = inv_queue_kernel<S, SCH, Q1>;
    const size_t smem = inv_queue_smem(sizeof(S), Q1);
    if (grid == 0)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_kernel(k, grid, kInvWarps * 32, smem, st, false, table, n, total, head, done, err);
}

template <class S, int SCH>
static cudaError_t inv_queue_q(int q1, const BatchEntry* table, int n, int total, int* head, int* done,
                               int* err, int grid, cudaStream_t st) {
    if (q1 == 2) return inv_queue_one<S, SCH, 2>(table, n, total, head, done, err, grid, st);
    if (q1 == 4) return inv_queue_one<S, SCH, 4>(table, n, total, head, done, err, grid, st);
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t inv_queue_s(int sch, int q1, const BatchEntry* table, int n, int total, int* head,
                               int* done, int* err, int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return inv_queue_q<S, SCH_SEP>(q1, table, n, total, head, done, err, grid, st);
        case SCH_NONSEP: return inv_queue_q<S, SCH_NONSEP>(q1, table, n, total, head, done, err, grid, st);
        case SCH_RED: return inv_queue_q<S, SCH_RED>(q1, table, n, total, head, done, err, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_inv_queue(int elem, int scheme, int q1, const BatchEntry* table, int n, int total,
                             int* head, int* done, int* err, int grid, cudaStream_t st) {
    switch (elem) {
        case 0: return inv_queue_s<float>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 1: return inv_queue_s<int>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 2: return inv_queue_s<__half>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 3: return inv_queue_s<__nv_bfloat16>(scheme, q1, table, n, total, head, done, err, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class S, int SCH, int NL, int Q1>
static cudaError_t inv_batched_one(const BatchEntry* table, int n, int grid, cudaStream_t st,
                                   bool pdl) {
    auto k = inv_batched_kernel<S, SCH, NL, Q1>;
    const size_t smem = inv_tma_smem_bytes(sizeof(S), NL, Q1);
    if (grid == 0)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_kernel(k, grid, kInvWarps * 32, smem, st, pdl, table, n);
}

template <class S, int SCH>
static cudaError_t inv_batched_nq(int nl, int q1, const BatchEntry* table, int n, int grid,
                                  cudaStream_t st, bool pdl) {
    if (q1 == 2) {
        if (nl == 1) return inv_batched_one<S, SCH, 1, 2>(table, n, grid, st, pdl);
        if (nl == 2) return inv_batched_one<S, SCH, 2, 2>(table, n, grid, st, pdl);
    } else if (q1 == 4) {
        if (nl == 1) return inv_batched_one<S, SCH, 1, 4>(table, n, grid, st, pdl);
        if (nl == 2) return inv_batched_one<S, SCH, 2, 4>(table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t inv_batched_s(int sch, int nl, int q1, const BatchEntry* table, int n, int grid,
                                 cudaStream_t st, bool pdl) {
    switch (sch) {
        case SCH_SEP: return inv_batched_nq<S, SCH_SEP>(nl, q1, table, n, grid, st, pdl);
        case SCH_NONSEP: return inv_batched_nq<S, SCH_NONSEP>(nl, q1, table, n, grid, st, pdl);
        case SCH_RED: return inv_batched_nq<S, SCH_RED>(nl, q1, table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_inv_batched(int elem, int scheme, int nl, int q1, const BatchEntry* table, int n,
                               int grid, cudaStream_t st, bool pdl) {
    switch (elem) {
        case 0: return inv_batched_s<float>(scheme, nl, q1, table, n, grid, st, pdl);
        case 1: return inv_batched_s<int>(scheme, nl, q1, table, n, grid, st, pdl);
        case 2: return inv_batched_s<__half>(scheme, nl, q1, table, n, grid, st, pdl);
        case 3: return inv_batched_s<__nv_bfloat16>(scheme, nl, q1, table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dwt
