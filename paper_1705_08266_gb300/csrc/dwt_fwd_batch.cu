// Forward transform over many images: the batched kernel (one launch per
// level group, fusion depth and storage type; warp w of the grid finds its
// image in a table) and the persistent queue kernel (one launch per storage
// type; warps take work items from a queue until it is empty).  Both run the
// warp body of the single-image kernel with 2 or 4 quadruple columns per lane.
#include "dwt_fwd_body.cuh"

namespace dwt {

// Many images in one launch: warp w of the grid works on entry i with
// first[i] <= w < first[i + 1] of a table in device memory.  The arguments
// come from registers instead of the constant bank, so the kernel gets the
// register budget of 12 warps per SM rather than 16 (8 bytes of spills per
// thread with 2 columns per lane, 32-40 with 4).
template <class S, int SCH, int NL, int Q1>
__global__ void __launch_bounds__(kFwdWarps * 32, 12 / kFwdWarps)
    fwd_batched_kernel(const BatchEntry* __restrict__ table, int n) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    grid_dependency_sync();
    const int gw = blockIdx.x * kFwdWarps + (threadIdx.x >> 5);
    const BatchEntry& e = table[find_entry(table, n, gw)];
    const int wid = gw - e.first_warp;
    const FusedArgs a = e.args;  // registers: the body's stores cannot alias it
    if (wid < 0 || wid >= a.nstrips * a.nsegs) return;
    fence_tensormap_acquire(&e.m[0]);
    fwd_body<S, SCH, NL, Q1>(&e.m[0], a, wid, smem_raw);
}

// Persistent form: every warp takes work items from the queue until it is
// empty.  Items are ordered by level group, so every item an item depends on
// was taken earlier by a running warp: the bounded wait always ends unless a
// warp failed, and then the status word already says so.  With both fusion
// depths' bodies in one kernel, 4 columns per lane need the register budget
// of 8 warps per SM (12 spill about 300 bytes per thread).
template <class S, int SCH, int Q1>
__global__ void __launch_bounds__(kFwdWarps * 32, fwd_queue_resident(Q1) / kFwdWarps)
    fwd_queue_kernel(const BatchEntry* __restrict__ table, int n, int total, int* head, int* done,
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
            ok = e.nl == 2 ? fwd_body<S, SCH, 2, Q1>(&e.m[0], a, wid, smem_raw)
                           : fwd_body<S, SCH, 1, Q1>(&e.m[0], a, wid, smem_raw);
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
static size_t queue_smem(int elem_bytes, int q1) {
    const size_t a = fwd_smem_bytes(elem_bytes, 1, q1), b = fwd_smem_bytes(elem_bytes, 2, q1);
    return a > b ? a : b;
}

template <class S, int SCH, int Q1>
static cudaError_t launch_queue_one(const BatchEntry* table, int n, int total, int* head, int* done,
                                    int* err, int grid, cudaStream_t st) {
    auto k = fwd_queue_kernel<S, SCH, Q1>;
    const size_t smem = queue_smem(sizeof(S), Q1);
    if (grid == 0)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_kernel(k, grid, kFwdWarps * 32, smem, st, false, table, n, total, head, done, err);
}

template <class S, int SCH>
static cudaError_t launch_queue_q(int q1, const BatchEntry* table, int n, int total, int* head,
                                  int* done, int* err, int grid, cudaStream_t st) {
    if (q1 == 2) return launch_queue_one<S, SCH, 2>(table, n, total, head, done, err, grid, st);
    if (q1 == 4) return launch_queue_one<S, SCH, 4>(table, n, total, head, done, err, grid, st);
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_queue_s(int sch, int q1, const BatchEntry* table, int n, int total,
                                  int* head, int* done, int* err, int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return launch_queue_q<S, SCH_SEP>(q1, table, n, total, head, done, err, grid, st);
        case SCH_NONSEP: return launch_queue_q<S, SCH_NONSEP>(q1, table, n, total, head, done, err, grid, st);
        case SCH_RED: return launch_queue_q<S, SCH_RED>(q1, table, n, total, head, done, err, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_queue(int elem, int scheme, int q1, const BatchEntry* table, int n, int total,
                             int* head, int* done, int* err, int grid, cudaStream_t st) {
    switch (elem) {
        case 0: return launch_queue_s<float>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 1: return launch_queue_s<int>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 2: return launch_queue_s<__half>(scheme, q1, table, n, total, head, done, err, grid, st);
        case 3: return launch_queue_s<__nv_bfloat16>(scheme, q1, table, n, total, head, done, err, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class S, int SCH, int NL, int Q1>
static cudaError_t launch_batched_one(const BatchEntry* table, int n, int grid, cudaStream_t st,
                                      bool pdl) {
    auto k = fwd_batched_kernel<S, SCH, NL, Q1>;
    const size_t smem = fwd_smem_bytes(sizeof(S), NL, Q1);
    if (grid == 0)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_kernel(k, grid, kFwdWarps * 32, smem, st, pdl, table, n);
}

template <class S, int SCH>
static cudaError_t launch_batched_nq(int nl, int q1, const BatchEntry* table, int n, int grid,
                                     cudaStream_t st, bool pdl) {
    if (q1 == 2) {
        if (nl == 1) return launch_batched_one<S, SCH, 1, 2>(table, n, grid, st, pdl);
        if (nl == 2) return launch_batched_one<S, SCH, 2, 2>(table, n, grid, st, pdl);
    } else if (q1 == 4) {
        if (nl == 1) return launch_batched_one<S, SCH, 1, 4>(table, n, grid, st, pdl);
        if (nl == 2) return launch_batched_one<S, SCH, 2, 4>(table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_batched_s(int sch, int nl, int q1, const BatchEntry* table, int n, int grid,
                                    cudaStream_t st, bool pdl) {
    switch (sch) {
        case SCH_SEP: return launch_batched_nq<S, SCH_SEP>(nl, q1, table, n, grid, st, pdl);
        case SCH_NONSEP: return launch_batched_nq<S, SCH_NONSEP>(nl, q1, table, n, grid, st, pdl);
        case SCH_RED: return launch_batched_nq<S, SCH_RED>(nl, q1, table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_batched(int elem, int scheme, int nl, int q1, const BatchEntry* table, int n,
                               int grid, cudaStream_t st, bool pdl) {
    switch (elem) {
        case 0: return launch_batched_s<float>(scheme, nl, q1, table, n, grid, st, pdl);
        case 1: return launch_batched_s<int>(scheme, nl, q1, table, n, grid, st, pdl);
        case 2: return launch_batched_s<__half>(scheme, nl, q1, table, n, grid, st, pdl);
        case 3: return launch_batched_s<__nv_bfloat16>(scheme, nl, q1, table, n, grid, st, pdl);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dwt
