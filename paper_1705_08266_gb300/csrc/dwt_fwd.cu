// Forward transform, one image per launch: the kernel over a launch's work
// items and its host-side dispatch (storage type, scheme, fused levels,
// quadruple columns per lane).
#include "dwt_fwd_body.cuh"

namespace dwt {

template <class S, int SCH, int NL, int Q1>
__global__ void __launch_bounds__(kFwdWarps * 32, fwd_min_blocks<NL, Q1>())
    fwd_fused_kernel(const __grid_constant__ CUtensorMap map, const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    grid_dependents_launch();  // the body waits for the previous grid after its setup
    const int wid = blockIdx.x * kFwdWarps + (threadIdx.x >> 5);
    if (wid >= a.nstrips * a.nsegs) return;
    fwd_body<S, SCH, NL, Q1>(&map, a, wid, smem_raw);
}

int fwd_slot_rows(int nl, int q1) { return 2 * ((q1 >= 4 && nl <= 2) ? 2 : 4); }

size_t fwd_smem_bytes(int elem_bytes, int nl, int q1) {
    return (size_t)kFwdWarps * kFwdSlots * fwd_slot_rows(nl, q1) * (64 * q1) * elem_bytes +
           (size_t)kFwdWarps * kFwdSlots * 8;
}

template <class S, int SCH, int NL, int Q1>
static cudaError_t launch_one(const CUtensorMap& map, const FusedArgs& a, int grid,
                              cudaStream_t st) {
    auto k = fwd_fused_kernel<S, SCH, NL, Q1>;
    const size_t smem = fwd_smem_bytes(sizeof(S), NL, Q1);
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return launch_kernel(k, grid, kFwdWarps * 32, smem, st, a.pdl != 0, map, a);
}

template <class T, int SCH>
static cudaError_t launch_nl(int nl, int q1, const CUtensorMap& map, const FusedArgs& a, int grid,
                             cudaStream_t st) {
    if (q1 == 2) {
        switch (nl) {
            case 1: return launch_one<T, SCH, 1, 2>(map, a, grid, st);
            case 2: return launch_one<T, SCH, 2, 2>(map, a, grid, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (nl) {
        case 1: return launch_one<T, SCH, 1, 4>(map, a, grid, st);
        case 2: return launch_one<T, SCH, 2, 4>(map, a, grid, st);
        case 3: return launch_one<T, SCH, 3, 4>(map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class T>
static cudaError_t launch_sch(int sch, int nl, int q1, const CUtensorMap& map, const FusedArgs& a,
                              int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return launch_nl<T, SCH_SEP>(nl, q1, map, a, grid, st);
        case SCH_NONSEP: return launch_nl<T, SCH_NONSEP>(nl, q1, map, a, grid, st);
        case SCH_RED: return launch_nl<T, SCH_RED>(nl, q1, map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

// 16-bit storage: 1 or 2 fused levels, 2 or 4 columns per lane
template <class S, int SCH>
static cudaError_t launch_nl16(int nl, int q1, const CUtensorMap& map, const FusedArgs& a, int grid,
                               cudaStream_t st) {
    if (nl == 1) return q1 == 4 ? launch_one<S, SCH, 1, 4>(map, a, grid, st)
                                : launch_one<S, SCH, 1, 2>(map, a, grid, st);
    if (nl == 2) return q1 == 4 ? launch_one<S, SCH, 2, 4>(map, a, grid, st)
                                : launch_one<S, SCH, 2, 2>(map, a, grid, st);
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_sch16(int sch, int nl, int q1, const CUtensorMap& map, const FusedArgs& a,
                                int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return launch_nl16<S, SCH_SEP>(nl, q1, map, a, grid, st);
        case SCH_NONSEP: return launch_nl16<S, SCH_NONSEP>(nl, q1, map, a, grid, st);
        case SCH_RED: return launch_nl16<S, SCH_RED>(nl, q1, map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_fused(int elem, int scheme, int nl, int q1, const CUtensorMap& map,
                             const FusedArgs& a, int grid, cudaStream_t st) {
    switch (elem) {
        case 0: return launch_sch<float>(scheme, nl, q1, map, a, grid, st);
        case 1: return launch_sch<int>(scheme, nl, q1, map, a, grid, st);
        // 16-bit storage: up to 2 fused levels
        case 2: return launch_sch16<__half>(scheme, nl, q1, map, a, grid, st);
        case 3: return launch_sch16<__nv_bfloat16>(scheme, nl, q1, map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dwt
