// Inverse transform, one image per launch: the kernel over a launch's work
// items and its host-side dispatch (storage type, scheme, fused levels,
// quadruple columns per lane).
#include "dwt_inv_body.cuh"

namespace dwt {

// 16 warps per SM (128 registers) with 2 quadruple columns per lane, 12 with
// 4 (slots of 2 quadruple rows); the plain non-separable steps (48
// multiply-adds per quadruple) measured faster with the register budget of 12
// warps
template <class S, int SCH, int NL, int Q1>
__global__ void __launch_bounds__(kInvWarps * 32,
                                  (Q1 <= 2 ? (SCH == SCH_NONSEP ? 12 : 16) : 12) / kInvWarps)
    inv_tma_kernel(const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap m2,
                   const __grid_constant__ CUtensorMap ml, const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    grid_dependents_launch();  // the body waits for the previous grid after its setup
    const int wid = blockIdx.x * kInvWarps + (threadIdx.x >> 5);
    if (wid >= a.nstrips * a.nsegs) return;
    inv_body<S, SCH, NL, Q1>(&m1, &m2, &ml, a, wid, smem_raw);
}

int inv_slot_rows(int q1) { return q1 >= 4 ? 2 : 4; }

size_t inv_tma_smem_bytes(int elem_bytes, int nl, int q1) {
    const int A = 16 / elem_bytes, E = 128 / elem_bytes;
    const int W1 = 32 * q1 + A, W2 = 32 * (q1 / 2) + A;
    const int sr = inv_slot_rows(q1);
    const int R1 = (sr * W1 + E - 1) / E * E, R2 = ((sr / 2) * W2 + E - 1) / E * E;
    const int slot = nl == 1 ? 4 * R1 : 3 * R1 + 4 * R2;
    return (size_t)kInvWarps * kInvSlots * slot * elem_bytes + (size_t)kInvWarps * kInvSlots * 8;
}

template <class S, int SCH, int NL, int Q1>
static cudaError_t inv_launch_one(const CUtensorMap& m1, const CUtensorMap& m2,
                                  const CUtensorMap& ml, const FusedArgs& a, int grid,
                                  cudaStream_t st) {
    auto k = inv_tma_kernel<S, SCH, NL, Q1>;
    const size_t smem = inv_tma_smem_bytes(sizeof(S), NL, Q1);
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return launch_kernel(k, grid, kInvWarps * 32, smem, st, a.pdl != 0, m1, m2, ml, a);
}

template <class T, int SCH>
static cudaError_t inv_launch_nl(int nl, int q1, const CUtensorMap& m1, const CUtensorMap& m2,
                                 const CUtensorMap& ml, const FusedArgs& a, int grid,
                                 cudaStream_t st) {
    if (q1 == 2) {
        if (nl == 1) return inv_launch_one<T, SCH, 1, 2>(m1, m2, ml, a, grid, st);
        if (nl == 2) return inv_launch_one<T, SCH, 2, 2>(m1, m2, ml, a, grid, st);
    } else if (q1 == 4) {
        if (nl == 1) return inv_launch_one<T, SCH, 1, 4>(m1, m2, ml, a, grid, st);
        if (nl == 2) return inv_launch_one<T, SCH, 2, 4>(m1, m2, ml, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class T>
static cudaError_t inv_launch_sch(int sch, int nl, int q1, const CUtensorMap& m1,
                                  const CUtensorMap& m2, const CUtensorMap& ml, const FusedArgs& a,
                                  int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return inv_launch_nl<T, SCH_SEP>(nl, q1, m1, m2, ml, a, grid, st);
        case SCH_NONSEP: return inv_launch_nl<T, SCH_NONSEP>(nl, q1, m1, m2, ml, a, grid, st);
        case SCH_RED: return inv_launch_nl<T, SCH_RED>(nl, q1, m1, m2, ml, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_inv_tma(int elem, int scheme, int nl, int q1, const CUtensorMap& m1,
                           const CUtensorMap& m2, const CUtensorMap& ml, const FusedArgs& a,
                           int grid, cudaStream_t st) {
    switch (elem) {
        case 0: return inv_launch_sch<float>(scheme, nl, q1, m1, m2, ml, a, grid, st);
        case 1: return inv_launch_sch<int>(scheme, nl, q1, m1, m2, ml, a, grid, st);
        case 2: return inv_launch_sch<__half>(scheme, nl, q1, m1, m2, ml, a, grid, st);
        case 3: return inv_launch_sch<__nv_bfloat16>(scheme, nl, q1, m1, m2, ml, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dwt
