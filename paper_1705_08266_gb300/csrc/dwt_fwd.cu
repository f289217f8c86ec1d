// Forward transform: TMA-fed warp-streaming kernel, 1..3 levels per launch.
//
// Each warp takes one work item (a strip of 256 input pixels, including a
// halo, and a segment of rows) and streams its rows through a private ring of
// shared-memory slots that the warp's lane 0 fills with 2-D TMA boxes.  The
// level-1 engine (4 quadruple columns per lane) emits finished rows; their
// detail bands are stored and their LL values are paired into level-2
// quadruple rows (2 columns per lane), and so on to level 3 (1 column per
// lane).  Only the LL of the last fused level leaves the chip besides the
// detail bands, so a launch that fuses k levels reads the input once and
// writes every coefficient once.
#include <type_traits>

#include "dwt_engine.cuh"
#include "dwt_internal.h"
#include "dwt_tma.cuh"

namespace dwt {

template <class T, int Q>
struct VecOf;
template <>
struct VecOf<float, 4> { using type = float4; };
template <>
struct VecOf<float, 2> { using type = float2; };
template <>
struct VecOf<float, 1> { using type = float; };
template <>
struct VecOf<int, 4> { using type = int4; };
template <>
struct VecOf<int, 2> { using type = int2; };
template <>
struct VecOf<int, 1> { using type = int; };

// Store Q consecutive values at p; `avail` columns remain inside the band.
template <class T, int Q>
__device__ __forceinline__ void store_cols(T* p, const T (&v)[Q], int avail, bool vec) {
    if (vec && avail >= Q) {
        using V = typename VecOf<T, Q>::type;
        V w;
        T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int j = 0; j < Q; ++j) wp[j] = v[j];
        *reinterpret_cast<V*>(p) = w;
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j < avail) p[j] = v[j];
    }
}

// Per-level store state of one lane.
struct StoreGeo {
    int ne_r, no_r, ne_c, no_c;
    int g0;            // first quadruple column of this lane
    int r_lo, r_hi;    // rows of this level that this work item stores
    bool vec_hl, vec_lh;
};

template <class T, int Q>
__device__ __forceinline__ void store_details(const Quads<T, Q>& a, int r, const StoreGeo& g,
                                              T* mallat, long long pitch, bool lane_ok) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    T* row = mallat + (long long)r * pitch;
    store_cols<T, Q>(row + g.ne_c + g.g0, a.c[1], g.no_c - g.g0, g.vec_hl);
    if (r < g.no_r) {
        T* row2 = mallat + (long long)(g.ne_r + r) * pitch;
        store_cols<T, Q>(row2 + g.g0, a.c[2], g.ne_c - g.g0, g.vec_lh);
        store_cols<T, Q>(row2 + g.ne_c + g.g0, a.c[3], g.no_c - g.g0, g.vec_hl);
    }
}

template <class T, int Q>
__device__ __forceinline__ void store_ll(const Quads<T, Q>& a, int r, const StoreGeo& g, T* ll,
                                         long long pitch, bool lane_ok, bool vec) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    store_cols<T, Q>(ll + (long long)r * pitch + g.g0, a.c[0], g.ne_c - g.g0, vec);
}

__device__ __forceinline__ StoreGeo make_geo(int h, int w, int g0, int Q, int r_lo, int r_hi,
                                             long long pitch) {
    StoreGeo g;
    g.ne_r = (h + 1) >> 1;
    g.no_r = h >> 1;
    g.ne_c = (w + 1) >> 1;
    g.no_c = w >> 1;
    g.g0 = g0;
    g.r_lo = r_lo;
    g.r_hi = r_hi;
    g.vec_hl = (g.ne_c % Q == 0) && (pitch % Q == 0);
    g.vec_lh = (pitch % Q == 0);
    return g;
}

// Pair two consecutive LL rows (even row e, odd row o) of Q values into a
// quadruple row of Q/2 columns for the next level.
template <class T, int Q>
__device__ __forceinline__ void pair_rows(const T (&e)[Q], const T (&o)[Q], Quads<T, Q / 2>& n) {
#pragma unroll
    for (int j = 0; j < Q / 2; ++j) {
        n.c[0][j] = e[2 * j];
        n.c[1][j] = e[2 * j + 1];
        n.c[2][j] = o[2 * j];
        n.c[3][j] = o[2 * j + 1];
    }
}

template <class T, int SCH, int NL>
__global__ void __launch_bounds__(kFwdWarps * 32)
    fwd_fused_kernel(const __grid_constant__ CUtensorMap map, const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int RHO = std::is_same<T, float>::value ? 2 : 1;
    using E1 = Engine<T, 4, SCH, true>;
    using E2 = Engine<T, 2, SCH, true>;
    using E3 = Engine<T, 1, SCH, true>;
    static_assert(E1::LAG == RHO && E2::LAG == RHO && E3::LAG == RHO, "lag");

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wid = blockIdx.x * kFwdWarps + warp;
    if (wid >= a.nstrips * a.nsegs) return;

    constexpr int kSlotElems = kFwdSlotRows * kBoxW;
    T* ring = reinterpret_cast<T*>(smem_raw) + (size_t)warp * kFwdSlots * kSlotElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kFwdWarps * kFwdSlots *
                                                              kSlotElems * sizeof(T)) +
                     warp * kFwdSlots;

    const int strip = wid % a.nstrips;
    const int seg = wid / a.nstrips;
    const int xb = strip * a.valid_px - a.xoff;
    const bool lane_ok = lane >= a.lane_lo && lane < a.lane_hi;

    // rows of the last fused level this item produces, and the input rows it needs
    const int neN = (a.lv[NL - 1].h + 1) >> 1;
    const int R0 = seg * a.segq;
    const int R1 = min(R0 + a.segq, neN);
    int f = R0, e = R1 - 1;
#pragma unroll
    for (int l = NL; l >= 1; --l) {
        f -= RHO;
        e += RHO;
        if (l > 1) {
            f *= 2;
            e = 2 * e + 1;
        }
    }
    const int qstart = max(f, 0);
    const int qend = e + 1;
    const int nslots = (2 * (qend - qstart) + kFwdSlotRows - 1) / kFwdSlotRows;

    // per-level lane geometry
    const int g1 = (xb >> 1) + 4 * lane;
    const LevelCtx x1 = make_ctx(g1, 4, a.lv[0].h, a.lv[0].w, a.lane_lo, a.lane_hi, a.lv[0].s);
    const StoreGeo s1 = make_geo(a.lv[0].h, a.lv[0].w, g1, 4, R0 << (NL - 1), R1 << (NL - 1),
                                 a.mallat_pitch);
    LevelCtx x2, x3;
    StoreGeo s2, s3;
    if constexpr (NL >= 2) {
        const int g2 = (xb >> 2) + 2 * lane;
        x2 = make_ctx(g2, 2, a.lv[1].h, a.lv[1].w, a.lane_lo, a.lane_hi, a.lv[1].s);
        s2 = make_geo(a.lv[1].h, a.lv[1].w, g2, 2, R0 << (NL - 2), R1 << (NL - 2), a.mallat_pitch);
    }
    if constexpr (NL >= 3) {
        const int g3 = (xb >> 3) + lane;
        x3 = make_ctx(g3, 1, a.lv[2].h, a.lv[2].w, a.lane_lo, a.lane_hi, a.lv[2].s);
        s3 = make_geo(a.lv[2].h, a.lv[2].w, g3, 1, R0, R1, a.mallat_pitch);
    }
    constexpr int QN = 4 >> (NL - 1);
    const bool vec_ll = (a.ll_pitch % QN) == 0;

    T* mallat = reinterpret_cast<T*>(a.mallat);
    T* ll = reinterpret_cast<T*>(a.ll);

    E1 e1;
    E2 e2;
    E3 e3;
    e1.init();
    if constexpr (NL >= 2) e2.init();
    if constexpr (NL >= 3) e3.init();
    T pend1[4], pend2[2];
    int pend1_r = -0x40000000, pend2_r = -0x40000000;

    // ---- TMA ring prologue
    const uint32_t ring_s = smem_u32(ring);
    const uint32_t bar_s = smem_u32(bars);
    constexpr uint32_t kSlotBytes = kSlotElems * sizeof(T);
    const int y0 = 2 * qstart;
    if (lane == 0) {
        for (int b = 0; b < kFwdSlots; ++b) mbar_init(bar_s + 8 * b, 1);
        fence_mbar_init();
        for (int s = 0; s < kFwdSlots && s < nslots; ++s) {
            mbar_arrive_expect_tx(bar_s + 8 * s, kSlotBytes);
            tma_load_2d(ring_s + s * kSlotBytes, &map, xb, y0 + s * kFwdSlotRows, bar_s + 8 * s);
        }
    }
    __syncwarp();

    int q = qstart;
    bool failed = false;
    int s = 0;
    for (; s < nslots; ++s) {
        const int b = s % kFwdSlots;
        const bool ok = mbar_wait_bounded(bar_s + 8 * b, (s / kFwdSlots) & 1, kWaitBudget);
        if (!__all_sync(kFull, ok)) {  // keep the warp's control flow uniform
            failed = true;
            break;
        }
        const T* slot = ring + b * kSlotElems;
#pragma unroll 1
        for (int k = 0; k < kFwdSlotRows / 2 && q < qend; ++k, ++q) {
            using V4 = typename VecOf<T, 4>::type;
            const V4* r0 = reinterpret_cast<const V4*>(slot + (2 * k) * kBoxW + kLanePx * lane);
            const V4* r1 = reinterpret_cast<const V4*>(slot + (2 * k + 1) * kBoxW + kLanePx * lane);
            const V4 a0 = r0[0], a1 = r0[1], b0 = r1[0], b1 = r1[1];
            Quads<T, 4> row;
            row.c[0][0] = a0.x; row.c[1][0] = a0.y; row.c[0][1] = a0.z; row.c[1][1] = a0.w;
            row.c[0][2] = a1.x; row.c[1][2] = a1.y; row.c[0][3] = a1.z; row.c[1][3] = a1.w;
            row.c[2][0] = b0.x; row.c[3][0] = b0.y; row.c[2][1] = b0.z; row.c[3][1] = b0.w;
            row.c[2][2] = b1.x; row.c[3][2] = b1.y; row.c[2][3] = b1.z; row.c[3][3] = b1.w;

            int r1i = q;
            if (!e1.push(row, r1i, x1)) continue;
            store_details<T, 4>(row, r1i, s1, mallat, a.mallat_pitch, lane_ok);
            if constexpr (NL == 1) {
                store_ll<T, 4>(row, r1i, s1, ll, a.ll_pitch, lane_ok, vec_ll);
            } else {
                if ((r1i & 1) == 0) {
                    copy_arr(pend1, row.c[0]);
                    pend1_r = r1i;
                    continue;
                }
                if (pend1_r != r1i - 1) continue;
                Quads<T, 2> row2;
                pair_rows<T, 4>(pend1, row.c[0], row2);
                int r2i = r1i >> 1;
                if (!e2.push(row2, r2i, x2)) continue;
                store_details<T, 2>(row2, r2i, s2, mallat, a.mallat_pitch, lane_ok);
                if constexpr (NL == 2) {
                    store_ll<T, 2>(row2, r2i, s2, ll, a.ll_pitch, lane_ok, vec_ll);
                } else {
                    if ((r2i & 1) == 0) {
                        copy_arr(pend2, row2.c[0]);
                        pend2_r = r2i;
                        continue;
                    }
                    if (pend2_r != r2i - 1) continue;
                    Quads<T, 1> row3;
                    pair_rows<T, 2>(pend2, row2.c[0], row3);
                    int r3i = r2i >> 1;
                    if (!e3.push(row3, r3i, x3)) continue;
                    store_details<T, 1>(row3, r3i, s3, mallat, a.mallat_pitch, lane_ok);
                    store_ll<T, 1>(row3, r3i, s3, ll, a.ll_pitch, lane_ok, vec_ll);
                }
            }
        }
        __syncwarp();
        if (lane == 0 && s + kFwdSlots < nslots) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar_s + 8 * b, kSlotBytes);
            tma_load_2d(ring_s + b * kSlotBytes, &map, xb, y0 + (s + kFwdSlots) * kFwdSlotRows,
                        bar_s + 8 * b);
        }
    }
    if (failed) {
        if (lane == 0) atomicExch(a.err, -6);
        // drain the copies still in flight before the warp leaves
        for (int t = s; t < nslots && t < s + kFwdSlots; ++t)
            mbar_wait_bounded(bar_s + 8 * (t % kFwdSlots), (t / kFwdSlots) & 1, kWaitBudget);
    }
}

size_t fwd_smem_bytes(int elem_bytes) {
    return (size_t)kFwdWarps * kFwdSlots * kFwdSlotRows * kBoxW * elem_bytes +
           (size_t)kFwdWarps * kFwdSlots * 8;
}

template <class T, int SCH, int NL>
static cudaError_t launch_one(const CUtensorMap& map, const FusedArgs& a, int grid,
                              cudaStream_t st) {
    auto k = fwd_fused_kernel<T, SCH, NL>;
    const size_t smem = fwd_smem_bytes(sizeof(T));
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<grid, kFwdWarps * 32, smem, st>>>(map, a);
    return cudaGetLastError();
}

template <class T, int SCH>
static cudaError_t launch_nl(int nl, const CUtensorMap& map, const FusedArgs& a, int grid,
                             cudaStream_t st) {
    switch (nl) {
        case 1: return launch_one<T, SCH, 1>(map, a, grid, st);
        case 2: return launch_one<T, SCH, 2>(map, a, grid, st);
        case 3: return launch_one<T, SCH, 3>(map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class T>
static cudaError_t launch_sch(int sch, int nl, const CUtensorMap& map, const FusedArgs& a,
                              int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return launch_nl<T, SCH_SEP>(nl, map, a, grid, st);
        case SCH_NONSEP: return launch_nl<T, SCH_NONSEP>(nl, map, a, grid, st);
        case SCH_RED: return launch_nl<T, SCH_RED>(nl, map, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_fused(int elem, int scheme, int nl, const CUtensorMap& map,
                             const FusedArgs& a, int grid, cudaStream_t st) {
    if (elem == 0) return launch_sch<float>(scheme, nl, map, a, grid, st);
    return launch_sch<int>(scheme, nl, map, a, grid, st);
}

}  // namespace dwt
