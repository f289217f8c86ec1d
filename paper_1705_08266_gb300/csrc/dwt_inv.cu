// Inverse transform: warp-streaming kernel, 1..3 levels per launch, coarse to fine.
//
// Each warp owns a strip of output columns and a segment of output rows.  The
// coarsest engine receives quadruple rows assembled from the LL band (or the
// LL written by the previous launch) and the three detail bands; every row it
// emits is two rows of the next finer LL, which the next engine combines with
// that level's detail bands, down to level 1, whose emitted rows are image
// rows.  Band rows are read with coalesced vector loads straight from HBM.
#include <type_traits>

#include "dwt_engine.cuh"
#include "dwt_internal.h"

namespace dwt {

template <class T, int Q>
struct VecI;
template <>
struct VecI<float, 4> { using type = float4; };
template <>
struct VecI<float, 2> { using type = float2; };
template <>
struct VecI<float, 1> { using type = float; };
template <>
struct VecI<int, 4> { using type = int4; };
template <>
struct VecI<int, 2> { using type = int2; };
template <>
struct VecI<int, 1> { using type = int; };

// Load Q values of one band row: columns g0 .. g0+Q-1 of a band of `ncols`
// columns and `nrows` rows; zero outside.
template <class T, int Q>
__device__ __forceinline__ void load_cols(T (&v)[Q], const T* base, long long pitch, int row,
                                          int nrows, int col0, int g0, int ncols, bool vec) {
    if (row < 0 || row >= nrows) {
#pragma unroll
        for (int j = 0; j < Q; ++j) v[j] = T(0);
        return;
    }
    const T* p = base + (long long)row * pitch + col0 + g0;
    if (vec && g0 >= 0 && g0 + Q <= ncols) {
        using V = typename VecI<T, Q>::type;
        const V w = __ldg(reinterpret_cast<const V*>(p));
        const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int j = 0; j < Q; ++j) v[j] = wp[j];
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int g = g0 + j;
            v[j] = (g >= 0 && g < ncols) ? __ldg(p + j) : T(0);
        }
    }
}

struct InvGeo {
    int ne_r, no_r, ne_c, no_c;
    int g0;
    bool vec_hl, vec_lh, vec_ll;
};

__device__ __forceinline__ InvGeo make_igeo(int h, int w, int g0, int Q, long long pitch,
                                            long long ll_pitch) {
    InvGeo g;
    g.ne_r = (h + 1) >> 1;
    g.no_r = h >> 1;
    g.ne_c = (w + 1) >> 1;
    g.no_c = w >> 1;
    g.g0 = g0;
    g.vec_hl = (g.ne_c % Q == 0) && (pitch % Q == 0);
    g.vec_lh = (pitch % Q == 0);
    g.vec_ll = (ll_pitch % Q == 0);
    return g;
}

template <class T, int Q>
__device__ __forceinline__ void load_details(Quads<T, Q>& a, int i, const InvGeo& g, const T* m,
                                             long long pitch) {
    load_cols<T, Q>(a.c[1], m, pitch, i, g.ne_r, g.ne_c, g.g0, g.no_c, g.vec_hl);
    load_cols<T, Q>(a.c[2], m + (long long)g.ne_r * pitch, pitch, i, g.no_r, 0, g.g0, g.ne_c,
                    g.vec_lh);
    load_cols<T, Q>(a.c[3], m + (long long)g.ne_r * pitch, pitch, i, g.no_r, g.ne_c, g.g0, g.no_c,
                    g.vec_hl);
}

template <class T, int SCH, int NL>
struct InvWarp {
    Engine<T, 4, SCH, false> e1;
    Engine<T, 2, SCH, false> e2;
    Engine<T, 1, SCH, false> e3;
    LevelCtx x[3];
    InvGeo g[3];
    const T* mallat;
    long long pitch;
    T* out;
    long long out_pitch;
    int out_h, out_w, xb, lane;
    int A0, A1;  // level-1 output quadruple rows this item stores
    bool lane_ok, vec_out;

    template <int L>
    __device__ __forceinline__ auto& eng() {
        if constexpr (L == 1) return e1;
        else if constexpr (L == 2) return e2;
        else return e3;
    }

    // Push input row i of level L (its LL values already in a.c[0]).
    template <int L>
    __device__ __forceinline__ void push(Quads<T, (4 >> (L - 1))>& a, int i) {
        constexpr int Q = 4 >> (L - 1);
        load_details<T, Q>(a, i, g[L - 1], mallat, pitch);
        int r = i;
        if (!eng<L>().template push_counted<true>(a, r, x[L - 1])) return;
        // emitted quadruple row r -> rows 2r (c0 c1 interleaved) and 2r+1 (c2 c3)
        if constexpr (L == 1) {
            if (!lane_ok || r < A0 || r >= A1) return;
            T ev[8], od[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ev[2 * j] = a.c[0][j];
                ev[2 * j + 1] = a.c[1][j];
                od[2 * j] = a.c[2][j];
                od[2 * j + 1] = a.c[3][j];
            }
            store_px(ev, 2 * r);
            store_px(od, 2 * r + 1);
        } else {
            constexpr int QF = 2 * Q;  // columns of the finer level
            Quads<T, QF> f0, f1;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                f0.c[0][2 * j] = a.c[0][j];
                f0.c[0][2 * j + 1] = a.c[1][j];
                f1.c[0][2 * j] = a.c[2][j];
                f1.c[0][2 * j + 1] = a.c[3][j];
            }
            push<L - 1>(f0, 2 * r);
            push<L - 1>(f1, 2 * r + 1);
        }
    }

    __device__ __forceinline__ void store_px(const T (&v)[8], int y) {
        if (y >= out_h) return;
        const int x0 = xb + 8 * lane;
        T* p = out + (long long)y * out_pitch + x0;
        if (!store_ok(p + max(-x0, 0), (min(x0 + 8, out_w) - max(x0, 0)) * (int)sizeof(T))) return;
        if (vec_out && x0 + 8 <= out_w) {
            using V = typename VecI<T, 4>::type;
            V w0, w1;
            T* a0 = reinterpret_cast<T*>(&w0);
            T* a1 = reinterpret_cast<T*>(&w1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                a0[j] = v[j];
                a1[j] = v[4 + j];
            }
            reinterpret_cast<V*>(p)[0] = w0;
            reinterpret_cast<V*>(p)[1] = w1;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (x0 + j >= 0 && x0 + j < out_w) p[j] = v[j];
        }
    }
};

template <class T, int SCH, int NL>
__global__ void __launch_bounds__(128) inv_fused_kernel(const FusedArgs a) {
    constexpr int RHO = std::is_same<T, float>::value ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= a.nstrips * a.nsegs) return;
    const int strip = wid % a.nstrips;

    InvWarp<T, SCH, NL> W;
    W.lane = lane;
    W.xb = strip * a.valid_px - a.xoff;
    W.lane_ok = lane >= a.lane_lo && lane < a.lane_hi;
    W.mallat = reinterpret_cast<const T*>(a.mallat);
    W.pitch = a.mallat_pitch;
    W.out = reinterpret_cast<T*>(a.out);
    W.out_pitch = a.out_pitch;
    W.out_h = a.lv[0].h;
    W.out_w = a.lv[0].w;
    W.vec_out = (a.out_pitch % 4) == 0;
    set_store_windows(a.out, a.out_elems * (long long)sizeof(T), nullptr, 0, a.err);
    const int ne1 = (a.lv[0].h + 1) >> 1;
    seg_rows(a, wid / a.nstrips, ne1, W.A0, W.A1);

#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const int Q = 4 >> l;
        const int g0 = (W.xb >> (l + 1)) + Q * lane;
        W.x[l] = make_ctx(g0, Q, a.lv[l].h, a.lv[l].w, a.lane_lo, a.lane_hi, a.lv[l].s);
        W.g[l] = make_igeo(a.lv[l].h, a.lv[l].w, g0, Q, a.mallat_pitch, a.ll_pitch);
    }
    W.e1.init();
    if constexpr (NL >= 2) W.e2.init();
    if constexpr (NL >= 3) W.e3.init();

    // coarsest input rows: the cone of output rows [A0, A1) of level 1
    int f = W.A0, e = W.A1 - 1;
#pragma unroll
    for (int l = 1; l <= NL; ++l) {
        f -= RHO;
        e += RHO;
        if (l < NL) {
            f >>= 1;  // floor
            e >>= 1;
        }
    }
    const int kstart = max(f, 0);
    const int kend = e + 1;

    constexpr int QN = 4 >> (NL - 1);
    const T* ll = reinterpret_cast<const T*>(a.ll);
    const InvGeo& gN = W.g[NL - 1];
#pragma unroll 1
    for (int k = kstart; k < kend; ++k) {
        Quads<T, QN> row;
        load_cols<T, QN>(row.c[0], ll, a.ll_pitch, k, gN.ne_r, 0, gN.g0, gN.ne_c, gN.vec_ll);
        W.template push<NL>(row, k);
    }
}

template <class T, int SCH, int NL>
static cudaError_t launch_one(const FusedArgs& a, int grid, cudaStream_t st) {
    inv_fused_kernel<T, SCH, NL><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T, int SCH>
static cudaError_t launch_nl(int nl, const FusedArgs& a, int grid, cudaStream_t st) {
    switch (nl) {
        case 1: return launch_one<T, SCH, 1>(a, grid, st);
        case 2: return launch_one<T, SCH, 2>(a, grid, st);
        case 3: return launch_one<T, SCH, 3>(a, grid, st);
    }
    return cudaErrorInvalidValue;
}

template <class T>
static cudaError_t launch_sch(int sch, int nl, const FusedArgs& a, int grid, cudaStream_t st) {
    switch (sch) {
        case SCH_SEP: return launch_nl<T, SCH_SEP>(nl, a, grid, st);
        case SCH_NONSEP: return launch_nl<T, SCH_NONSEP>(nl, a, grid, st);
        case SCH_RED: return launch_nl<T, SCH_RED>(nl, a, grid, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_inv_fused(int elem, int scheme, int nl, const FusedArgs& a, int grid,
                             cudaStream_t st) {
    if (elem == 0) return launch_sch<float>(scheme, nl, a, grid, st);
    return launch_sch<int>(scheme, nl, a, grid, st);
}

}  // namespace dwt
