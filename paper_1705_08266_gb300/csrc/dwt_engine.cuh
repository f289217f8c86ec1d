// Warp-streaming lifting engine.
//
// One warp owns a vertical strip of the image: lane l holds Q adjacent
// quadruple columns of every quadruple row in registers.  Rows stream top to
// bottom through a chain of lifting stages; a stage that reads the lower row
// (a predict with a vertical part) delays its output by one row, a stage that
// reads the upper row (an update with a vertical part) keeps the previous
// row's odd-row components.  Horizontal neighbours come from the adjacent lane
// by warp shuffle.  This is the on-chip exchange of the paper's OpenCL
// mapping (Sec. 3: overlapping blocks, results exchanged on chip, some kept
// in registers) with the block replaced by a warp and the exchange by shuffles.
//
// Borders (whole-sample symmetric extension, exact for the symmetric lifting
// filters): a right neighbour past the last even column is the column itself,
// a left neighbour of column 0 is the column itself, a lower neighbour past
// the last even row is the row itself, an upper neighbour of row 0 is the row
// itself; an odd column / row that does not exist (odd width / height) takes
// the value of the column / row before it, before every update step.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "dwt_internal.h"
#include "dwt_steps.cuh"

namespace dwt {

constexpr unsigned kFull = 0xffffffffu;

template <class T, int Q>
struct Quads {
    T c[4][Q];  // c[component][column within lane]
};

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

__host__ __device__ constexpr int floordiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

// Storage type S in memory, arithmetic type T in registers: FP16 / BF16
// coefficients are lifted in FP32.
template <class S>
struct Storage;
template <>
struct Storage<float> {
    using T = float;
    __device__ __forceinline__ static float ld(float v) { return v; }
    __device__ __forceinline__ static float st(float v) { return v; }
};
template <>
struct Storage<int> {
    using T = int;
    __device__ __forceinline__ static int ld(int v) { return v; }
    __device__ __forceinline__ static int st(int v) { return v; }
};
template <>
struct Storage<__half> {
    using T = float;
    __device__ __forceinline__ static float ld(__half v) { return __half2float(v); }
    __device__ __forceinline__ static __half st(float v) { return __float2half_rn(v); }
};
template <>
struct Storage<__nv_bfloat16> {
    using T = float;
    __device__ __forceinline__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// Bounds-checked builds (-DDWT_BOUNDS_CHECK): every global store of the
// streaming kernels is tested against the byte windows of the buffers the
// warp may write (set per work item); a store outside them is skipped and
// DWT2D_ERR_BOUNDS (-7) is recorded in the status word.
struct StoreWindows {
    const char* lo[2];
    const char* hi[2];
    int* err;
};
#ifdef DWT_BOUNDS_CHECK
__shared__ StoreWindows g_store_windows[32];  // one per warp of the CTA
__device__ __forceinline__ void set_store_windows(const void* b0, long long n0, const void* b1,
                                                  long long n1, int* err) {
    StoreWindows& w = g_store_windows[threadIdx.x >> 5];
    w.lo[0] = static_cast<const char*>(b0);
    w.hi[0] = w.lo[0] + n0;
    w.lo[1] = static_cast<const char*>(b1);
    w.hi[1] = w.lo[1] + n1;
    w.err = err;
}
__device__ __forceinline__ bool store_ok(const void* p, int bytes) {
    if (bytes <= 0) return true;  // nothing is written
    const StoreWindows& w = g_store_windows[threadIdx.x >> 5];
    const char* c = static_cast<const char*>(p);
    for (int k = 0; k < 2; ++k)
        if (w.lo[k] && c >= w.lo[k] && c + bytes <= w.hi[k]) return true;
    atomicExch(w.err, -7);
    return false;
}
#else
__device__ __forceinline__ void set_store_windows(const void*, long long, const void*, long long, int*) {}
__device__ __forceinline__ bool store_ok(const void*, int) { return true; }
#endif

// Raw vector of a given byte size (2, 4, 8 or 16).
template <int BYTES>
struct RawVec;
template <>
struct RawVec<2> { using type = unsigned short; };
template <>
struct RawVec<4> { using type = unsigned int; };
template <>
struct RawVec<8> { using type = uint2; };
template <>
struct RawVec<16> { using type = uint4; };

// N consecutive S values at p (aligned to min(16, N sizeof(S)) bytes).
template <class S, int N>
__device__ __forceinline__ void ld_vec(S (&v)[N], const S* p) {
    constexpr int B = N * (int)sizeof(S);
    if constexpr (B <= 16) {
        using R = typename RawVec<B>::type;
        const R r = *reinterpret_cast<const R*>(p);
        const S* q = reinterpret_cast<const S*>(&r);
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = q[j];
    } else {
        constexpr int H = N / 2;
        S* lo = v;
        S* hi = v + H;
        ld_vec<S, H>(*reinterpret_cast<S(*)[H]>(lo), p);
        ld_vec<S, H>(*reinterpret_cast<S(*)[H]>(hi), p + H);
    }
}
template <class S, int N>
__device__ __forceinline__ void st_vec(S* p, const S (&v)[N]) {
    constexpr int B = N * (int)sizeof(S);
    if constexpr (B <= 16) {
        using R = typename RawVec<B>::type;
        R r;
        S* q = reinterpret_cast<S*>(&r);
#pragma unroll
        for (int j = 0; j < N; ++j) q[j] = v[j];
        *reinterpret_cast<R*>(p) = r;
    } else {
        constexpr int H = N / 2;
        st_vec<S, H>(p, *reinterpret_cast<const S(*)[H]>(v));
        st_vec<S, H>(p + H, *reinterpret_cast<const S(*)[H]>(v + H));
    }
}

// st_vec with an L2 evict-last policy, for rows the next launch reads back:
// the LL a forward launch hands on would otherwise leave the L2 under the
// launch's detail-band stream (kept, its write-back also leaves the launch).
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;  // a pure value: the compiler may compute it once
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// (the "memory" clobbers keep these stores ordered with every other memory
// access of the thread, as plain stores are)
__device__ __forceinline__ void st_hint(void* p, unsigned short r, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(r), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(void* p, unsigned int r, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(r), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(void* p, uint2 r, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(r.x), "r"(r.y),
                 "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(void* p, uint4 r, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(r.x),
                 "r"(r.y), "r"(r.z), "r"(r.w), "l"(pol) : "memory");
}
template <class S, int N>
__device__ __forceinline__ void st_vec_keep(S* p, const S (&v)[N]) {
    constexpr int B = N * (int)sizeof(S);
    if constexpr (B <= 16) {
        using R = typename RawVec<B>::type;
        R r;
        S* q = reinterpret_cast<S*>(&r);
#pragma unroll
        for (int j = 0; j < N; ++j) q[j] = v[j];
        st_hint(p, r, l2_evict_last());
    } else {
        constexpr int H = N / 2;
        st_vec_keep<S, H>(p, *reinterpret_cast<const S(*)[H]>(v));
        st_vec_keep<S, H>(p + H, *reinterpret_cast<const S(*)[H]>(v + H));
    }
}

// Batched kernels: the last table entry whose first_warp <= g (entries sorted
// by first_warp, n >= 1).
__device__ __forceinline__ int find_entry(const BatchEntry* __restrict__ table, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].first_warp <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-level information of one lane (horizontal) and of the level (vertical).
struct LevelCtx {
    unsigned right;  // bit j: column j has its right (even) neighbour inside the image
    unsigned left;   // bit j: column j is not column 0
    unsigned odd;    // bit j: column j has odd samples (c1, c3)
    bool need_hsub;  // warp-uniform: some column of this warp lacks its odd samples
    int ne_r, no_r;  // quadruple rows with an even / an odd image row
    bool ha, va;     // horizontal / vertical axis longer than 1
    float hf, vf;    // 1.0f if the axis is active, else 0.0f
    float s[4];      // scale of LL, HL, LH, HH (forward) or its inverse (inverse)
};

__device__ __forceinline__ LevelCtx make_ctx(int g0, int Q, int h, int w, int lane_lo,
                                             int lane_hi, const float* s) {
    (void)lane_lo;
    (void)lane_hi;
    LevelCtx x;
    const int ne_c = (w + 1) >> 1, no_c = w >> 1;
    x.right = x.left = x.odd = 0u;
    for (int j = 0; j < Q; ++j) {
        const int g = g0 + j;
        if (g + 1 < ne_c) x.right |= 1u << j;
        if (g > 0) x.left |= 1u << j;
        if (g < no_c) x.odd |= 1u << j;
    }
    // a column without odd samples exists only for odd widths (column no_c)
    const int gw0 = __shfl_sync(kFull, g0, 0);
    const int gw1 = __shfl_sync(kFull, g0, 31) + Q;
    x.need_hsub = (w & 1) && no_c >= gw0 && no_c < gw1;
    x.ne_r = (h + 1) >> 1;
    x.no_r = h >> 1;
    x.ha = w > 1;
    x.va = h > 1;
    x.hf = x.ha ? 1.0f : 0.0f;
    x.vf = x.va ? 1.0f : 0.0f;
    for (int k = 0; k < 4; ++k) x.s[k] = s[k];
    return x;
}

template <class T>
__device__ __forceinline__ T shfl_dn(T v) {
    return __shfl_down_sync(kFull, v, 1);
}
template <class T>
__device__ __forceinline__ T shfl_up(T v) {
    return __shfl_up_sync(kFull, v, 1);
}

// R[j] = v at column j+1, mirrored at the right border (EDGE) or not (interior).
template <bool EDGE, class T, int Q>
__device__ __forceinline__ void right_nb(const T (&v)[Q], T (&R)[Q], unsigned m) {
    const T n = shfl_dn(v[0]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T nb = (j + 1 < Q) ? v[j + 1] : n;
        if (EDGE) R[j] = ((m >> j) & 1u) ? nb : v[j];
        else R[j] = nb;
    }
}
// L[j] = v at column j-1, mirrored at the left border (EDGE) or not (interior).
template <bool EDGE, class T, int Q>
__device__ __forceinline__ void left_nb(const T (&v)[Q], T (&L)[Q], unsigned m) {
    const T p = shfl_up(v[Q - 1]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T nb = (j > 0) ? v[j - 1] : p;
        if (EDGE) L[j] = ((m >> j) & 1u) ? nb : v[j];
        else L[j] = nb;
    }
}
// Columns without odd samples take the odd sample of the column before.
template <class T, int Q>
__device__ __forceinline__ void subst_odd(T (&v)[Q], unsigned odd) {
    const T p = shfl_up(v[Q - 1]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T nb = (j > 0) ? v[j - 1] : p;
        if (!((odd >> j) & 1u)) v[j] = nb;
    }
}

template <class T, int Q>
__device__ __forceinline__ void copy_arr(T (&d)[Q], const T (&s)[Q]) {
#pragma unroll
    for (int j = 0; j < Q; ++j) d[j] = s[j];
}

// Packed (float2) lifting on two columns of a lane at once.  PK selects the
// pairing: 1 pairs adjacent columns (j, j + 1); 2 pairs columns half a lane
// apart (j, j + Q/2), so that a pair's right neighbours (j + 1, j + 1 + Q/2)
// are again a pair for every pair but the last.  pair_head(i) is the first
// column of pair i (i < Q/2), pk / unpk pack and unpack pair i.
template <int PK, int Q>
__device__ __forceinline__ constexpr int pair_head(int i) { return PK == 2 ? i : 2 * i; }
template <int PK, int Q>
__device__ __forceinline__ constexpr int pair_step() { return PK == 2 ? Q / 2 : 1; }
template <int PK, int Q>
__device__ __forceinline__ float2 pk(const float (&v)[Q], int i) {
    return make_float2(v[pair_head<PK, Q>(i)], v[pair_head<PK, Q>(i) + pair_step<PK, Q>()]);
}
template <int PK, int Q>
__device__ __forceinline__ void unpk(float2 p, float (&v)[Q], int i) {
    v[pair_head<PK, Q>(i)] = p.x;
    v[pair_head<PK, Q>(i) + pair_step<PK, Q>()] = p.y;
}

// Row segment of the k-th segment slot when segments are taken in F
// interleaved groups ({0, F, 2F, ..}, then {1, F + 1, ..}, ..): with F waves
// of warps, a segment starts about when the one above it ends, so the halo
// rows they share are still in L2.
__device__ __forceinline__ int seg_order(int k, int nsegs, int f) {
    if (f <= 1 || nsegs <= 1) return k;
    const int q = nsegs / f, r = nsegs % f;
    int i, j;
    if (k < r * (q + 1)) {
        i = k / (q + 1);
        j = k % (q + 1);
    } else {
        const int kk = k - r * (q + 1);
        i = r + kk / q;
        j = kk % q;
    }
    return j * f + i;
}

// Rows [r0, r1) of the level a launch's segments are counted in (`rows` in
// all) for segment slot k (warp id / strips).  The first nbig slots are the
// segments of segq rows, in interleaved order; later slots are the shorter
// segments of segq2 rows that follow them, in order, so that the last warps
// a launch starts are short and the launch drains quickly.
__device__ __forceinline__ void seg_rows(const FusedArgs& a, int k, int rows, int& r0, int& r1) {
    if (k < a.nbig) {
        r0 = (a.seg_lo + seg_order(k, a.nbig, a.seg_f)) * a.segq;
        r1 = min(r0 + a.segq, rows);
    } else {
        r0 = (a.seg_lo + a.nbig) * a.segq + (k - a.nbig) * a.segq2;
        r1 = min(r0 + a.segq2, rows);
    }
}

enum Kind { K_NONE = 0, K_DOWN = 1, K_UP = 2 };

// ------------------------------------------------------------------ ops ----
// Every op names its vertical dependency (kind) and whether it needs the own
// odd samples mirrored horizontally before it runs (kHsub).  EDGE = false is
// the interior form: no border substitution and both axes active, so the
// coefficients are compile-time constants.

template <int ID, int SIGN>
struct Coef;
template <int SIGN>
struct Coef<0, SIGN> { static constexpr float v = SIGN * kAlpha; };
template <int SIGN>
struct Coef<1, SIGN> { static constexpr float v = SIGN * kBeta; };
template <int SIGN>
struct Coef<2, SIGN> { static constexpr float v = SIGN * kGamma; };
template <int SIGN>
struct Coef<3, SIGN> { static constexpr float v = SIGN * kDelta; };

template <bool EDGE>
__device__ __forceinline__ float hcoef(float c, const LevelCtx& x) { return EDGE ? c * x.hf : c; }
template <bool EDGE>
__device__ __forceinline__ float vcoef(float c, const LevelCtx& x) { return EDGE ? c * x.vf : c; }
template <bool EDGE>
__device__ __forceinline__ bool hact(const LevelCtx& x) { return EDGE ? x.ha : true; }
template <bool EDGE>
__device__ __forceinline__ bool vact(const LevelCtx& x) { return EDGE ? x.va : true; }

// float, separable (Sec. 2 matrices)
template <int ID, int SIGN, int PK>
struct OpFTH {
    static constexpr int kind = K_NONE;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const LevelCtx& x) {
        float c0r[Q], c2r[Q];
        right_nb<EDGE>(a.c[0], c0r, x.right);
        right_nb<EDGE>(a.c[2], c2r, x.right);
        const float p = hcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c1 = pk<PK, Q>(a.c[1], j), c3 = pk<PK, Q>(a.c[3], j);
                f_TH(c1, c3, pk<PK, Q>(a.c[0], j), pk<PK, Q>(c0r, j), pk<PK, Q>(a.c[2], j), pk<PK, Q>(c2r, j), p);
                unpk<PK, Q>(c1, a.c[1], j);
                unpk<PK, Q>(c3, a.c[3], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) f_TH(a.c[1][j], a.c[3][j], a.c[0][j], c0r[j], a.c[2][j], c2r[j], p);
        }
    }
};
template <int ID, int SIGN, int PK>
struct OpFTV {
    static constexpr int kind = K_DOWN;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&n0)[Q],
                                                 const float (&n1)[Q], const LevelCtx& x) {
        const float p = vcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c2 = pk<PK, Q>(a.c[2], j), c3 = pk<PK, Q>(a.c[3], j);
                f_TV(c2, c3, pk<PK, Q>(a.c[0], j), pk<PK, Q>(n0, j), pk<PK, Q>(a.c[1], j), pk<PK, Q>(n1, j), p);
                unpk<PK, Q>(c2, a.c[2], j);
                unpk<PK, Q>(c3, a.c[3], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) f_TV(a.c[2][j], a.c[3][j], a.c[0][j], n0[j], a.c[1][j], n1[j], p);
        }
    }
};
template <int ID, int SIGN, int PK>
struct OpFSH {
    static constexpr int kind = K_NONE;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const LevelCtx& x) {
        if (EDGE && x.need_hsub) {
            subst_odd(a.c[1], x.odd);
            subst_odd(a.c[3], x.odd);
        }
        float c1l[Q], c3l[Q];
        left_nb<EDGE>(a.c[1], c1l, x.left);
        left_nb<EDGE>(a.c[3], c3l, x.left);
        const float u = hcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c0 = pk<PK, Q>(a.c[0], j), c2 = pk<PK, Q>(a.c[2], j);
                f_SH(c0, c2, pk<PK, Q>(a.c[1], j), pk<PK, Q>(c1l, j), pk<PK, Q>(a.c[3], j), pk<PK, Q>(c3l, j), u);
                unpk<PK, Q>(c0, a.c[0], j);
                unpk<PK, Q>(c2, a.c[2], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) f_SH(a.c[0][j], a.c[2][j], a.c[1][j], c1l[j], a.c[3][j], c3l[j], u);
        }
    }
};
template <int ID, int SIGN, int PK>
struct OpFSV {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = false;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&up2)[Q],
                                                 const float (&up3)[Q], const LevelCtx& x) {
        const float u = vcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c0 = pk<PK, Q>(a.c[0], j), c1 = pk<PK, Q>(a.c[1], j);
                f_SV(c0, c1, pk<PK, Q>(a.c[2], j), pk<PK, Q>(up2, j), pk<PK, Q>(a.c[3], j), pk<PK, Q>(up3, j), u);
                unpk<PK, Q>(c0, a.c[0], j);
                unpk<PK, Q>(c1, a.c[1], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) f_SV(a.c[0][j], a.c[1][j], a.c[2][j], up2[j], a.c[3][j], up3[j], u);
        }
    }
};

// float, non-separable (Sec. 3; RED = reduced form)
template <int ID, int SIGN, bool RED, int PK>
struct OpFT {
    static constexpr int kind = K_DOWN;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&n0)[Q],
                                                 const float (&n1)[Q], const LevelCtx& x) {
        float c0r[Q], c2r[Q], n0r[Q];
        right_nb<EDGE>(a.c[0], c0r, x.right);
        right_nb<EDGE>(a.c[2], c2r, x.right);
        right_nb<EDGE>(n0, n0r, x.right);
        const float ph = hcoef<EDGE>(Coef<ID, SIGN>::v, x), pv = vcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c1 = pk<PK, Q>(a.c[1], j), c2 = pk<PK, Q>(a.c[2], j), c3 = pk<PK, Q>(a.c[3], j);
                if (RED)
                    f_T_red(c1, c2, c3, pk<PK, Q>(a.c[0], j), pk<PK, Q>(c0r, j), pk<PK, Q>(c2r, j), pk<PK, Q>(n0, j), pk<PK, Q>(n1, j),
                            pk<PK, Q>(n0r, j), ph, pv);
                else
                    f_T_plain(c1, c2, c3, pk<PK, Q>(a.c[0], j), pk<PK, Q>(c0r, j), pk<PK, Q>(c2r, j), pk<PK, Q>(n0, j), pk<PK, Q>(n1, j),
                              pk<PK, Q>(n0r, j), ph, pv);
                unpk<PK, Q>(c1, a.c[1], j);
                unpk<PK, Q>(c2, a.c[2], j);
                unpk<PK, Q>(c3, a.c[3], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (RED)
                    f_T_red(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                            n0r[j], ph, pv);
                else
                    f_T_plain(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                              n0r[j], ph, pv);
            }
        }
    }
};
template <int ID, int SIGN, bool RED, int PK>
struct OpFS {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = true;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&up2)[Q],
                                                 const float (&up3)[Q], const LevelCtx& x) {
        float c1l[Q], c3l[Q], u3l[Q];
        left_nb<EDGE>(a.c[1], c1l, x.left);
        left_nb<EDGE>(a.c[3], c3l, x.left);
        left_nb<EDGE>(up3, u3l, x.left);
        const float uh = hcoef<EDGE>(Coef<ID, SIGN>::v, x), uv = vcoef<EDGE>(Coef<ID, SIGN>::v, x);
        if constexpr (PK != 0 && Q % 2 == 0) {
#pragma unroll
            for (int j = 0; j < Q / 2; ++j) {
                float2 c0 = pk<PK, Q>(a.c[0], j), c1 = pk<PK, Q>(a.c[1], j), c2 = pk<PK, Q>(a.c[2], j);
                if (RED)
                    f_S_red(c0, c1, c2, pk<PK, Q>(a.c[3], j), pk<PK, Q>(c1l, j), pk<PK, Q>(c3l, j), pk<PK, Q>(up2, j), pk<PK, Q>(up3, j),
                            pk<PK, Q>(u3l, j), uh, uv);
                else
                    f_S_plain(c0, c1, c2, pk<PK, Q>(a.c[3], j), pk<PK, Q>(c1l, j), pk<PK, Q>(c3l, j), pk<PK, Q>(up2, j),
                              pk<PK, Q>(up3, j), pk<PK, Q>(u3l, j), uh, uv);
                unpk<PK, Q>(c0, a.c[0], j);
                unpk<PK, Q>(c1, a.c[1], j);
                unpk<PK, Q>(c2, a.c[2], j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (RED)
                    f_S_red(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j],
                            up3[j], u3l[j], uh, uv);
                else
                    f_S_plain(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j],
                              up3[j], u3l[j], uh, uv);
            }
        }
    }
};

// integer, separable (SIGN = +1 forward, -1 undo)
template <int SIGN>
struct OpITH {
    static constexpr int kind = K_NONE;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const LevelCtx& x) {
        int c0r[Q], c2r[Q];
        right_nb<EDGE>(a.c[0], c0r, x.right);
        right_nb<EDGE>(a.c[2], c2r, x.right);
#pragma unroll
        for (int j = 0; j < Q; ++j)
            i_TH(a.c[1][j], a.c[3][j], a.c[0][j], c0r[j], a.c[2][j], c2r[j], hact<EDGE>(x), SIGN);
    }
};
template <int SIGN>
struct OpITV {
    static constexpr int kind = K_DOWN;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&n0)[Q],
                                                 const int (&n1)[Q], const LevelCtx& x) {
#pragma unroll
        for (int j = 0; j < Q; ++j)
            i_TV(a.c[2][j], a.c[3][j], a.c[0][j], n0[j], a.c[1][j], n1[j], vact<EDGE>(x), SIGN);
    }
};
template <int SIGN>
struct OpISH {
    static constexpr int kind = K_NONE;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const LevelCtx& x) {
        if (EDGE && x.need_hsub) {
            subst_odd(a.c[1], x.odd);
            subst_odd(a.c[3], x.odd);
        }
        int c1l[Q], c3l[Q];
        left_nb<EDGE>(a.c[1], c1l, x.left);
        left_nb<EDGE>(a.c[3], c3l, x.left);
#pragma unroll
        for (int j = 0; j < Q; ++j)
            i_SH(a.c[0][j], a.c[2][j], a.c[1][j], c1l[j], a.c[3][j], c3l[j], hact<EDGE>(x), SIGN);
    }
};
template <int SIGN>
struct OpISV {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = false;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&up2)[Q],
                                                 const int (&up3)[Q], const LevelCtx& x) {
#pragma unroll
        for (int j = 0; j < Q; ++j)
            i_SV(a.c[0][j], a.c[1][j], a.c[2][j], up2[j], a.c[3][j], up3[j], vact<EDGE>(x), SIGN);
    }
};

// integer, non-separable with nested floors
template <bool FWD>
struct OpIT {
    static constexpr int kind = K_DOWN;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&n0)[Q],
                                                 const int (&n1)[Q], const LevelCtx& x) {
        int c0r[Q], c2r[Q], n0r[Q];
        right_nb<EDGE>(a.c[0], c0r, x.right);
        right_nb<EDGE>(a.c[2], c2r, x.right);
        right_nb<EDGE>(n0, n0r, x.right);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (FWD)
                i_T_fwd(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                        n0r[j], hact<EDGE>(x), vact<EDGE>(x));
            else
                i_T_inv(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                        n0r[j], hact<EDGE>(x), vact<EDGE>(x));
        }
    }
};
template <bool FWD>
struct OpIS {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = true;
    template <bool EDGE, int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&up2)[Q],
                                                 const int (&up3)[Q], const LevelCtx& x) {
        int c1l[Q], c3l[Q], u3l[Q];
        left_nb<EDGE>(a.c[1], c1l, x.left);
        left_nb<EDGE>(a.c[3], c3l, x.left);
        left_nb<EDGE>(up3, u3l, x.left);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (FWD)
                i_S_fwd(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j], up3[j],
                        u3l[j], hact<EDGE>(x), vact<EDGE>(x));
            else
                i_S_inv(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j], up3[j],
                        u3l[j], hact<EDGE>(x), vact<EDGE>(x));
        }
    }
};

// ---------------------------------------------------------------- stages ----
// A stage consumes a block of RB consecutive quadruple rows at a time.  Doing
// every lifting step on the whole block before the next step gives each lane
// RB x Q independent quadruples per step; the stage keeps only one row (or the
// odd half of one row) from the previous block.
template <class T, int Q, int RB>
struct Block {
    Quads<T, Q> r[RB];
};

template <class T, int Q, int KIND>
struct StageState {};
template <class T, int Q>
struct StageState<T, Q, K_DOWN> {
    Quads<T, Q> saved;  // the last input row of the previous block (pre-step)
};
template <class T, int Q>
struct StageState<T, Q, K_UP> {
    T p2[Q], p3[Q];  // odd-row components of the previous block's last row (pre-step, mirrored)
};

template <bool EDGE, class T, int Q, int RB, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_NONE>&, Block<T, Q, RB>& b, int&,
                                          const LevelCtx& x) {
#pragma unroll
    for (int j = 0; j < RB; ++j) Op::template apply<EDGE>(b.r[j], x);
}

// A predict reading the lower row.  Input rows [r0, r0 + RB); output rows
// [r0 - 1, r0 + RB - 1): row r0 - 1 (kept from the last block) completes now and
// the last input row waits for the next block.
template <bool EDGE, class T, int Q, int RB, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_DOWN>& st, Block<T, Q, RB>& b, int& r0,
                                          const LevelCtx& x) {
    const Quads<T, Q> keep = b.r[RB - 1];
#pragma unroll
    for (int j = RB - 1; j >= 0; --j) {
        Quads<T, Q> o = (j > 0) ? b.r[j - 1] : st.saved;  // output row r0 - 1 + j
        T n0[Q], n1[Q];                                     // its lower row, pre-step
        // the lower row is past the last even row: mirror (the row itself)
        const bool real = !EDGE || (r0 + j) < x.ne_r;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            n0[i] = real ? b.r[j].c[0][i] : o.c[0][i];
            n1[i] = real ? b.r[j].c[1][i] : o.c[1][i];
        }
        Op::template apply<EDGE>(o, n0, n1, x);
        b.r[j] = o;
    }
    st.saved = keep;
    r0 -= 1;
}

// An update reading the upper row.  Input and output rows [r0, r0 + RB).
template <bool EDGE, class T, int Q, int RB, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_UP>& st, Block<T, Q, RB>& b, int& r0,
                                          const LevelCtx& x) {
    if (EDGE) {
        if (Op::kHsub && x.need_hsub) {
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                subst_odd(b.r[j].c[1], x.odd);
                subst_odd(b.r[j].c[3], x.odd);
            }
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            if (r0 + j >= x.no_r) {  // odd height: the last row has no odd image row
                if (j > 0) {
                    copy_arr(b.r[j].c[2], b.r[j - 1].c[2]);
                    copy_arr(b.r[j].c[3], b.r[j - 1].c[3]);
                } else {
                    copy_arr(b.r[j].c[2], st.p2);
                    copy_arr(b.r[j].c[3], st.p3);
                }
            }
        }
    }
    T n2[Q], n3[Q];
    copy_arr(n2, b.r[RB - 1].c[2]);
    copy_arr(n3, b.r[RB - 1].c[3]);
#pragma unroll
    for (int j = RB - 1; j >= 0; --j) {  // downwards: the upper row is still pre-step
        T up2[Q], up3[Q];
        if (j > 0) {
            copy_arr(up2, b.r[j - 1].c[2]);
            copy_arr(up3, b.r[j - 1].c[3]);
        } else {
            copy_arr(up2, st.p2);
            copy_arr(up3, st.p3);
        }
        if (EDGE && r0 + j == 0) {  // image top: the upper row is the row itself
            copy_arr(up2, b.r[j].c[2]);
            copy_arr(up3, b.r[j].c[3]);
        }
        Op::template apply<EDGE>(b.r[j], up2, up3, x);
    }
    copy_arr(st.p2, n2);
    copy_arr(st.p3, n3);
}

template <class T, int Q, class... Ops>
struct Chain {
    static constexpr int LAG = 0;
    __device__ __forceinline__ void init() {}
    template <bool EDGE, int RB>
    __device__ __forceinline__ void push(Block<T, Q, RB>&, int&, const LevelCtx&) {}
};
template <class T, int Q, class Op, class... Rest>
struct Chain<T, Q, Op, Rest...> {
    StageState<T, Q, Op::kind> st;
    Chain<T, Q, Rest...> rest;
    static constexpr int LAG = (Op::kind == K_DOWN ? 1 : 0) + Chain<T, Q, Rest...>::LAG;
    __device__ __forceinline__ void init() {
        zero(st);
        rest.init();
    }
    template <bool EDGE, int RB>
    __device__ __forceinline__ void push(Block<T, Q, RB>& b, int& r0, const LevelCtx& x) {
        run_stage<EDGE, T, Q, RB, Op>(st, b, r0, x);
        rest.template push<EDGE, RB>(b, r0, x);
    }

   private:
    __device__ __forceinline__ static void zero(StageState<T, Q, K_NONE>&) {}
    __device__ __forceinline__ static void zero(StageState<T, Q, K_DOWN>& s) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < Q; ++j) s.saved.c[k][j] = T(0);
    }
    __device__ __forceinline__ static void zero(StageState<T, Q, K_UP>& s) {
#pragma unroll
        for (int j = 0; j < Q; ++j) s.p2[j] = s.p3[j] = T(0);
    }
};

// The op chains of every (element type, scheme, direction).
template <class T, int Q, int SCH, bool FWD>
struct Pipe;

// CDF 9/7 forward: pairs (alpha, beta), (gamma, delta).  The forward runs the
// scalar form of the float steps at 2 columns per lane (its register budget of
// 128 leaves no room for the register pairs) and the packed form at 4
// (kFwdPack4: 1 adjacent, 2 strided pairs); the inverse runs the packed form
// on adjacent pairs.  Each was measured faster for its kernel.
#ifndef DWT_FWD_PACK4
#define DWT_FWD_PACK4 2
#endif
constexpr int kFwdPack4 = DWT_FWD_PACK4;
template <int Q>
constexpr int fwd_pk() { return Q >= 4 ? kFwdPack4 : 0; }
template <int Q>
struct Pipe<float, Q, SCH_SEP, true> {
    static constexpr int P = fwd_pk<Q>();
    using type = Chain<float, Q, OpFTH<0, 1, P>, OpFTV<0, 1, P>, OpFSH<1, 1, P>, OpFSV<1, 1, P>,
                       OpFTH<2, 1, P>, OpFTV<2, 1, P>, OpFSH<3, 1, P>, OpFSV<3, 1, P>>;
};
template <int Q>
struct Pipe<float, Q, SCH_NONSEP, true> {
    static constexpr int P = fwd_pk<Q>();
    using type = Chain<float, Q, OpFT<0, 1, false, P>, OpFS<1, 1, false, P>, OpFT<2, 1, false, P>,
                       OpFS<3, 1, false, P>>;
};
template <int Q>
struct Pipe<float, Q, SCH_RED, true> {
    static constexpr int P = fwd_pk<Q>();
    using type = Chain<float, Q, OpFT<0, 1, true, P>, OpFS<1, 1, true, P>, OpFT<2, 1, true, P>,
                       OpFS<3, 1, true, P>>;
};
// CDF 9/7 inverse: undo every step in reverse order (packed; strided pairs
// at 4 columns per lane).
template <int Q>
constexpr int inv_pk() { return Q >= 4 ? 2 : 1; }
template <int Q>
struct Pipe<float, Q, SCH_SEP, false> {
    static constexpr int P = inv_pk<Q>();
    using type = Chain<float, Q, OpFSV<3, -1, P>, OpFSH<3, -1, P>, OpFTV<2, -1, P>, OpFTH<2, -1, P>,
                       OpFSV<1, -1, P>, OpFSH<1, -1, P>, OpFTV<0, -1, P>, OpFTH<0, -1, P>>;
};
template <int Q>
struct Pipe<float, Q, SCH_NONSEP, false> {
    static constexpr int P = inv_pk<Q>();
    using type = Chain<float, Q, OpFS<3, -1, false, P>, OpFT<2, -1, false, P>,
                       OpFS<1, -1, false, P>, OpFT<0, -1, false, P>>;
};
template <int Q>
struct Pipe<float, Q, SCH_RED, false> {
    static constexpr int P = inv_pk<Q>();
    using type = Chain<float, Q, OpFS<3, -1, true, P>, OpFT<2, -1, true, P>,
                       OpFS<1, -1, true, P>, OpFT<0, -1, true, P>>;
};
// LeGall 5/3 (reversible): the reduced scheme keeps the floors on whole 1-D
// sums and is therefore the same integer dataflow as the non-separable one.
template <int Q>
struct Pipe<int, Q, SCH_SEP, true> {
    using type = Chain<int, Q, OpITH<1>, OpITV<1>, OpISH<1>, OpISV<1>>;
};
template <int Q>
struct Pipe<int, Q, SCH_NONSEP, true> {
    using type = Chain<int, Q, OpIT<true>, OpIS<true>>;
};
template <int Q>
struct Pipe<int, Q, SCH_RED, true> {
    using type = Chain<int, Q, OpIT<true>, OpIS<true>>;
};
template <int Q>
struct Pipe<int, Q, SCH_SEP, false> {
    using type = Chain<int, Q, OpISV<-1>, OpISH<-1>, OpITV<-1>, OpITH<-1>>;
};
template <int Q>
struct Pipe<int, Q, SCH_NONSEP, false> {
    using type = Chain<int, Q, OpIS<false>, OpIT<false>>;
};
template <int Q>
struct Pipe<int, Q, SCH_RED, false> {
    using type = Chain<int, Q, OpIS<false>, OpIT<false>>;
};

// CDF 9/7 scale of LL, HL, LH, HH when both axes are active: 1/K^2, 1, 1, K^2,
// rounded once from double, exactly as the host rounds the per-level scales
// the border code uses (so both code paths give the same bits).
constexpr double kKd = 1.230174104914001;
constexpr float kScaleLL = (float)(1.0 / (kKd * kKd));
constexpr float kScaleHH = (float)(kKd * kKd);

// One level of the transform for one warp: the chain plus the 9/7 scaling.
template <class T, int Q, int SCH, bool FWD>
struct Engine {
    using ChainT = typename Pipe<T, Q, SCH, FWD>::type;
    static constexpr int LAG = ChainT::LAG;
    ChainT chain;
    int npush;
    __device__ __forceinline__ void init() {
        chain.init();
        npush = 0;
    }
    // Push input rows [r0, r0 + RB); on return `b` holds the emitted rows
    // [r0 - LAG, r0 - LAG + RB) (garbage while the pipeline fills).
    template <bool EDGE, int RB>
    __device__ __forceinline__ void push(Block<T, Q, RB>& b, int r0, const LevelCtx& x) {
        if (!FWD) {
#pragma unroll
            for (int j = 0; j < RB; ++j) scale<EDGE>(b.r[j], x);
        }
        chain.template push<EDGE, RB>(b, r0, x);
        if (FWD) {
#pragma unroll
            for (int j = 0; j < RB; ++j) scale<EDGE>(b.r[j], x);
        }
    }
    // One row; returns false while the pipeline is still filling, and sets r to
    // the emitted row.
    template <bool EDGE>
    __device__ __forceinline__ bool push_counted(Quads<T, Q>& a, int& r, const LevelCtx& x) {
        Block<T, Q, 1> b;
        b.r[0] = a;
        push<EDGE, 1>(b, r, x);
        a = b.r[0];
        r -= LAG;
        return ++npush > LAG;
    }

   private:
    template <bool EDGE>
    __device__ __forceinline__ static void scale(Quads<int, Q>&, const LevelCtx&) {}
    template <bool EDGE>
    __device__ __forceinline__ static void scale(Quads<float, Q>& a, const LevelCtx& x) {
        if (EDGE) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int j = 0; j < Q; ++j) a.c[k][j] *= x.s[k];
        } else {
            // both axes active: HL and LH keep their scale 1
            const float sll = FWD ? kScaleLL : kScaleHH, shh = FWD ? kScaleHH : kScaleLL;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                a.c[0][j] *= sll;
                a.c[3][j] *= shh;
            }
        }
    }
};

}  // namespace dwt
