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

#include <stdint.h>

#include "dwt_internal.h"
#include "dwt_steps.cuh"

namespace dwt {

constexpr unsigned kFull = 0xffffffffu;

template <class T, int Q>
struct Quads {
    T c[4][Q];  // c[component][column within lane]
};

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

// R[j] = v at column j+1, mirrored at the right border.
template <class T, int Q>
__device__ __forceinline__ void right_nb(const T (&v)[Q], T (&R)[Q], unsigned m) {
    const T n = shfl_dn(v[0]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T nb = (j + 1 < Q) ? v[j + 1] : n;
        R[j] = ((m >> j) & 1u) ? nb : v[j];
    }
}
// L[j] = v at column j-1, mirrored at the left border.
template <class T, int Q>
__device__ __forceinline__ void left_nb(const T (&v)[Q], T (&L)[Q], unsigned m) {
    const T p = shfl_up(v[Q - 1]);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T nb = (j > 0) ? v[j - 1] : p;
        L[j] = ((m >> j) & 1u) ? nb : v[j];
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

enum Kind { K_NONE = 0, K_DOWN = 1, K_UP = 2 };

// ------------------------------------------------------------------ ops ----
// Every op names its vertical dependency (kind) and whether it needs the own
// odd samples mirrored horizontally before it runs (kHsub).

// float, separable
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

template <int ID, int SIGN>
struct OpFTH {
    static constexpr int kind = K_NONE;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const LevelCtx& x) {
        float c0r[Q], c2r[Q];
        right_nb(a.c[0], c0r, x.right);
        right_nb(a.c[2], c2r, x.right);
        const float p = Coef<ID, SIGN>::v * x.hf;
#pragma unroll
        for (int j = 0; j < Q; ++j) f_TH(a.c[1][j], a.c[3][j], a.c[0][j], c0r[j], a.c[2][j], c2r[j], p);
    }
};
template <int ID, int SIGN>
struct OpFTV {
    static constexpr int kind = K_DOWN;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&n0)[Q],
                                                 const float (&n1)[Q], const LevelCtx& x) {
        const float p = Coef<ID, SIGN>::v * x.vf;
#pragma unroll
        for (int j = 0; j < Q; ++j) f_TV(a.c[2][j], a.c[3][j], a.c[0][j], n0[j], a.c[1][j], n1[j], p);
    }
};
template <int ID, int SIGN>
struct OpFSH {
    static constexpr int kind = K_NONE;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const LevelCtx& x) {
        if (x.need_hsub) {
            subst_odd(a.c[1], x.odd);
            subst_odd(a.c[3], x.odd);
        }
        float c1l[Q], c3l[Q];
        left_nb(a.c[1], c1l, x.left);
        left_nb(a.c[3], c3l, x.left);
        const float u = Coef<ID, SIGN>::v * x.hf;
#pragma unroll
        for (int j = 0; j < Q; ++j) f_SH(a.c[0][j], a.c[2][j], a.c[1][j], c1l[j], a.c[3][j], c3l[j], u);
    }
};
template <int ID, int SIGN>
struct OpFSV {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = false;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&up2)[Q],
                                                 const float (&up3)[Q], const LevelCtx& x) {
        const float u = Coef<ID, SIGN>::v * x.vf;
#pragma unroll
        for (int j = 0; j < Q; ++j) f_SV(a.c[0][j], a.c[1][j], a.c[2][j], up2[j], a.c[3][j], up3[j], u);
    }
};

// float, non-separable (RED = reduced form)
template <int ID, int SIGN, bool RED>
struct OpFT {
    static constexpr int kind = K_DOWN;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&n0)[Q],
                                                 const float (&n1)[Q], const LevelCtx& x) {
        float c0r[Q], c2r[Q], n0r[Q];
        right_nb(a.c[0], c0r, x.right);
        right_nb(a.c[2], c2r, x.right);
        right_nb(n0, n0r, x.right);
        const float ph = Coef<ID, SIGN>::v * x.hf, pv = Coef<ID, SIGN>::v * x.vf;
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
};
template <int ID, int SIGN, bool RED>
struct OpFS {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = true;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<float, Q>& a, const float (&up2)[Q],
                                                 const float (&up3)[Q], const LevelCtx& x) {
        float c1l[Q], c3l[Q], u3l[Q];
        left_nb(a.c[1], c1l, x.left);
        left_nb(a.c[3], c3l, x.left);
        left_nb(up3, u3l, x.left);
        const float uh = Coef<ID, SIGN>::v * x.hf, uv = Coef<ID, SIGN>::v * x.vf;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (RED)
                f_S_red(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j], up3[j],
                        u3l[j], uh, uv);
            else
                f_S_plain(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j],
                          up3[j], u3l[j], uh, uv);
        }
    }
};

// integer, separable (SIGN = +1 forward, -1 undo)
template <int SIGN>
struct OpITH {
    static constexpr int kind = K_NONE;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const LevelCtx& x) {
        int c0r[Q], c2r[Q];
        right_nb(a.c[0], c0r, x.right);
        right_nb(a.c[2], c2r, x.right);
#pragma unroll
        for (int j = 0; j < Q; ++j) i_TH(a.c[1][j], a.c[3][j], a.c[0][j], c0r[j], a.c[2][j], c2r[j], x.ha, SIGN);
    }
};
template <int SIGN>
struct OpITV {
    static constexpr int kind = K_DOWN;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&n0)[Q],
                                                 const int (&n1)[Q], const LevelCtx& x) {
#pragma unroll
        for (int j = 0; j < Q; ++j) i_TV(a.c[2][j], a.c[3][j], a.c[0][j], n0[j], a.c[1][j], n1[j], x.va, SIGN);
    }
};
template <int SIGN>
struct OpISH {
    static constexpr int kind = K_NONE;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const LevelCtx& x) {
        if (x.need_hsub) {
            subst_odd(a.c[1], x.odd);
            subst_odd(a.c[3], x.odd);
        }
        int c1l[Q], c3l[Q];
        left_nb(a.c[1], c1l, x.left);
        left_nb(a.c[3], c3l, x.left);
#pragma unroll
        for (int j = 0; j < Q; ++j) i_SH(a.c[0][j], a.c[2][j], a.c[1][j], c1l[j], a.c[3][j], c3l[j], x.ha, SIGN);
    }
};
template <int SIGN>
struct OpISV {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = false;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&up2)[Q],
                                                 const int (&up3)[Q], const LevelCtx& x) {
#pragma unroll
        for (int j = 0; j < Q; ++j) i_SV(a.c[0][j], a.c[1][j], a.c[2][j], up2[j], a.c[3][j], up3[j], x.va, SIGN);
    }
};

// integer, non-separable with nested floors
template <bool FWD>
struct OpIT {
    static constexpr int kind = K_DOWN;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&n0)[Q],
                                                 const int (&n1)[Q], const LevelCtx& x) {
        int c0r[Q], c2r[Q], n0r[Q];
        right_nb(a.c[0], c0r, x.right);
        right_nb(a.c[2], c2r, x.right);
        right_nb(n0, n0r, x.right);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (FWD)
                i_T_fwd(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                        n0r[j], x.ha, x.va);
            else
                i_T_inv(a.c[1][j], a.c[2][j], a.c[3][j], a.c[0][j], c0r[j], c2r[j], n0[j], n1[j],
                        n0r[j], x.ha, x.va);
        }
    }
};
template <bool FWD>
struct OpIS {
    static constexpr int kind = K_UP;
    static constexpr bool kHsub = true;
    template <int Q>
    __device__ __forceinline__ static void apply(Quads<int, Q>& a, const int (&up2)[Q],
                                                 const int (&up3)[Q], const LevelCtx& x) {
        int c1l[Q], c3l[Q], u3l[Q];
        left_nb(a.c[1], c1l, x.left);
        left_nb(a.c[3], c3l, x.left);
        left_nb(up3, u3l, x.left);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (FWD)
                i_S_fwd(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j], up3[j],
                        u3l[j], x.ha, x.va);
            else
                i_S_inv(a.c[0][j], a.c[1][j], a.c[2][j], a.c[3][j], c1l[j], c3l[j], up2[j], up3[j],
                        u3l[j], x.ha, x.va);
        }
    }
};

// ---------------------------------------------------------------- stages ----
template <class T, int Q, int KIND>
struct StageState {};
template <class T, int Q>
struct StageState<T, Q, K_DOWN> {
    Quads<T, Q> saved;  // the previous input row
};
template <class T, int Q>
struct StageState<T, Q, K_UP> {
    T p2[Q], p3[Q];  // odd-row components of the previous input row (pre-step, mirrored)
    bool primed;
};

template <class T, int Q, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_NONE>&, Quads<T, Q>& a, int&,
                                          const LevelCtx& x) {
    Op::apply(a, x);
}

// A predict reading the lower row: emits row r-1 when row r arrives.
template <class T, int Q, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_DOWN>& st, Quads<T, Q>& a, int& r,
                                          const LevelCtx& x) {
    Quads<T, Q> out = st.saved;
    const bool real = r < x.ne_r;  // else row r is the mirror of row r-1
    T n0[Q], n1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        n0[j] = real ? a.c[0][j] : out.c[0][j];
        n1[j] = real ? a.c[1][j] : out.c[1][j];
    }
    st.saved = a;
    Op::apply(out, n0, n1, x);
    a = out;
    r = r - 1;
}

// An update reading the upper row: emits row r at once.
template <class T, int Q, class Op>
__device__ __forceinline__ void run_stage(StageState<T, Q, K_UP>& st, Quads<T, Q>& a, int& r,
                                          const LevelCtx& x) {
    if (st.primed && r >= x.no_r) {  // odd height: the last row has no odd image row
        copy_arr(a.c[2], st.p2);
        copy_arr(a.c[3], st.p3);
    }
    if (Op::kHsub && x.need_hsub) {
        subst_odd(a.c[1], x.odd);
        subst_odd(a.c[3], x.odd);
    }
    T up2[Q], up3[Q];
    const bool use_prev = st.primed && r != 0;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        up2[j] = use_prev ? st.p2[j] : a.c[2][j];
        up3[j] = use_prev ? st.p3[j] : a.c[3][j];
    }
    copy_arr(st.p2, a.c[2]);
    copy_arr(st.p3, a.c[3]);
    st.primed = true;
    Op::apply(a, up2, up3, x);
}

template <class T, int Q, class... Ops>
struct Chain {
    static constexpr int LAG = 0;
    __device__ __forceinline__ void init() {}
    __device__ __forceinline__ void push(Quads<T, Q>&, int&, const LevelCtx&) {}
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
    __device__ __forceinline__ void push(Quads<T, Q>& a, int& r, const LevelCtx& x) {
        run_stage<T, Q, Op>(st, a, r, x);
        rest.push(a, r, x);
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
        s.primed = false;
    }
};

// The op chains of every (element type, scheme, direction).

template <class T, int Q, int SCH, bool FWD>
struct Pipe;

// CDF 9/7 forward: pairs (alpha, beta), (gamma, delta).
template <int Q>
struct Pipe<float, Q, SCH_SEP, true> {
    using type = Chain<float, Q, OpFTH<0, 1>, OpFTV<0, 1>, OpFSH<1, 1>, OpFSV<1, 1>, OpFTH<2, 1>,
                       OpFTV<2, 1>, OpFSH<3, 1>, OpFSV<3, 1>>;
};
template <int Q>
struct Pipe<float, Q, SCH_NONSEP, true> {
    using type = Chain<float, Q, OpFT<0, 1, false>, OpFS<1, 1, false>, OpFT<2, 1, false>,
                       OpFS<3, 1, false>>;
};
template <int Q>
struct Pipe<float, Q, SCH_RED, true> {
    using type =
        Chain<float, Q, OpFT<0, 1, true>, OpFS<1, 1, true>, OpFT<2, 1, true>, OpFS<3, 1, true>>;
};
// CDF 9/7 inverse: undo every step in reverse order.
template <int Q>
struct Pipe<float, Q, SCH_SEP, false> {
    using type = Chain<float, Q, OpFSV<3, -1>, OpFSH<3, -1>, OpFTV<2, -1>, OpFTH<2, -1>,
                       OpFSV<1, -1>, OpFSH<1, -1>, OpFTV<0, -1>, OpFTH<0, -1>>;
};
template <int Q>
struct Pipe<float, Q, SCH_NONSEP, false> {
    using type = Chain<float, Q, OpFS<3, -1, false>, OpFT<2, -1, false>, OpFS<1, -1, false>,
                       OpFT<0, -1, false>>;
};
template <int Q>
struct Pipe<float, Q, SCH_RED, false> {
    using type = Chain<float, Q, OpFS<3, -1, true>, OpFT<2, -1, true>, OpFS<1, -1, true>,
                       OpFT<0, -1, true>>;
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
    // Push row r; on return `a` / `r` hold the emitted row.  Returns false
    // while the pipeline is still filling.
    __device__ __forceinline__ bool push(Quads<T, Q>& a, int& r, const LevelCtx& x) {
        if (!FWD) scale(a, x);
        chain.push(a, r, x);
        if (FWD) scale(a, x);
        return ++npush > LAG;
    }

   private:
    __device__ __forceinline__ static void scale(Quads<int, Q>&, const LevelCtx&) {}
    __device__ __forceinline__ static void scale(Quads<float, Q>& a, const LevelCtx& x) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < Q; ++j) a.c[k][j] *= x.s[k];
    }
};

}  // namespace dwt
