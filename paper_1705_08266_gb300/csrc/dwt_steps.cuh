// Lifting arithmetic of one quadruple, shared by every kernel.
//
// Barina et al., arXiv 1705.08266.  Quadruple (c0, c1, c2, c3) = samples
// (2r, 2c), (2r, 2c+1), (2r+1, 2c), (2r+1, 2c+1).  Filters: P = p (1 + z)
// (reads the right / lower neighbour quadruple), U = u (1 + z^-1) (reads the
// left / upper one); P* and U* are the vertical (transposed) filters.
//
// Naming of neighbour values (all pre-step unless stated):
//   c0r, c2r  c0 / c2 of the right quadruple    n0, n1  c0 / c1 of the lower one
//   n0r       c0 of the lower-right quadruple
//   c1l, c3l  c1 / c3 of the left quadruple     up2, up3  c2 / c3 of the upper one
//   u3l       c3 of the upper-left quadruple
// Callers substitute mirrored values at the image border (whole-sample
// symmetric extension) before calling; coefficients of an inactive axis
// (length 1) are passed as 0 (float) or the axis flag is false (integer).
#pragma once

#include <cuda_runtime.h>

namespace dwt {

// CDF 9/7 lifting constants (Daubechies & Sweldens factorisation, cited by the
// paper for Eq. 2) and the scaling constant K.
constexpr float kAlpha = -1.586134342059924f;
constexpr float kBeta = -0.052980118572961f;
constexpr float kGamma = 0.882911075530934f;
constexpr float kDelta = 0.443506852043971f;
constexpr float kK = 1.230174104914001f;

// ---------------------------------------------------------------- float ----
// Every float step is written once for V = float (one quadruple) and V =
// float2 (two adjacent quadruples of a lane, one packed FP32 instruction per
// pair).  Adds and multiplies are explicit round-to-nearest operations, so no
// contraction differs between the two forms: both give the same bits.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <class V>
__device__ __forceinline__ V splat(float x);
template <>
__device__ __forceinline__ float splat<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 splat<float2>(float x) { return make_float2(x, x); }

// Separable steps (Sec. 2 matrices T_P^H, T_P^V, S_U^H, S_U^V).
template <class V>
__device__ __forceinline__ void f_TH(V& c1, V& c3, V c0, V c0r, V c2, V c2r, float p) {
    const V P = splat<V>(p);
    c1 = vfma(P, vadd(c0, c0r), c1);
    c3 = vfma(P, vadd(c2, c2r), c3);
}
template <class V>
__device__ __forceinline__ void f_TV(V& c2, V& c3, V c0, V n0, V c1, V n1, float p) {
    const V P = splat<V>(p);
    c2 = vfma(P, vadd(c0, n0), c2);
    c3 = vfma(P, vadd(c1, n1), c3);
}
template <class V>
__device__ __forceinline__ void f_SH(V& c0, V& c2, V c1, V c1l, V c3, V c3l, float u) {
    const V U = splat<V>(u);
    c0 = vfma(U, vadd(c1, c1l), c0);
    c2 = vfma(U, vadd(c3, c3l), c2);
}
template <class V>
__device__ __forceinline__ void f_SV(V& c0, V& c1, V c2, V up2, V c3, V up3, float u) {
    const V U = splat<V>(u);
    c0 = vfma(U, vadd(c2, up2), c0);
    c1 = vfma(U, vadd(c3, up3), c1);
}

// Spatial predict T_P (Sec. 3): rows [1,0,0,0], [P,1,0,0], [P*,0,1,0], [PP*,P*,P,1],
// every term from pre-step values.  ph / pv: horizontal / vertical coefficient.
template <class V>
__device__ __forceinline__ void f_T_plain(V& c1, V& c2, V& c3, V c0, V c0r, V c2r, V n0, V n1,
                                          V n0r, float ph, float pv) {
    const V PH = splat<V>(ph), PV = splat<V>(pv), PHV = splat<V>(ph * pv);
    const V s00 = vadd(c0, c0r);
    const V s0d = vadd(c0, n0);
    const V q = vfma(vadd(c2, c2r), PH, vmul(vadd(c1, n1), PV));
    const V n1new = vfma(PHV, vadd(s00, vadd(n0, n0r)), q);
    c1 = vfma(PH, s00, c1);
    c2 = vfma(PV, s0d, c2);
    c3 = vadd(c3, n1new);
}

// Spatial update S_U (Sec. 3): rows [1,U,U*,UU*], [0,1,0,U*], [0,0,1,U], [0,0,0,1].
template <class V>
__device__ __forceinline__ void f_S_plain(V& c0, V& c1, V& c2, V c3, V c1l, V c3l, V up2, V up3,
                                          V u3l, float uh, float uv) {
    const V UH = splat<V>(uh), UV = splat<V>(uv), UHV = splat<V>(uh * uv);
    const V t = vfma(vadd(c1, c1l), UH, vmul(vadd(c2, up2), UV));
    const V d = vfma(UHV, vadd(vadd(c3, c3l), vadd(up3, u3l)), t);
    c1 = vfma(UV, vadd(c3, up3), c1);
    c2 = vfma(UH, vadd(c3, c3l), c2);
    c0 = vadd(c0, d);
}

// Reduced spatial predict (Sec. 3, P = P0 + P1): the neighbour part P1 in the
// non-separable matrix, then the constant part P0 in the separable scheme
// (T^H(P0) then T^V(P0)); no barrier between the two.  9 MACs.
template <class V>
__device__ __forceinline__ void f_T_red(V& c1, V& c2, V& c3, V c0, V c0r, V c2r, V n0, V n1, V n0r,
                                        float ph, float pv) {
    const V PH = splat<V>(ph), PV = splat<V>(pv), PHV = splat<V>(ph * pv);
    c1 = vfma(PH, c0r, c1);
    c2 = vfma(PV, n0, c2);
    c3 = vfma(PH, c2r, c3);
    c3 = vfma(PV, n1, c3);
    c3 = vfma(PHV, n0r, c3);
    c1 = vfma(PH, c0, c1);
    c3 = vfma(PH, c2, c3);
    c2 = vfma(PV, c0, c2);
    c3 = vfma(PV, c1, c3);
}

// Reduced spatial update: U1 part non-separably, then S^H(U0), S^V(U0).  9 MACs.
template <class V>
__device__ __forceinline__ void f_S_red(V& c0, V& c1, V& c2, V c3, V c1l, V c3l, V up2, V up3, V u3l,
                                        float uh, float uv) {
    const V UH = splat<V>(uh), UV = splat<V>(uv), UHV = splat<V>(uh * uv);
    c0 = vfma(UH, c1l, c0);
    c0 = vfma(UV, up2, c0);
    c0 = vfma(UHV, u3l, c0);
    c1 = vfma(UV, up3, c1);
    c2 = vfma(UH, c3l, c2);
    c0 = vfma(UH, c1, c0);
    c2 = vfma(UH, c3, c2);
    c0 = vfma(UV, c2, c0);
    c1 = vfma(UV, c3, c1);
}

// -------------------------------------------------------------- integer ----
// Reversible LeGall 5/3.  Floors are arithmetic right shifts (round toward
// -inf).  The order T^H, T^V, S^H, S^V is the definition; the non-separable
// forms reproduce it exactly by recomputing a neighbour's intermediate value
// ("nested floors") instead of reading it after a barrier.
__device__ __forceinline__ int fl2(int v) { return v >> 1; }
__device__ __forceinline__ int fl4r(int v) { return (v + 2) >> 2; }

// sign = +1 forward, -1 undo
__device__ __forceinline__ void i_TH(int& c1, int& c3, int c0, int c0r, int c2, int c2r, bool ha,
                                     int sign) {
    if (ha) {
        c1 -= sign * fl2(c0 + c0r);
        c3 -= sign * fl2(c2 + c2r);
    }
}
__device__ __forceinline__ void i_TV(int& c2, int& c3, int c0, int n0, int c1, int n1, bool va,
                                     int sign) {
    if (va) {
        c2 -= sign * fl2(c0 + n0);
        c3 -= sign * fl2(c1 + n1);
    }
}
__device__ __forceinline__ void i_SH(int& c0, int& c2, int c1, int c1l, int c3, int c3l, bool ha,
                                     int sign) {
    if (ha) {
        c0 += sign * fl4r(c1l + c1);
        c2 += sign * fl4r(c3l + c3);
    }
}
__device__ __forceinline__ void i_SV(int& c0, int& c1, int c2, int up2, int c3, int up3, bool va,
                                     int sign) {
    if (va) {
        c0 += sign * fl4r(up2 + c2);
        c1 += sign * fl4r(up3 + c3);
    }
}

// Spatial predict, forward: T^V(T^H(.)) in one step; the lower quadruple's c1
// after T^H is recomputed from its own pre-step values.
__device__ __forceinline__ void i_T_fwd(int& c1, int& c2, int& c3, int c0, int c0r, int c2r, int n0,
                                        int n1, int n0r, bool ha, bool va) {
    if (ha) {
        c1 -= fl2(c0 + c0r);
        c3 -= fl2(c2 + c2r);
        n1 -= fl2(n0 + n0r);
    }
    if (va) {
        c2 -= fl2(c0 + n0);
        c3 -= fl2(c1 + n1);
    }
}
// Spatial predict, undone: T^V undone first, then T^H; the right quadruple's
// c2 with T^V undone is recomputed.
__device__ __forceinline__ void i_T_inv(int& c1, int& c2, int& c3, int c0, int c0r, int c2r, int n0,
                                        int n1, int n0r, bool ha, bool va) {
    if (va) {
        c2r += fl2(c0r + n0r);
        c2 += fl2(c0 + n0);
        c3 += fl2(c1 + n1);
    }
    if (ha) {
        c1 += fl2(c0 + c0r);
        c3 += fl2(c2 + c2r);
    }
}
// Spatial update, forward: S^V(S^H(.)); the upper quadruple's c2 after S^H is
// recomputed.
__device__ __forceinline__ void i_S_fwd(int& c0, int& c1, int& c2, int c3, int c1l, int c3l, int up2,
                                        int up3, int u3l, bool ha, bool va) {
    if (ha) {
        c0 += fl4r(c1l + c1);
        c2 += fl4r(c3l + c3);
        up2 += fl4r(u3l + up3);
    }
    if (va) {
        c0 += fl4r(up2 + c2);
        c1 += fl4r(up3 + c3);
    }
}
// Spatial update, undone: S^V undone first, then S^H; the left quadruple's c1
// with S^V undone is recomputed.
__device__ __forceinline__ void i_S_inv(int& c0, int& c1, int& c2, int c3, int c1l, int c3l, int up2,
                                        int up3, int u3l, bool ha, bool va) {
    if (va) {
        c0 -= fl4r(up2 + c2);
        c1 -= fl4r(up3 + c3);
        c1l -= fl4r(u3l + c3l);
    }
    if (ha) {
        c0 -= fl4r(c1l + c1);
        c2 -= fl4r(c3l + c3);
    }
}

}  // namespace dwt
