// Multipass schemes: every lifting step is one kernel over the whole level,
// exchanging all coefficients through HBM.
//
// This restates the paper's pixel-shader mapping (Sec. 3, last paragraphs:
// data live in 2-D textures, nothing is kept in registers, every barrier step
// is a separate pass and results travel through off-chip memory) as CUDA
// kernels.  One thread owns one quadruple.  Neighbours are read at mirrored
// sample positions (whole-sample symmetric extension of the pre-step values,
// which the symmetric lifting filters keep exact), so no special case is
// needed at the borders.  The separable scheme makes four passes per lifting
// pair, the non-separable schemes two: the step count of Table 1 becomes the
// number of HBM round trips.
#include <type_traits>

#include "dwt_internal.h"
#include "dwt_steps.cuh"

namespace dwt {

__device__ __forceinline__ int mirror(int x, int n) {
    if (x < 0) x = -x;
    if (x >= n) x = 2 * (n - 1) - x;
    return min(max(x, 0), n - 1);
}

template <class T>
struct Access {
    Layout L;
    int h, w, ne_r, ne_c;
    // address of sample (y, x) of the level, y < h, x < w
    __device__ __forceinline__ T* at(int y, int x) const {
        T* base = reinterpret_cast<T*>(const_cast<void*>(L.p));
        if (L.kind == 0) return base + (long long)y * L.pitch + x;
        const int r = y >> 1, c = x >> 1;
        switch (((y & 1) << 1) | (x & 1)) {
            case 0: return reinterpret_cast<T*>(const_cast<void*>(L.ll)) + (long long)r * L.ll_pitch + c;
            case 1: return base + (long long)r * L.pitch + ne_c + c;
            case 2: return base + (long long)(ne_r + r) * L.pitch + c;
            default: return base + (long long)(ne_r + r) * L.pitch + ne_c + c;
        }
    }
};

template <class T>
__device__ __forceinline__ T scale_v(T v, float s);
template <>
__device__ __forceinline__ float scale_v<float>(float v, float s) { return v * s; }
template <>
__device__ __forceinline__ int scale_v<int>(int v, float) { return v; }

template <class T, int KIND, bool FWD>
__global__ void __launch_bounds__(256) pass_kernel(const PassArgs a) {
    const int qc = blockIdx.x * blockDim.x + threadIdx.x;
    const int qr = blockIdx.y * blockDim.y + threadIdx.y;
    const int ne_r = (a.h + 1) >> 1, ne_c = (a.w + 1) >> 1;
    if (qr >= ne_r || qc >= ne_c) return;
    Access<T> src{a.src, a.h, a.w, ne_r, ne_c};
    Access<T> dst{a.dst, a.h, a.w, ne_r, ne_c};
    // component k of quadruple (r, c), mirrored into the level
    auto ld = [&](int k, int r, int c) -> T {
        const int y = mirror(2 * r + (k >> 1), a.h);
        const int x = mirror(2 * c + (k & 1), a.w);
        const T v = *src.at(y, x);
        return a.scale_in ? scale_v<T>(v, a.s[k]) : v;
    };
    const bool ha = a.w > 1, va = a.h > 1;
    const float ph = ha ? a.coef : 0.f, pv = va ? a.coef : 0.f;
    constexpr int sgn = FWD ? 1 : -1;
    T c0 = ld(0, qr, qc), c1 = ld(1, qr, qc), c2 = ld(2, qr, qc), c3 = ld(3, qr, qc);
    constexpr bool F = std::is_same<T, float>::value;

    if constexpr (KIND == P_TH) {
        const T c0r = ld(0, qr, qc + 1), c2r = ld(2, qr, qc + 1);
        if constexpr (F) f_TH(c1, c3, c0, c0r, c2, c2r, ph);
        else i_TH(c1, c3, c0, c0r, c2, c2r, ha, sgn);
    } else if constexpr (KIND == P_TV) {
        const T n0 = ld(0, qr + 1, qc), n1 = ld(1, qr + 1, qc);
        if constexpr (F) f_TV(c2, c3, c0, n0, c1, n1, pv);
        else i_TV(c2, c3, c0, n0, c1, n1, va, sgn);
    } else if constexpr (KIND == P_SH) {
        const T c1l = ld(1, qr, qc - 1), c3l = ld(3, qr, qc - 1);
        if constexpr (F) f_SH(c0, c2, c1, c1l, c3, c3l, ph);
        else i_SH(c0, c2, c1, c1l, c3, c3l, ha, sgn);
    } else if constexpr (KIND == P_SV) {
        const T up2 = ld(2, qr - 1, qc), up3 = ld(3, qr - 1, qc);
        if constexpr (F) f_SV(c0, c1, c2, up2, c3, up3, pv);
        else i_SV(c0, c1, c2, up2, c3, up3, va, sgn);
    } else if constexpr (KIND == P_T || KIND == P_TR) {
        const T c0r = ld(0, qr, qc + 1), c2r = ld(2, qr, qc + 1);
        const T n0 = ld(0, qr + 1, qc), n1 = ld(1, qr + 1, qc), n0r = ld(0, qr + 1, qc + 1);
        if constexpr (F) {
            if constexpr (KIND == P_T) f_T_plain(c1, c2, c3, c0, c0r, c2r, n0, n1, n0r, ph, pv);
            else f_T_red(c1, c2, c3, c0, c0r, c2r, n0, n1, n0r, ph, pv);
        } else {
            if constexpr (FWD) i_T_fwd(c1, c2, c3, c0, c0r, c2r, n0, n1, n0r, ha, va);
            else i_T_inv(c1, c2, c3, c0, c0r, c2r, n0, n1, n0r, ha, va);
        }
    } else {  // P_S, P_SR
        const T c1l = ld(1, qr, qc - 1), c3l = ld(3, qr, qc - 1);
        const T up2 = ld(2, qr - 1, qc), up3 = ld(3, qr - 1, qc), u3l = ld(3, qr - 1, qc - 1);
        if constexpr (F) {
            if constexpr (KIND == P_S) f_S_plain(c0, c1, c2, c3, c1l, c3l, up2, up3, u3l, ph, pv);
            else f_S_red(c0, c1, c2, c3, c1l, c3l, up2, up3, u3l, ph, pv);
        } else {
            if constexpr (FWD) i_S_fwd(c0, c1, c2, c3, c1l, c3l, up2, up3, u3l, ha, va);
            else i_S_inv(c0, c1, c2, c3, c1l, c3l, up2, up3, u3l, ha, va);
        }
    }

    const T v[4] = {c0, c1, c2, c3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int y = 2 * qr + (k >> 1), x = 2 * qc + (k & 1);
        if (y < a.h && x < a.w) *dst.at(y, x) = a.scale_out ? scale_v<T>(v[k], a.s[k]) : v[k];
    }
}

template <class T, bool FWD>
static cudaError_t launch_kind(int kind, const PassArgs& a, cudaStream_t st) {
    const dim3 block(64, 4);
    const dim3 grid(((a.w + 1) / 2 + block.x - 1) / block.x, ((a.h + 1) / 2 + block.y - 1) / block.y);
    switch (kind) {
        case P_TH: pass_kernel<T, P_TH, FWD><<<grid, block, 0, st>>>(a); break;
        case P_TV: pass_kernel<T, P_TV, FWD><<<grid, block, 0, st>>>(a); break;
        case P_SH: pass_kernel<T, P_SH, FWD><<<grid, block, 0, st>>>(a); break;
        case P_SV: pass_kernel<T, P_SV, FWD><<<grid, block, 0, st>>>(a); break;
        case P_T: pass_kernel<T, P_T, FWD><<<grid, block, 0, st>>>(a); break;
        case P_S: pass_kernel<T, P_S, FWD><<<grid, block, 0, st>>>(a); break;
        case P_TR: pass_kernel<T, P_TR, FWD><<<grid, block, 0, st>>>(a); break;
        case P_SR: pass_kernel<T, P_SR, FWD><<<grid, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pass(int elem, int kind, bool fwd, const PassArgs& a, cudaStream_t st) {
    if (elem == 0) return fwd ? launch_kind<float, true>(kind, a, st) : launch_kind<float, false>(kind, a, st);
    return fwd ? launch_kind<int, true>(kind, a, st) : launch_kind<int, false>(kind, a, st);
}

}  // namespace dwt
