// Separable convolution scheme N^V | N^H (Sec. 2, Eq. 1): the CDF 9/7 analysis
// filter bank G0 (9 taps, low) and G1 (7 taps, high) followed by subsampling,
// first along rows, then along columns, one level per launch.
//
// A CTA owns a 64 x 64 output tile: it loads the tile plus a 4-pixel halo
// (whole-sample symmetric extension by mirrored indices) into shared memory,
// filters every row of the halo-extended tile horizontally (step N^H), waits
// on one barrier, filters the columns of both half-results vertically (step
// N^V), scales nothing (the taps already carry the normalisation) and writes
// the four bands.  Taps come from the host, derived from the lifting steps.
#include <type_traits>

#include "dwt_engine.cuh"
#include "dwt_internal.h"

namespace dwt {

constexpr int kConvTile = 64;                  // output pixels per tile side
constexpr int kConvHalo = 4;                   // 9/7 analysis support radius
constexpr int kConvIn = kConvTile + 2 * kConvHalo;  // 72

__device__ __forceinline__ int cmirror(int x, int n) {
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    x %= period;
    if (x < 0) x += period;
    return x >= n ? period - x : x;
}

template <class S>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const ConvArgs a) {
    using T = typename Storage<S>::T;
    __shared__ float tin[kConvIn][kConvIn + 1];
    __shared__ float lo[kConvIn][kConvTile / 2 + 1];
    __shared__ float hi[kConvIn][kConvTile / 2 + 1];
    const int tx0 = blockIdx.x * kConvTile, ty0 = blockIdx.y * kConvTile;
    const int h = a.h, w = a.w;
    const S* src = reinterpret_cast<const S*>(a.src);
    // load the halo-extended tile through mirrored indices
    for (int i = threadIdx.x; i < kConvIn * kConvIn; i += blockDim.x) {
        const int r = i / kConvIn, c = i % kConvIn;
        const int y = cmirror(ty0 - kConvHalo + r, h), x = cmirror(tx0 - kConvHalo + c, w);
        tin[r][c] = (float)Storage<S>::ld(src[(long long)y * a.src_pitch + x]);
    }
    __syncthreads();
    // N^H: low[n] = sum h[k] x[2n + k], high[n] = sum g[k] x[2n + 1 + k]
    const bool hact = w > 1, vact = h > 1;
    for (int i = threadIdx.x; i < kConvIn * (kConvTile / 2); i += blockDim.x) {
        const int r = i / (kConvTile / 2), n = i % (kConvTile / 2);
        const int c = kConvHalo + 2 * n;  // column of x[2n] in the tile
        float l = 0.f, g = 0.f;
        if (hact) {
#pragma unroll
            for (int k = -4; k <= 4; ++k) l = fmaf(a.h0[k + 4], tin[r][c + k], l);
#pragma unroll
            for (int k = -3; k <= 3; ++k) g = fmaf(a.g0[k + 3], tin[r][c + 1 + k], g);
        } else {
            l = tin[r][c];
        }
        lo[r][n] = l;
        hi[r][n] = g;
    }
    __syncthreads();
    // N^V on both half-bands, then the band writes
    S* dst = reinterpret_cast<S*>(a.dst);
    S* ll = reinterpret_cast<S*>(a.ll);
    const int ne_r = (h + 1) >> 1, no_r = h >> 1, ne_c = (w + 1) >> 1, no_c = w >> 1;
    for (int i = threadIdx.x; i < (kConvTile / 2) * (kConvTile / 2); i += blockDim.x) {
        const int m = i / (kConvTile / 2), n = i % (kConvTile / 2);
        const int r = kConvHalo + 2 * m;
        float ll_ = 0.f, lh_ = 0.f, hl_ = 0.f, hh_ = 0.f;
        if (vact) {
#pragma unroll
            for (int k = -4; k <= 4; ++k) {
                ll_ = fmaf(a.h0[k + 4], lo[r + k][n], ll_);
                hl_ = fmaf(a.h0[k + 4], hi[r + k][n], hl_);
            }
#pragma unroll
            for (int k = -3; k <= 3; ++k) {
                lh_ = fmaf(a.g0[k + 3], lo[r + 1 + k][n], lh_);
                hh_ = fmaf(a.g0[k + 3], hi[r + 1 + k][n], hh_);
            }
        } else {
            ll_ = lo[r][n];
            hl_ = hi[r][n];
        }
        const int qr = ty0 / 2 + m, qc = tx0 / 2 + n;
        if (qr < ne_r && qc < ne_c) ll[(long long)qr * a.ll_pitch + qc] = Storage<S>::st(ll_);
        if (qr < ne_r && qc < no_c) dst[(long long)qr * a.dst_pitch + ne_c + qc] = Storage<S>::st(hl_);
        if (qr < no_r && qc < ne_c) dst[(long long)(ne_r + qr) * a.dst_pitch + qc] = Storage<S>::st(lh_);
        if (qr < no_r && qc < no_c)
            dst[(long long)(ne_r + qr) * a.dst_pitch + ne_c + qc] = Storage<S>::st(hh_);
    }
}

cudaError_t launch_conv_fwd(int elem, const ConvArgs& a, cudaStream_t st) {
    const dim3 grid((a.w + kConvTile - 1) / kConvTile, (a.h + kConvTile - 1) / kConvTile);
    switch (elem) {
        case 0: conv_fwd_kernel<float><<<grid, 256, 0, st>>>(a); break;
        case 2: conv_fwd_kernel<__half><<<grid, 256, 0, st>>>(a); break;
        case 3: conv_fwd_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dwt
