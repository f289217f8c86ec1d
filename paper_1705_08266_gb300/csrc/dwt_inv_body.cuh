#pragma once
// Inverse transform: the warp body of the TMA-fed warp-streaming kernels (one
// image per launch, batched, and persistent queue), 1 or 2 levels per work
// item.
//
// Coarse to fine.  A warp owns a strip of output columns and a segment of
// output rows.  Each slot of its shared-memory ring holds, for four level-1
// quadruple rows, the three level-1 detail bands and (two fused levels) the
// LL and three detail bands of the two level-2 rows that produce those
// level-1 rows' LL values.  Every box is 2-D TMA; a box starts at the column
// rounded down to 16 bytes and the lane reads from the remainder on.  The
// level-2 engine runs LAG + RHO rows ahead of level 1 (its first slots of a
// work item load and push level 2 only), so the LL rows it hands down are
// exact from the first level-1 row of the item on.
#include <type_traits>

#include "dwt_engine.cuh"
#include "dwt_internal.h"
#include "dwt_tma.cuh"

namespace dwt {

constexpr int kInvWarps = kInvTmaWarps;  // warps per CTA (independent)
constexpr int kInvSlots = 3;  // ring depth per warp

// Level-1 quadruple rows per slot: 4, or 2 with 4 columns per lane (the same
// 8 quadruples per lane per lifting step as 2 columns in 4 rows).
template <int Q1>
__host__ __device__ constexpr int inv_slot_quads() { return Q1 >= 4 ? 2 : 4; }

// Box widths carry A extra elements (16 bytes) so a box can start at the
// column rounded down to 16 bytes.
template <class S, int NL, int Q1>
struct InvLayout {
    static constexpr int SR = inv_slot_quads<Q1>();  // level-1 rows per slot
    static constexpr int SR2 = SR / 2;               // level-2 rows per slot
    static constexpr int A = 16 / (int)sizeof(S);
    static constexpr int Q2 = Q1 / 2;
    static constexpr int W1 = 32 * Q1 + A;     // level-1 box width (elements)
    static constexpr int W2 = 32 * Q2 + A;     // level-2 box width
    static constexpr int E128 = 128 / (int)sizeof(S);
    static constexpr int R1 = (SR * W1 + E128 - 1) / E128 * E128;   // one level-1 box region, 128-B multiple
    static constexpr int R2 = (SR2 * W2 + E128 - 1) / E128 * E128;  // one level-2 box region
    // NL == 1: LL1 HL1 LH1 HH1; NL == 2: HL1 LH1 HH1, LL2 HL2 LH2 HH2
    static constexpr int SLOT = NL == 1 ? 4 * R1 : 3 * R1 + 4 * R2;
    static constexpr uint32_t BYTES1 = SR * W1 * sizeof(S);  // bytes one level-1 box brings
    static constexpr uint32_t BYTES2 = SR2 * W2 * sizeof(S);
};

// Lane's Q values of one band row held in shared memory at p (+ lane * Q).
template <class S, class T, int Q>
__device__ __forceinline__ void lds_cols(T (&v)[Q], const S* p) {
#pragma unroll
    for (int j = 0; j < Q; ++j) v[j] = Storage<S>::ld(p[j]);
}

template <class S, int SCH, int NL, int Q1>
struct InvWarpT {
    using T = typename Storage<S>::T;
    using Lay = InvLayout<S, NL, Q1>;
    static constexpr int LAG = std::is_same<T, float>::value ? 2 : 1;
    static constexpr int Q2 = Lay::Q2;
    Engine<T, Q1, SCH, false> e1;
    Engine<T, (Q2 > 0 ? Q2 : 1), SCH, false> e2;
    LevelCtx x1, x2;
    // column offsets of lane 0 inside each box (elements)
    int o1h, o1l, o2h, o2l;
    S* out;
    long long opitch;
    int out_h, out_w, xb, lane, A0, A1;
    int x0l;        // first output column of this lane
    bool lane_ok, vec_out;
    bool vec_row;   // this lane's 2 Q1 output columns are one aligned vector inside the row

    static constexpr int SR = Lay::SR;
    static constexpr int SR2 = Lay::SR2;

    template <bool EDGE>
    __device__ __forceinline__ void slot(const S* sm, int q0, bool level1) {
        Block<T, Q1, SR> b1;
        if constexpr (NL == 2) {
            constexpr int QQ = Q2;
            Block<T, QQ, SR2> b2;
            const S* base2 = sm + 3 * Lay::R1;
#pragma unroll
            for (int k = 0; k < SR2; ++k) {
                lds_cols<S, T, QQ>(b2.r[k].c[0], base2 + 0 * Lay::R2 + k * Lay::W2 + o2l + QQ * lane);
                lds_cols<S, T, QQ>(b2.r[k].c[1], base2 + 1 * Lay::R2 + k * Lay::W2 + o2h + QQ * lane);
                lds_cols<S, T, QQ>(b2.r[k].c[2], base2 + 2 * Lay::R2 + k * Lay::W2 + o2l + QQ * lane);
                lds_cols<S, T, QQ>(b2.r[k].c[3], base2 + 3 * Lay::R2 + k * Lay::W2 + o2h + QQ * lane);
            }
            e2.template push<EDGE, SR2>(b2, q0 / 2 + LAG, x2);
            if (!level1) return;
            // level-2 rows q0/2 .. q0/2 + SR2 - 1 -> LL rows q0 .. q0 + SR - 1 of level 1
#pragma unroll
            for (int k = 0; k < SR2; ++k) {
#pragma unroll
                for (int j = 0; j < QQ; ++j) {
                    b1.r[2 * k].c[0][2 * j] = b2.r[k].c[0][j];
                    b1.r[2 * k].c[0][2 * j + 1] = b2.r[k].c[1][j];
                    b1.r[2 * k + 1].c[0][2 * j] = b2.r[k].c[2][j];
                    b1.r[2 * k + 1].c[0][2 * j + 1] = b2.r[k].c[3][j];
                }
            }
#pragma unroll
            for (int k = 0; k < SR; ++k) {
                lds_cols<S, T, Q1>(b1.r[k].c[1], sm + 0 * Lay::R1 + k * Lay::W1 + o1h + Q1 * lane);
                lds_cols<S, T, Q1>(b1.r[k].c[2], sm + 1 * Lay::R1 + k * Lay::W1 + o1l + Q1 * lane);
                lds_cols<S, T, Q1>(b1.r[k].c[3], sm + 2 * Lay::R1 + k * Lay::W1 + o1h + Q1 * lane);
            }
        } else {
#pragma unroll
            for (int k = 0; k < SR; ++k) {
                lds_cols<S, T, Q1>(b1.r[k].c[0], sm + 0 * Lay::R1 + k * Lay::W1 + o1l + Q1 * lane);
                lds_cols<S, T, Q1>(b1.r[k].c[1], sm + 1 * Lay::R1 + k * Lay::W1 + o1h + Q1 * lane);
                lds_cols<S, T, Q1>(b1.r[k].c[2], sm + 2 * Lay::R1 + k * Lay::W1 + o1l + Q1 * lane);
                lds_cols<S, T, Q1>(b1.r[k].c[3], sm + 3 * Lay::R1 + k * Lay::W1 + o1h + Q1 * lane);
            }
        }
        e1.template push<EDGE, SR>(b1, q0, x1);
        const int r1 = q0 - LAG;
        // quadruple row r -> output rows 2r (c0 c1 interleaved) and 2r + 1
        // (c2 c3); one row address per slot, advanced by the pitch
        S* p = out + (long long)(2 * r1) * opitch + x0l;
#pragma unroll
        for (int k = 0; k < SR; ++k) {
            const int r = r1 + k;
            const bool ok = lane_ok && r >= A0 && r < A1;
            T ev[2 * Q1], od[2 * Q1];
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                ev[2 * j] = b1.r[k].c[0][j];
                ev[2 * j + 1] = b1.r[k].c[1][j];
                od[2 * j] = b1.r[k].c[2][j];
                od[2 * j + 1] = b1.r[k].c[3][j];
            }
            if constexpr (!EDGE) {
                // border-free slot: whole vectors inside the image, one predicate
                store_fast_px(ev, p, ok);
                store_fast_px(od, p + opitch, ok);
            } else if (ok) {
                store_px(ev, 2 * r, p);
                store_px(od, 2 * r + 1, p + opitch);
            }
            p += 2 * opitch;
        }
    }

    __device__ __forceinline__ void store_fast_px(const T (&v)[2 * Q1], S* p, bool ok) {
        S w[2 * Q1];
#pragma unroll
        for (int j = 0; j < 2 * Q1; ++j) w[j] = Storage<S>::st(v[j]);
        if (ok && store_ok(p, 2 * Q1 * (int)sizeof(S))) st_vec<S, 2 * Q1>(p, w);
    }

    // Output row y at p (= out + y * opitch + x0l).
    __device__ __forceinline__ void store_px(const T (&v)[2 * Q1], int y, S* p) {
        if (y >= out_h) return;
        S w[2 * Q1];
#pragma unroll
        for (int j = 0; j < 2 * Q1; ++j) w[j] = Storage<S>::st(v[j]);
        if (!store_ok(p + max(-x0l, 0), (min(x0l + 2 * Q1, out_w) - max(x0l, 0)) * (int)sizeof(S)))
            return;
        if (vec_row) {
            st_vec<S, 2 * Q1>(p, w);
        } else {
#pragma unroll
            for (int j = 0; j < 2 * Q1; ++j)
                if (x0l + j >= 0 && x0l + j < out_w) p[j] = w[j];
        }
    }
};

__device__ __forceinline__ bool inv_rows_interior(int q0, int sr, int nl, int lag, const int* no_r) {
    // level 1: rows [q0, q0 + sr - 1]; level 2: rows [q0/2 + lag, q0/2 + lag + sr/2 - 1]
    if (q0 - lag - 1 < 0 || q0 + sr >= no_r[0]) return false;
    if (nl >= 2) {
        const int lo = q0 / 2 + lag;
        if (lo - lag - 1 < 0 || lo + sr / 2 >= no_r[1]) return false;
    }
    return true;
}

// Returns false if a bounded wait gave up (the status word is set).
template <class S, int SCH, int NL, int Q1>
__device__ __forceinline__ bool inv_body(const CUtensorMap* m1p, const CUtensorMap* m2p,
                                         const CUtensorMap* mlp, const FusedArgs& a, int wid,
                                         unsigned char* smem_raw) {
    using W = InvWarpT<S, SCH, NL, Q1>;
    using Lay = InvLayout<S, NL, Q1>;
    constexpr int LAG = W::LAG;
    constexpr int RHO = LAG;
    constexpr int SR = Lay::SR;
    constexpr int PRO = NL == 2 ? 2 * LAG : 0;  // level-2 rows pushed ahead (LAG + RHO)
    constexpr int PRO_SLOTS = PRO / (SR / 2);    // slots that feed level 2 only

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    S* ring = reinterpret_cast<S*>(smem_raw) + (size_t)warp * kInvSlots * Lay::SLOT;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kInvWarps * kInvSlots *
                                                              Lay::SLOT * sizeof(S)) +
                     warp * kInvSlots;

    const int strip = wid % a.nstrips;
    W w;
    w.lane = lane;
    w.xb = strip * a.valid_px - a.xoff;
    w.lane_ok = lane >= a.lane_lo && lane < a.lane_hi;
    w.out = reinterpret_cast<S*>(a.out);
    w.opitch = a.out_pitch;
    w.out_h = a.lv[0].h;
    w.out_w = a.lv[0].w;
    w.vec_out = (a.out_pitch % (2 * Q1)) == 0;
    w.x0l = w.xb + 2 * Q1 * lane;
    set_store_windows(a.out, a.out_elems * (long long)sizeof(S), nullptr, 0, a.err);
    w.vec_row = w.vec_out && w.x0l >= 0 && w.x0l + 2 * Q1 <= a.lv[0].w;
    const int ne1 = (a.lv[0].h + 1) >> 1;
    seg_rows(a, wid / a.nstrips, ne1, w.A0, w.A1);

    int no_r[2] = {a.lv[0].h >> 1, NL >= 2 ? (a.lv[1].h >> 1) : 0};
    const int g1w = w.xb >> 1;
    const int ne_c1 = (a.lv[0].w + 1) >> 1, ne_r1 = ne1;
    w.x1 = make_ctx(g1w + Q1 * lane, Q1, a.lv[0].h, a.lv[0].w, a.lane_lo, a.lane_hi, a.lv[0].s);
    const int xh1 = ne_c1 + g1w, xl1 = g1w;
    constexpr int AM = Lay::A - 1;
    const int bx1h = xh1 & ~AM, bx1l = xl1 & ~AM;
    w.o1h = xh1 - bx1h;
    w.o1l = xl1 - bx1l;
    bool hfast = g1w >= 2 && g1w + 32 * Q1 + 2 <= (a.lv[0].w >> 1);
    int bx2h = 0, bx2l = 0, ne_r2 = 0;
    if constexpr (NL >= 2) {
        const int g2w = w.xb >> 2;
        const int ne_c2 = (a.lv[1].w + 1) >> 1;
        ne_r2 = (a.lv[1].h + 1) >> 1;
        w.x2 = make_ctx(g2w + W::Q2 * lane, W::Q2, a.lv[1].h, a.lv[1].w, a.lane_lo, a.lane_hi, a.lv[1].s);
        const int xh2 = ne_c2 + g2w, xl2 = g2w;
        bx2h = xh2 & ~AM;
        bx2l = xl2 & ~AM;
        w.o2h = xh2 - bx2h;
        w.o2l = xl2 - bx2l;
        hfast = hfast && g2w >= 2 && g2w + 32 * W::Q2 + 2 <= (a.lv[1].w >> 1);
    }
    hfast = hfast && w.vec_out;  // the border-free code stores whole vectors
    w.e1.init();
    if constexpr (NL >= 2) w.e2.init();

    // level-1 input rows of this item: outputs [A0, A1) need [A0 - RHO, A1 - 1 + LAG]
    const int qstart = max(w.A0 - RHO, 0) & ~(SR - 1);
    const int nmain = (w.A1 + LAG - qstart + SR - 1) / SR;
    const int nslots = nmain + PRO_SLOTS;
    const int qbase = qstart - SR * PRO_SLOTS;

    // everything above came from the parameters: wait for the previous grid
    // (its output is this launch's input) only now
    grid_dependency_wait();

    const uint32_t ring_s = smem_u32(ring);
    const uint32_t bar_s = smem_u32(bars);
    auto issue = [&](int s) {
        const int b = s % kInvSlots;
        const uint32_t dst = ring_s + (uint32_t)(b * Lay::SLOT * sizeof(S));
        const uint32_t bar = bar_s + 8 * b;
        const int q0 = qbase + SR * s;
        const bool l1 = s >= PRO_SLOTS;
        uint32_t bytes = 0;
        if (l1) bytes += (NL == 1 ? 4 : 3) * Lay::BYTES1;
        if (NL == 2) bytes += 4 * Lay::BYTES2;
        mbar_arrive_expect_tx(bar, bytes);
        if constexpr (NL == 1) {
            tma_load_2d(dst + 0 * Lay::R1 * sizeof(S), mlp, bx1l, q0, bar);
            tma_load_2d(dst + 1 * Lay::R1 * sizeof(S), m1p, bx1h, q0, bar);
            tma_load_2d(dst + 2 * Lay::R1 * sizeof(S), m1p, bx1l, ne_r1 + q0, bar);
            tma_load_2d(dst + 3 * Lay::R1 * sizeof(S), m1p, bx1h, ne_r1 + q0, bar);
        } else {
            if (l1) {
                tma_load_2d(dst + 0 * Lay::R1 * sizeof(S), m1p, bx1h, q0, bar);
                tma_load_2d(dst + 1 * Lay::R1 * sizeof(S), m1p, bx1l, ne_r1 + q0, bar);
                tma_load_2d(dst + 2 * Lay::R1 * sizeof(S), m1p, bx1h, ne_r1 + q0, bar);
            }
            const uint32_t d2 = dst + 3 * Lay::R1 * sizeof(S);
            const int y2 = q0 / 2 + LAG;
            tma_load_2d(d2 + 0 * Lay::R2 * sizeof(S), mlp, bx2l, y2, bar);
            tma_load_2d(d2 + 1 * Lay::R2 * sizeof(S), m2p, bx2h, y2, bar);
            tma_load_2d(d2 + 2 * Lay::R2 * sizeof(S), m2p, bx2l, ne_r2 + y2, bar);
            tma_load_2d(d2 + 3 * Lay::R2 * sizeof(S), m2p, bx2h, ne_r2 + y2, bar);
        }
    };
    if (lane == 0) {
        for (int b = 0; b < kInvSlots; ++b) mbar_init(bar_s + 8 * b, 1);
        fence_mbar_init();
        for (int s = 0; s < kInvSlots && s < nslots; ++s) issue(s);
    }
    __syncwarp();

    // the border-free slots form one run [si0, si1) (see the forward body)
    int si0 = nslots, si1 = nslots;
    if (hfast) {
        si0 = 0;
        while (si0 < nslots && !inv_rows_interior(qbase + SR * si0, SR, NL, LAG, no_r)) ++si0;
        si1 = nslots;
        while (si1 > si0 && !inv_rows_interior(qbase + SR * (si1 - 1), SR, NL, LAG, no_r)) --si1;
    }

    bool failed = false;
    int s = 0;
    for (; s < nslots; ++s) {
        const int b = s % kInvSlots;
        const bool ok = mbar_wait_bounded(bar_s + 8 * b, (s / kInvSlots) & 1, kWaitBudget);
        if (!__all_sync(kFull, ok)) {
            failed = true;
            break;
        }
        const int q0 = qbase + SR * s;
        const bool l1 = s >= PRO_SLOTS;
        if (s >= si0 && s < si1)
            w.template slot<false>(ring + b * Lay::SLOT, q0, l1);
        else
            w.template slot<true>(ring + b * Lay::SLOT, q0, l1);
        __syncwarp();
        if (lane == 0 && s + kInvSlots < nslots) {
            fence_proxy_async_smem();
            issue(s + kInvSlots);
        }
    }
    if (failed) {
        if (lane == 0) atomicExch(a.err, -6);
        for (int t = s; t < nslots && t < s + kInvSlots; ++t)
            mbar_wait_bounded(bar_s + 8 * (t % kInvSlots), (t / kInvSlots) & 1, kWaitBudget);
        return false;
    }
    // every copy has landed: the barriers may be initialised again
    if (lane == 0)
        for (int b = 0; b < kInvSlots; ++b) mbar_inval(bar_s + 8 * b);
    __syncwarp();
    return true;
}

}  // namespace dwt
