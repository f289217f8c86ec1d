#pragma once
// Forward transform: the warp body of the TMA-fed warp-streaming kernels
// (one image per launch, batched, and persistent queue), 1..3 levels per
// work item.
//
// Each warp takes one work item (a strip of 64 Q1 input pixels, including a
// halo, and a segment of rows) and streams its rows through a private ring of
// shared-memory slots that the warp's lane 0 fills with 2-D TMA boxes.  The
// level-1 engine (Q1 quadruple columns per lane) emits finished rows; their
// detail bands are stored and their LL values are paired into level-2
// quadruple rows (Q1/2 columns per lane), and so on to level 3.  Values are
// stored as S (float, int, half or bfloat16) and lifted as float or int.
// Only the LL of the last fused level leaves the chip besides the detail
// bands, so a launch that fuses k levels reads the input once and
// writes every coefficient once.
#include <type_traits>

#include "dwt_engine.cuh"
#include "dwt_internal.h"
#include "dwt_tma.cuh"

namespace dwt {

// Store Q consecutive values at p; `avail` columns remain inside the band.
// keep: the next launch reads the values back (L2 evict-last).
template <class S, class T, int Q>
__device__ __forceinline__ void store_cols(S* p, const T (&v)[Q], int avail, bool vec,
                                           bool keep = false) {
    S w[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) w[j] = Storage<S>::st(v[j]);
    if (!store_ok(p, (avail < Q ? (avail > 0 ? avail : 0) : Q) * (int)sizeof(S))) return;
    if (vec && avail >= Q) {
        if (keep) st_vec_keep<S, Q>(p, w);
        else st_vec<S, Q>(p, w);
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j < avail) p[j] = w[j];
    }
}

// Border-free store of a lane's Q values at p: every column lies inside its
// band and p is vector aligned; ok = the lane stores and the row belongs to
// the work item (one predicate, no branches per column).
template <class S, class T, int Q>
__device__ __forceinline__ void st_fast(S* p, const T (&v)[Q], bool ok, bool keep = false) {
    S w[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) w[j] = Storage<S>::st(v[j]);
    if (ok && store_ok(p, Q * (int)sizeof(S))) {
        if (keep) st_vec_keep<S, Q>(p, w);
        else st_vec<S, Q>(p, w);
    }
}

// Per-level store state of one lane.
struct StoreGeo {
    int ne_r, no_r, ne_c, no_c;
    int g0;            // first quadruple column of this lane
    int r_lo, r_hi;    // rows of this level that this work item stores
    bool vec_hl, vec_lh;
};

// Row r's bands at `base` = mallat + r * pitch + g0; dlh = ne_r * pitch.
template <class S, class T, int Q>
__device__ __forceinline__ void store_details_at(const Quads<T, Q>& a, int r, const StoreGeo& g,
                                                 S* base, long long dlh, bool lane_ok) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    store_cols<S, T, Q>(base + g.ne_c, a.c[1], g.no_c - g.g0, g.vec_hl);
    if (r < g.no_r) {
        store_cols<S, T, Q>(base + dlh, a.c[2], g.ne_c - g.g0, g.vec_lh);
        store_cols<S, T, Q>(base + dlh + g.ne_c, a.c[3], g.no_c - g.g0, g.vec_hl);
    }
}

template <class S, class T, int Q>
__device__ __forceinline__ void store_details(const Quads<T, Q>& a, int r, const StoreGeo& g,
                                              S* mallat, long long pitch, bool lane_ok) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    S* row = mallat + (long long)r * pitch;
    store_cols<S, T, Q>(row + g.ne_c + g.g0, a.c[1], g.no_c - g.g0, g.vec_hl);
    if (r < g.no_r) {
        S* row2 = mallat + (long long)(g.ne_r + r) * pitch;
        store_cols<S, T, Q>(row2 + g.g0, a.c[2], g.ne_c - g.g0, g.vec_lh);
        store_cols<S, T, Q>(row2 + g.ne_c + g.g0, a.c[3], g.no_c - g.g0, g.vec_hl);
    }
}

// Row r's LL at `at` = ll + r * pitch + g0.
template <class S, class T, int Q>
__device__ __forceinline__ void store_ll_at(const Quads<T, Q>& a, int r, const StoreGeo& g, S* at,
                                            bool lane_ok, bool vec, bool keep) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    store_cols<S, T, Q>(at, a.c[0], g.ne_c - g.g0, vec, keep);
}

template <class S, class T, int Q>
__device__ __forceinline__ void store_ll(const Quads<T, Q>& a, int r, const StoreGeo& g, S* ll,
                                         long long pitch, bool lane_ok, bool vec, bool keep) {
    if (!lane_ok || r < g.r_lo || r >= g.r_hi || r >= g.ne_r) return;
    store_cols<S, T, Q>(ll + (long long)r * pitch + g.g0, a.c[0], g.ne_c - g.g0, vec, keep);
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

// Quadruple rows per slot (one TMA box of 2 SR image rows): 4, or 2 with 4
// columns per lane and at most 2 fused levels (the same 8 quadruples per
// lane per lifting step, and a box of the same bytes).
template <int NL, int Q1>
__host__ __device__ constexpr int fwd_slot_quads() { return (Q1 >= 4 && NL <= 2) ? 2 : 4; }

// All state of one warp's work item: the level engines, per-level geometry and
// the pending even LL rows, plus the static per-slot schedule.  Q1 quadruple
// columns per lane at level 1 (2 Q1 pixels), Q1/2 at level 2, Q1/4 at level 3.
template <class S, int SCH, int NL, int Q1>
struct FwdWarp {
    using T = typename Storage<S>::T;
    static constexpr int LAG = std::is_same<T, float>::value ? 2 : 1;
    static constexpr int Q2 = Q1 / 2 > 0 ? Q1 / 2 : 1;
    static constexpr int Q3 = Q1 / 4 > 0 ? Q1 / 4 : 1;
    static constexpr int BW = 64 * Q1;  // box width in pixels
    static constexpr int SR = fwd_slot_quads<NL, Q1>();  // quadruple rows per slot
    static_assert(NL <= 2 || SR == 4, "three fused levels need slots of 4 quadruple rows");
    Engine<T, Q1, SCH, true> e1;
    Engine<T, Q2, SCH, true> e2;
    Engine<T, Q3, SCH, true> e3;
    LevelCtx x1, x2, x3;
    StoreGeo s1, s2, s3;
    T pend1[Q1], pend2[Q2];
    S* mallat;
    S* ll;
    long long mpitch, llpitch;
    bool lane_ok, vec_ll;
    bool ll_keep;  // the next launch reads the LL back: store it L2 evict-last
    int lane;

    // One slot: level-1 input quadruple rows q0 .. q0+SR-1 (q0 a multiple of
    // SR) in shared memory (2 SR image rows of BW pixels), pushed as one
    // block.  With q0 % SR == 0 the rows every level emits, and how LL rows
    // pair into the next level's quadruple rows, are fixed by the pipeline lag
    // alone.
    // Level-2 input rows of the slot at q0: LL rows q0 - 2 .. q0 + SR - 3
    // paired into quadruple rows q0/2 - 1 .. q0/2 + SR/2 - 2.
    template <int R2>
    __device__ __forceinline__ void pair_level1(const Block<T, Q1, SR>& b1, Block<T, Q2, R2>& b2) {
        if constexpr (LAG == 2) {  // emitted rows q0-2 .. q0+SR-3
#pragma unroll
            for (int j = 0; j < R2; ++j) pair_rows<T, Q1>(b1.r[2 * j].c[0], b1.r[2 * j + 1].c[0], b2.r[j]);
        } else {  // emitted rows q0-1 .. q0+SR-2; row q0-2 was kept from the last slot
            pair_rows<T, Q1>(pend1, b1.r[0].c[0], b2.r[0]);
#pragma unroll
            for (int j = 1; j < R2; ++j) pair_rows<T, Q1>(b1.r[2 * j - 1].c[0], b1.r[2 * j].c[0], b2.r[j]);
            copy_arr(pend1, b1.r[SR - 1].c[0]);
        }
    }

    // Store the R2 level-2 rows a level-2 push of input rows from in2 emitted.
    template <bool EDGE, int R2>
    __device__ __forceinline__ void store_level2(const Block<T, Q2, R2>& b2, int in2) {
        const int r2 = in2 - LAG;
        if constexpr (!EDGE) {
            S* hl = mallat + (long long)r2 * mpitch + (s2.g0 + s2.ne_c);
            S* lh = hl + ((long long)s2.ne_r * mpitch - s2.ne_c);
            S* lrow = ll + (long long)r2 * llpitch + s2.g0;
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                const bool ok = lane_ok && r2 + k >= s2.r_lo && r2 + k < s2.r_hi;
                st_fast<S, T, Q2>(hl, b2.r[k].c[1], ok);
                st_fast<S, T, Q2>(lh, b2.r[k].c[2], ok);
                st_fast<S, T, Q2>(lh + s2.ne_c, b2.r[k].c[3], ok);
                hl += mpitch;
                lh += mpitch;
                if constexpr (NL == 2) {
                    st_fast<S, T, Q2>(lrow, b2.r[k].c[0], ok, ll_keep);
                    lrow += llpitch;
                }
            }
        } else {
            S* base = mallat + (long long)r2 * mpitch + s2.g0;
            const long long dlh = (long long)s2.ne_r * mpitch;
            S* lrow = ll + (long long)r2 * llpitch + s2.g0;
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                store_details_at<S, T, Q2>(b2.r[k], r2 + k, s2, base, dlh, lane_ok);
                base += mpitch;
                if constexpr (NL == 2) {
                    store_ll_at<S, T, Q2>(b2.r[k], r2 + k, s2, lrow, lane_ok, vec_ll, ll_keep);
                    lrow += llpitch;
                }
            }
        }
    }

    template <bool EDGE>
    __device__ __forceinline__ void slot(const S* sm, int q0) {
        Block<T, Q1, SR> b1;
#pragma unroll
        for (int k = 0; k < SR; ++k) {
            Quads<T, Q1>& row = b1.r[k];
            S ev[2 * Q1], od[2 * Q1];
            ld_vec<S, 2 * Q1>(ev, sm + (2 * k) * BW + 2 * Q1 * lane);
            ld_vec<S, 2 * Q1>(od, sm + (2 * k + 1) * BW + 2 * Q1 * lane);
#pragma unroll
            for (int j = 0; j < Q1; ++j) {
                row.c[0][j] = Storage<S>::ld(ev[2 * j]);
                row.c[1][j] = Storage<S>::ld(ev[2 * j + 1]);
                row.c[2][j] = Storage<S>::ld(od[2 * j]);
                row.c[3][j] = Storage<S>::ld(od[2 * j + 1]);
            }
        }
        e1.template push<EDGE, SR>(b1, q0, x1);
        const int r1 = q0 - LAG;  // first emitted level-1 row
        if constexpr (!EDGE) {
            // border-free slot: band addresses advanced by the pitch, one
            // predicate per row
            S* hl = mallat + (long long)r1 * mpitch + (s1.g0 + s1.ne_c);
            S* lh = hl + ((long long)s1.ne_r * mpitch - s1.ne_c);
            S* lrow = ll + (long long)r1 * llpitch + s1.g0;
#pragma unroll
            for (int k = 0; k < SR; ++k) {
                const bool ok = lane_ok && r1 + k >= s1.r_lo && r1 + k < s1.r_hi;
                st_fast<S, T, Q1>(hl, b1.r[k].c[1], ok);
                st_fast<S, T, Q1>(lh, b1.r[k].c[2], ok);
                st_fast<S, T, Q1>(lh + s1.ne_c, b1.r[k].c[3], ok);
                hl += mpitch;
                lh += mpitch;
                if constexpr (NL == 1) {
                    st_fast<S, T, Q1>(lrow, b1.r[k].c[0], ok, ll_keep);
                    lrow += llpitch;
                }
            }
        } else {
            // one row address per slot, advanced by the pitch (bands of row r
            // at base, base + ne_c, base + ne_r pitch (+ ne_c))
            S* base = mallat + (long long)r1 * mpitch + s1.g0;
            const long long dlh = (long long)s1.ne_r * mpitch;
            S* lrow = ll + (long long)r1 * llpitch + s1.g0;
#pragma unroll
            for (int k = 0; k < SR; ++k) {
                store_details_at<S, T, Q1>(b1.r[k], r1 + k, s1, base, dlh, lane_ok);
                base += mpitch;
                if constexpr (NL == 1) {
                    store_ll_at<S, T, Q1>(b1.r[k], r1 + k, s1, lrow, lane_ok, vec_ll, ll_keep);
                    lrow += llpitch;
                }
            }
        }
        if constexpr (NL >= 2) {
            // level-2 input rows q0/2 - 1 .. q0/2 + R2 - 2 = LL rows q0 - 2 .. q0 + SR - 3
            constexpr int R2 = SR / 2;
            Block<T, Q2, R2> b2;
            pair_level1<R2>(b1, b2);
            const int in2 = q0 / 2 - 1;
            e2.template push<EDGE, R2>(b2, in2, x2);
            store_level2<EDGE, R2>(b2, in2);
            if constexpr (NL >= 3) {
                static_assert(Q1 >= 4, "three fused levels need 4 columns per lane");
                Block<T, Q3, 1> b3;
                int in3;
                if constexpr (LAG == 2) {  // level-2 rows q0/2-3, q0/2-2; q0/2-4 kept
                    pair_rows<T, Q2>(pend2, b2.r[0].c[0], b3.r[0]);
                    copy_arr(pend2, b2.r[1].c[0]);
                    in3 = q0 / 4 - 2;
                } else {  // level-2 rows q0/2-2, q0/2-1
                    pair_rows<T, Q2>(b2.r[0].c[0], b2.r[1].c[0], b3.r[0]);
                    in3 = q0 / 4 - 1;
                }
                e3.template push<EDGE, 1>(b3, in3, x3);
                store_details<S, T, Q3>(b3.r[0], in3 - LAG, s3, mallat, mpitch, lane_ok);
                store_ll<S, T, Q3>(b3.r[0], in3 - LAG, s3, ll, llpitch, lane_ok, vec_ll, ll_keep);
            }
        }
    }
};

// Rows of level l pushed in the slot of level-1 rows [q0, q0 + sr) lie in
// [lo, hi]; the interior code is valid if every stage row touched is at least
// one row away from the top and stays clear of the last odd row.
__device__ __forceinline__ bool rows_interior(int q0, int sr, int nl, int lag, const int* no_r) {
    int lo = q0, hi = q0 + sr - 1;
    for (int l = 0; l < nl; ++l) {
        if (lo - lag - 1 < 0 || hi + 1 >= no_r[l]) return false;
        lo = floordiv2(lo - lag) - 1;
        hi = floordiv2(hi - lag);
    }
    return true;
}

// CTAs per SM the register budget is sized for: 16 warps (128 registers) with
// 2 quadruple columns per lane; with 4, 12 warps (168 registers) for slots of
// 2 quadruple rows, 8 for three fused levels.
// (measured: 13-16 warps with 4 columns, at 128 registers and 32-60 bytes
// of spills, were 2-20 % slower than 12 at 168 registers)
template <int NL, int Q1>
__host__ __device__ constexpr int fwd_min_blocks() {
    return (Q1 <= 2 ? 16 : (fwd_slot_quads<NL, Q1>() == 2 ? 12 : 8)) / kFwdWarps;
}

// One warp's work item `wid` of a launch described by `a` (input through the
// tensor map at `mapp`).
// Returns false if a bounded wait gave up (the status word is set).
template <class S, int SCH, int NL, int Q1>
__device__ __forceinline__ bool fwd_body(const CUtensorMap* mapp, const FusedArgs& a, int wid,
                                         unsigned char* smem_raw) {
    using FW = FwdWarp<S, SCH, NL, Q1>;
    using T = typename FW::T;
    constexpr int RHO = FW::LAG;
    constexpr int BW = FW::BW;
    constexpr int SR = FW::SR;
    constexpr int SLOT_ROWS = 2 * SR;  // image rows per TMA box
    static_assert(Engine<T, Q1, SCH, true>::LAG == RHO && Engine<T, 1, SCH, true>::LAG == RHO, "lag");

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    constexpr int kSlotElems = SLOT_ROWS * BW;
    S* ring = reinterpret_cast<S*>(smem_raw) + (size_t)warp * kFwdSlots * kSlotElems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kFwdWarps * kFwdSlots *
                                                              kSlotElems * sizeof(S)) +
                     warp * kFwdSlots;

    const int strip = wid % a.nstrips;
    const int xb = strip * a.valid_px - a.xoff;

    // rows of the last fused level this item produces, and the input rows it needs
    const int neN = (a.lv[NL - 1].h + 1) >> 1;
    int R0, R1;
    seg_rows(a, wid / a.nstrips, neN, R0, R1);
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
    const int qstart = max(f, 0) & ~(SR - 1);  // slots hold SR quadruple rows, aligned
    const int qend = e + 1;
    const int nslots = (qend - qstart + SR - 1) / SR;

    FW W;
    W.lane = lane;
    W.lane_ok = lane >= a.lane_lo && lane < a.lane_hi;
    W.mallat = reinterpret_cast<S*>(a.mallat);
    W.mpitch = a.mallat_pitch;
    W.ll = reinterpret_cast<S*>(a.ll);
    W.llpitch = a.ll_pitch;
    constexpr int QN = NL == 1 ? Q1 : (NL == 2 ? FW::Q2 : FW::Q3);
    W.vec_ll = (a.ll_pitch % QN) == 0;
    W.ll_keep = a.ll_keep != 0;
    int no_r[3] = {0, 0, 0};
    bool hfast = true;
    {
        const int g1 = (xb >> 1) + Q1 * lane;
        W.x1 = make_ctx(g1, Q1, a.lv[0].h, a.lv[0].w, a.lane_lo, a.lane_hi, a.lv[0].s);
        W.s1 = make_geo(a.lv[0].h, a.lv[0].w, g1, Q1, R0 << (NL - 1), R1 << (NL - 1), a.mallat_pitch);
        no_r[0] = a.lv[0].h >> 1;
        hfast = hfast && (xb >> 1) >= 2 && (xb >> 1) + 32 * Q1 + 2 <= (a.lv[0].w >> 1);
    }
    if constexpr (NL >= 2) {
        const int g2 = (xb >> 2) + FW::Q2 * lane;
        W.x2 = make_ctx(g2, FW::Q2, a.lv[1].h, a.lv[1].w, a.lane_lo, a.lane_hi, a.lv[1].s);
        W.s2 = make_geo(a.lv[1].h, a.lv[1].w, g2, FW::Q2, R0 << (NL - 2), R1 << (NL - 2), a.mallat_pitch);
        no_r[1] = a.lv[1].h >> 1;
        hfast = hfast && (xb >> 2) >= 2 && (xb >> 2) + 32 * FW::Q2 + 2 <= (a.lv[1].w >> 1);
    }
    if constexpr (NL >= 3) {
        const int g3 = (xb >> 3) + FW::Q3 * lane;
        W.x3 = make_ctx(g3, FW::Q3, a.lv[2].h, a.lv[2].w, a.lane_lo, a.lane_hi, a.lv[2].s);
        W.s3 = make_geo(a.lv[2].h, a.lv[2].w, g3, FW::Q3, R0, R1, a.mallat_pitch);
        no_r[2] = a.lv[2].h >> 1;
        hfast = hfast && (xb >> 3) >= 2 && (xb >> 3) + 32 * FW::Q3 + 2 <= (a.lv[2].w >> 1);
    }
    // the border-free code stores whole vectors only
    hfast = hfast && W.s1.vec_hl && W.s1.vec_lh && W.vec_ll;
    if constexpr (NL >= 2) hfast = hfast && W.s2.vec_hl && W.s2.vec_lh;
    if constexpr (NL >= 3) hfast = hfast && W.s3.vec_hl && W.s3.vec_lh;
    W.e1.init();
    if constexpr (NL >= 2) W.e2.init();
    if constexpr (NL >= 3) W.e3.init();
    set_store_windows(a.mallat, a.mallat_elems * (long long)sizeof(S), a.ll,
                      a.ll_elems * (long long)sizeof(S), a.err);

    // everything above came from the parameters: wait for the previous grid
    // (its output is this launch's input) only now
    grid_dependency_wait();

    // ---- TMA ring prologue
    const uint32_t ring_s = smem_u32(ring);
    const uint32_t bar_s = smem_u32(bars);
    constexpr uint32_t kSlotBytes = kSlotElems * sizeof(S);
    const int y0 = 2 * qstart;
    if (lane == 0) {
        for (int b = 0; b < kFwdSlots; ++b) mbar_init(bar_s + 8 * b, 1);
        fence_mbar_init();
        for (int s = 0; s < kFwdSlots && s < nslots; ++s) {
            mbar_arrive_expect_tx(bar_s + 8 * s, kSlotBytes);
            tma_load_2d(ring_s + s * kSlotBytes, mapp, xb, y0 + s * SLOT_ROWS, bar_s + 8 * s);
        }
    }
    __syncwarp();

    // the border-free slots form one run [si0, si1): the test holds from some
    // slot on (rows far enough from the top) and up to some slot (clear of the
    // bottom), so two scans find it instead of one test per slot
    int si0 = nslots, si1 = nslots;
    if (hfast) {
        si0 = 0;
        while (si0 < nslots && !rows_interior(qstart + SR * si0, SR, NL, RHO, no_r)) ++si0;
        si1 = nslots;
        while (si1 > si0 && !rows_interior(qstart + SR * (si1 - 1), SR, NL, RHO, no_r)) --si1;
    }

    bool failed = false;
    int s = 0;
    for (; s < nslots; ++s) {
        const int b = s % kFwdSlots;
        const bool ok = mbar_wait_bounded(bar_s + 8 * b, (s / kFwdSlots) & 1, kWaitBudget);
        if (!__all_sync(kFull, ok)) {  // keep the warp's control flow uniform
            failed = true;
            break;
        }
        const int q0 = qstart + SR * s;
        if (s >= si0 && s < si1)
            W.template slot<false>(ring + b * kSlotElems, q0);
        else
            W.template slot<true>(ring + b * kSlotElems, q0);
        __syncwarp();
        if (lane == 0 && s + kFwdSlots < nslots) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar_s + 8 * b, kSlotBytes);
            tma_load_2d(ring_s + b * kSlotBytes, mapp, xb, y0 + (s + kFwdSlots) * SLOT_ROWS,
                        bar_s + 8 * b);
        }
    }
    if (failed) {
        if (lane == 0) atomicExch(a.err, -6);
        // drain the copies still in flight before the warp leaves
        for (int t = s; t < nslots && t < s + kFwdSlots; ++t)
            mbar_wait_bounded(bar_s + 8 * (t % kFwdSlots), (t / kFwdSlots) & 1, kWaitBudget);
        return false;
    }
    // every copy has landed: the barriers may be initialised again
    if (lane == 0)
        for (int b = 0; b < kFwdSlots; ++b) mbar_inval(bar_s + 8 * b);
    __syncwarp();
    return true;
}

}  // namespace dwt
