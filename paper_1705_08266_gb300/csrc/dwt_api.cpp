// C ABI of the library: plans, workspace layout, level grouping, dispatch.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "dwt2d.h"
#include "dwt_internal.h"

using namespace dwt;

namespace {

constexpr size_t kHeader = 256;  // status word + padding at the start of the workspace

struct Group {
    int first;  // first level of the group (0-based)
    int n;      // levels fused
};

}  // namespace

constexpr int kMaxHostBands = 64;  // row bands of the pipelined host-buffer entry points

struct dwt2d_plan_s {
    int H, W, levels;
    dwt2d_wavelet wavelet;
    dwt2d_scheme scheme;
    dwt2d_dtype dtype;
    int elem;         // bytes per element
    int hs[17], ws[17];  // extent transformed by level l (l = 0 .. levels-1)
    Group groups[16];
    int ngroups;
    int sm_count;
    long long l2_bytes;  // L2 cache of the device the plan was made on
    int fwd_warps_target, inv_warps_target;
    // a forward launch whose rows allow segments of at least large_segq rows
    // at fwd_warps_large warps runs that many (several waves even out the
    // strips' unequal costs); smaller launches keep fwd_warps_target
    int fwd_warps_large, large_segq;
    int inv_warps_large;  // the same rule for inverse launches
    int fwd_q1;  // quadruple columns per lane of the forward kernel (2 or 4; 0: automatic)
    int fwd_warps_large4, fwd_short4;  // the large-launch rule at 4 columns per lane
    int inv_warps_large4;
    int inv_q1;  // the same for the inverse
    int min_segq;
    int pdl;  // device entry points: launches with programmatic stream serialization
    int fwd_short, inv_short;  // short last-wave segments: divisor (0: off)
    int fwd_seg_f;  // forward segment interleave (0: as many groups as waves)
    int inv_seg_f;  // inverse segment interleave (0: as many groups as waves)
    int host_pipeline;  // *_host entry points overlap copies and transform
    // workspace layout (bytes from the start of the workspace)
    size_t off_a, off_b, off_x, off_y;
    size_t size_a, size_b;  // bytes of the two LL buffers
    long long pitch_a, pitch_b, pitch_x;  // elements
    size_t ws_bytes;
    // profiling hook: events[2i] / events[2i+1] around launch i
    cudaEvent_t* events;
    int nevents;
    // host-buffer forward: copy streams and events (created on first use)
    bool host_ready;
    cudaStream_t host_in, host_out;
    cudaEvent_t host_ev[2 * kMaxHostBands + 3];
    int host_bands;  // row bands of the pipelined host-buffer entry points
};

// A batch: per-image plans, workspace regions and the launch list.
struct dwt2d_batch_s {
    struct Launch {
        int fwd, elem_kind, nl;
        int first, count;  // entries [first, first + count) of the table
        int grid;
    };
    dwt2d_scheme scheme;
    bool pdl;  // launches with programmatic stream serialization
    int q1;    // quadruple columns per lane of every launch (2 or 4)
    std::vector<dwt2d_batch_item> items;
    std::vector<dwt2d_plan_s*> plans;
    std::vector<size_t> region;             // workspace offset of each image's LL buffers
    std::vector<Launch> launches;            // in issue order
    std::vector<std::pair<int, int>> refs;   // table entry -> (image, launch k of the image)
    std::vector<int> segq;                   // table entry -> rows per warp (quadruple rows)
    std::vector<dwt::BatchEntry> table;      // host copy, filled at upload
    size_t table_off, ws_bytes;
    long long warps;
    // queue mode: one persistent launch per (direction, storage type) over a
    // queue of every level group's work items; qtable holds the entries queue
    // by queue (table index order within a queue), counters the queue heads
    // and one done counter per (image, level group)
    bool queue;
    struct Queue {
        int fwd, elem_kind;
        int first, count;  // entries [first, first + count) of qtable
        long long items;
    };
    std::vector<Queue> queues;
    std::vector<int> qorder;                 // qtable entry -> table entry
    std::vector<dwt::BatchEntry> qtable;
    size_t qtable_off, counters_off, counters_bytes;
    int max_groups, sms;
    ~dwt2d_batch_s() {
        for (auto* p : plans) free(p);
    }
};

namespace {

long long round_pitch(long long w, int elem) {
    const long long bytes = (w * elem + 15) / 16 * 16;
    return bytes / elem;
}

bool multipass(dwt2d_scheme s) {
    return s >= DWT2D_SEPARABLE_MULTIPASS && s <= DWT2D_NONSEP_REDUCED_MULTIPASS;
}
bool convolution(dwt2d_scheme s) { return s == DWT2D_SEPARABLE_CONVOLUTION; }

// CDF 9/7 analysis filters (low: 9 taps, high: 7 taps, centred) derived from
// the lifting steps: the impulse responses of one 1-D forward lifting pass
// (Eq. 2 factors Eq. 1), computed in double precision.
void cdf97_taps(float h0[9], float g0[7]) {
    const double a = -1.586134342059924, b = -0.052980118572961, c = 0.882911075530934,
                 d = 0.443506852043971, K = 1.230174104914001;
    const int N = 40;
    for (int p = 20; p <= 21; ++p) {
        double x[N] = {0};
        x[p] = 1.0;
        const double pu[2][2] = {{a, b}, {c, d}};
        for (int k = 0; k < 2; ++k) {
            for (int i = 1; i + 1 < N; i += 2) x[i] += pu[k][0] * (x[i - 1] + x[i + 1]);
            for (int i = 2; i + 1 < N; i += 2) x[i] += pu[k][1] * (x[i - 1] + x[i + 1]);
        }
        for (int n = 0; 2 * n < N; ++n) {
            const int kh = p - 2 * n, kg = p - 2 * n - 1;
            if (kh >= -4 && kh <= 4) h0[kh + 4] = (float)(x[2 * n] / K);
            if (kg >= -3 && kg <= 3 && 2 * n + 1 < N) g0[kg + 3] = (float)(x[2 * n + 1] * K);
        }
    }
}

int base_scheme(dwt2d_scheme s) {
    switch (s) {
        case DWT2D_SEPARABLE_CONVOLUTION: return SCH_RED;  // its inverse
        case DWT2D_SEPARABLE:
        case DWT2D_SEPARABLE_MULTIPASS: return SCH_SEP;
        case DWT2D_NONSEP:
        case DWT2D_NONSEP_MULTIPASS: return SCH_NONSEP;
        default: return SCH_RED;
    }
}


void level_scale(int h, int w, bool inverse, float s[4]) {
    const double K = 1.230174104914001;
    const double kh = w > 1 ? K : 1.0, kv = h > 1 ? K : 1.0;
    // each factor computed directly (not as a reciprocal of the other
    // direction's), the way the kernels' border-free code rounds its constants
    const double f[4] = {1.0 / (kh * kv), kh / kv, kv / kh, kh * kv};
    const double g[4] = {kh * kv, kv / kh, kh / kv, 1.0 / (kh * kv)};
    for (int k = 0; k < 4; ++k) s[k] = (float)(inverse ? g[k] : f[k]);
}

// Lanes whose every column at the deepest fused level is valid, for a warp of
// 32 lanes x 4 level-1 quadruple columns and a lifting radius rho (quadruples).
void valid_lanes(int nl, int rho, int q1, int* lo_out, int* hi_out) {
    int lo = rho, hi = 32 * q1 - rho;  // level-1 valid quadruple columns [lo, hi)
    for (int l = 2; l <= nl; ++l) {
        const int nlo = (lo + 2 * rho + 1) / 2;          // ceil((lo + 2 rho) / 2)
        const int nhi = (hi - 2 - 2 * rho) / 2 + 1;      // floor((hi - 2 - 2 rho) / 2) + 1
        lo = nlo;
        hi = nhi;
    }
    const int q = q1 >> (nl - 1);
    int llo = 32, lhi = 0;
    for (int l = 0; l < 32; ++l) {
        if (l * q >= lo && l * q + q <= hi) {
            if (l < llo) llo = l;
            lhi = l + 1;
        }
    }
    *lo_out = llo;
    *hi_out = lhi;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// kind: 0 float32, 1 int32, 2 float16, 3 bfloat16
dwt2d_status make_map(CUtensorMap* map, const void* base, int h, int w, long long pitch_elems,
                      int elem, int kind, int box_w, int box_h = kFwdSlotRows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return DWT2D_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * elem)};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = kind == 1   ? CU_TENSOR_MAP_DATA_TYPE_INT32
                                   : kind == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : kind == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUresult r = fn(map, dt,
                          2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DWT2D_OK : DWT2D_ERR_CUDA;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

dwt2d_status check_buffers(const dwt2d_plan_s* p, const void* src, int64_t sp, const void* dst,
                           int64_t dp, const void* ws) {
    if (!p || !src || !dst || !ws) return DWT2D_ERR_INVALID;
    if (!aligned16(src) || !aligned16(dst) || !aligned16(ws)) return DWT2D_ERR_ALIGN;
    if (sp % 16 || dp % 16) return DWT2D_ERR_ALIGN;
    const int64_t row = (int64_t)p->W * p->elem;
    if (sp < row || dp < row) return DWT2D_ERR_INVALID;
    return DWT2D_OK;
}

// Warps of a streaming kernel resident per SM (their register budgets).
int resident_per_sm(bool fwd, int nl, int q1, int scheme) {
    if (fwd) return q1 <= 2 ? 16 : (nl <= 2 ? 12 : 8);
    return q1 <= 2 ? (scheme == SCH_NONSEP ? 12 : 16) : 12;
}

// Warp work decomposition of one streaming launch.
// Rows per warp: enough segments for target_warps warps, or segq_fixed (> 0).
// With short_div > 1 the rows at the bottom that one wave of resident warps
// (resident per SM) takes are cut into segments short_div times shorter and
// taken last: the launch's last warps are short, so it drains quickly.
void decompose(const dwt2d_plan_s* p, int w_first, int rows, int nl, int rho, int q1,
               int target_warps, FusedArgs* a, int* grid, int warps_per_block, int segq_fixed = 0,
               int resident = 16, int short_div = 0, int seg_f_opt = 0) {
    valid_lanes(nl, rho, q1, &a->lane_lo, &a->lane_hi);
    const int qn = q1 >> (nl - 1);
    const int ppl = qn * (1 << nl);  // input pixels per lane
    // TMA boxes start at a multiple of 16 bytes: strip starts must be aligned
    const int align = 16 / p->elem;
    while ((a->lane_lo * ppl) % align) ++a->lane_lo;
    while (((a->lane_hi - a->lane_lo) * ppl) % align) --a->lane_hi;
    a->valid_px = (a->lane_hi - a->lane_lo) * ppl;
    a->xoff = a->lane_lo * ppl;
    a->nstrips = (w_first + a->valid_px - 1) / a->valid_px;
    int segq = segq_fixed;
    if (segq <= 0) {
        int nsegs = target_warps / a->nstrips;
        if (nsegs < 1) nsegs = 1;
        segq = (rows + nsegs - 1) / nsegs;
    }
    if (segq < p->min_segq) segq = p->min_segq;
    if (segq > rows) segq = rows;
    if (segq < 1) segq = 1;
    a->segq = segq;
    a->nsegs = (rows + segq - 1) / segq;
    a->nbig = a->nsegs;
    a->segq2 = segq;
    const int res_warps = p->sm_count * resident;
    if (short_div > 1 && segq_fixed <= 0) {
        const int sq2 = std::max(std::max(p->min_segq, 1), segq / short_div);
        const int nshort = std::max(1, res_warps / a->nstrips);  // one wave of short segments
        const int big = (rows - nshort * sq2) / segq;               // whole long segments above them
        if (sq2 < segq && big >= 1) {
            a->nbig = big;
            a->segq2 = sq2;
            a->nsegs = big + (rows - big * segq + sq2 - 1) / sq2;
        }
    }
    const int items = a->nstrips * a->nsegs;
    *grid = (items + warps_per_block - 1) / warps_per_block;
    // long segments in as many interleaved groups as they fill waves of
    // resident warps, so vertically adjacent segments run one after the other
    // and share their halo rows through L2 (measured 1-2 %)
    const int big_items = a->nstrips * a->nbig;
    a->seg_f = seg_f_opt > 0 ? seg_f_opt : (big_items + res_warps / 2) / res_warps;
    if (a->seg_f < 1) a->seg_f = 1;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void mark(const dwt2d_plan_s* p, int launch, int side, cudaStream_t st) {
    if (p->events && launch < p->nevents) cudaEventRecord(p->events[2 * launch + side], st);
}

int elem_kind_of(dwt2d_dtype d) {
    switch (d) {
        case DWT2D_I32: return 1;
        case DWT2D_F16: return 2;
        case DWT2D_BF16: return 3;
        default: return 0;
    }
}

// One streaming launch of a plan: level group `gi`, its argument block, its
// tensor maps and its grid.
struct GroupLaunch {
    int path;  // 0: forward (TMA); 1: inverse (TMA ring); 2: inverse (row-wise loads)
    int nl, q1, grid;
    FusedArgs a;
    CUtensorMap m[3];
};

// Launch k of a plan in its direction (forward: group k; inverse: group
// ngroups - 1 - k).  Inter-launch LL buffers live in the plan's workspace
// layout at `ws`; the status word is `err`.
dwt2d_status build_group(const dwt2d_plan_s* p, bool fwd, int k, const void* src, long long src_pe,
                         void* dst, long long dst_pe, char* ws, int* err, int fwd_target,
                         int inv_target, GroupLaunch* out, int segq_fixed = 0,
                         bool uniform_segments = false, bool plan_only = false) {
    const int sch = base_scheme(p->scheme);
    const int elem_kind = elem_kind_of(p->dtype);
    const int rho = p->wavelet == DWT2D_CDF97 ? 2 : 1;
    void* bufs[2] = {ws + p->off_a, ws + p->off_b};
    const long long bpitch[2] = {p->pitch_a, p->pitch_b};
    const long long belems[2] = {(long long)(p->size_a / p->elem), (long long)(p->size_b / p->elem)};
    FusedArgs& a = out->a;
    memset(&a, 0, sizeof(a));
    a.err = err;
    if (fwd) {
        const int gi = k;
        const Group g = p->groups[gi];
        for (int i = 0; i < g.n; ++i) {
            a.lv[i].h = p->hs[g.first + i];
            a.lv[i].w = p->ws[g.first + i];
            level_scale(a.lv[i].h, a.lv[i].w, false, a.lv[i].s);
        }
        // input: the image, else the LL the previous launch wrote
        const void* in = gi == 0 ? src : bufs[(gi - 1) & 1];
        const long long in_pitch = gi == 0 ? src_pe : bpitch[(gi - 1) & 1];
        a.mallat = dst;
        a.mallat_pitch = dst_pe;
        a.mallat_elems = (long long)p->H * dst_pe;
        const bool last = gi == p->ngroups - 1;
        a.ll = last ? dst : bufs[gi & 1];
        a.ll_pitch = last ? dst_pe : bpitch[gi & 1];
        a.ll_elems = last ? a.mallat_elems : belems[gi & 1];
        const int hN = a.lv[g.n - 1].h;
        // an LL the next launch reads stays in L2 (evict-last stores) when it
        // takes at most a third of it: 2-4 % faster at 8192^2 float32 and
        // 16384^2 16-bit, slower once it crowds out the launch's own stream
        const long long ll_bytes = (long long)((hN + 1) / 2) * ((a.lv[g.n - 1].w + 1) / 2) * p->elem;
        a.ll_keep = !last && 3 * ll_bytes <= p->l2_bytes;
        const int rows = (hN + 1) / 2;
        // quadruple columns per lane: 4 for three fused levels; with
        // fwd_q1 == 0 (automatic), 4 for a float launch whose rows still give
        // long segments at the 4-column wave count (measured faster there:
        // less halo and shuffle work per pixel), else 2
        int q1 = g.n >= 3 ? 4 : (p->fwd_q1 == 4 ? 4 : 2);
        FusedArgs big4;
        int grid4 = 0;
        bool use4 = false;
        if (g.n <= 2 && p->fwd_q1 == 0 && segq_fixed <= 0 && elem_kind != 1 && p->fwd_warps_large4 > 0) {
            big4 = a;
            decompose(p, a.lv[0].w, rows, g.n, rho, 4, p->fwd_warps_large4, &big4, &grid4, kFwdWarps, 0,
                      resident_per_sm(true, g.n, 4, sch), uniform_segments ? 0 : p->fwd_short4,
                      p->fwd_seg_f);
            use4 = big4.segq >= p->large_segq;
            if (use4) q1 = 4;
        }
        dwt2d_status s = plan_only ? DWT2D_OK
                                   : make_map(&out->m[0], in, a.lv[0].h, a.lv[0].w, in_pitch, p->elem,
                                              elem_kind, 64 * q1, fwd_slot_rows(g.n, q1));
        if (s != DWT2D_OK) return s;
        if (use4) {
            a = big4;
            out->grid = grid4;
        } else {
            const int res = resident_per_sm(true, g.n, q1, sch);
            const int large = q1 == 4 ? p->fwd_warps_large4 : p->fwd_warps_large;
            const int sd = uniform_segments ? 0 : (q1 == 4 ? p->fwd_short4 : p->fwd_short);
            decompose(p, a.lv[0].w, rows, g.n, rho, q1, fwd_target, &a, &out->grid, kFwdWarps,
                      segq_fixed, res, 0, p->fwd_seg_f);
            if (segq_fixed <= 0 && large > fwd_target) {
                FusedArgs b = a;
                int grid_b = 0;
                decompose(p, a.lv[0].w, rows, g.n, rho, q1, large, &b, &grid_b, kFwdWarps, 0, res, sd,
                          p->fwd_seg_f);
                if (b.segq >= p->large_segq) {
                    a = b;
                    out->grid = grid_b;
                }
            }
        }
        out->path = 0;
        out->nl = g.n;
        out->q1 = q1;
        return DWT2D_OK;
    }
    // inverse: coarse group first; the coarsest LL sits at the top-left of the
    // Mallat array, later ones in the buffer the previous launch wrote
    const int gi = p->ngroups - 1 - k;
    const Group g = p->groups[gi];
    for (int i = 0; i < g.n; ++i) {
        a.lv[i].h = p->hs[g.first + i];
        a.lv[i].w = p->ws[g.first + i];
        level_scale(a.lv[i].h, a.lv[i].w, true, a.lv[i].s);
    }
    const void* ll_in = k == 0 ? src : bufs[(k - 1) & 1];
    const long long ll_pitch = k == 0 ? src_pe : bpitch[(k - 1) & 1];
    a.mallat = const_cast<void*>(src);
    a.mallat_pitch = src_pe;
    a.ll = const_cast<void*>(ll_in);
    a.ll_pitch = ll_pitch;
    const bool last = gi == 0;
    a.out = last ? dst : bufs[k & 1];
    a.out_pitch = last ? dst_pe : bpitch[k & 1];
    a.out_elems = last ? (long long)p->H * dst_pe : belems[k & 1];
    out->nl = g.n;
    if (g.n <= 2) {
        // TMA ring: boxes of the Mallat array and of the LL source.  2 columns
        // per lane unless 4 are asked for (measured: 4 is 7 % slower for the
        // 8192^2 finest launch, 5 % faster at 16384^2 float32)
        const int rows = (a.lv[0].h + 1) / 2;
        const int q1 = p->inv_q1 == 4 ? 4 : 2;
        const int al = 16 / p->elem;  // boxes start at a 16-byte boundary
        const int w1 = 32 * q1 + al, w2 = 16 * q1 + al;
        const int sr = inv_slot_rows(q1);  // level-1 box rows; level-2 boxes sr / 2
        dwt2d_status s = plan_only ? DWT2D_OK
                                   : make_map(&out->m[0], src, p->H, p->W, src_pe, p->elem, elem_kind, w1, sr);
        if (s == DWT2D_OK && !plan_only)
            s = make_map(&out->m[1], src, p->H, p->W, src_pe, p->elem, elem_kind, w2, sr / 2);
        const int llh = (a.lv[g.n - 1].h + 1) / 2, llw = (a.lv[g.n - 1].w + 1) / 2;
        const bool ll_is_src = k == 0;
        if (s == DWT2D_OK && !plan_only)
            s = make_map(&out->m[2], ll_in, ll_is_src ? p->H : llh, ll_is_src ? p->W : llw, ll_pitch,
                         p->elem, elem_kind, g.n == 1 ? w1 : w2, g.n == 1 ? sr : sr / 2);
        if (s != DWT2D_OK) return s;
        const int res = resident_per_sm(false, g.n, q1, sch);
        const int large = q1 == 4 ? p->inv_warps_large4 : p->inv_warps_large;
        const int sd = uniform_segments ? 0 : p->inv_short;
        // the inverse measured fastest with its segments top to bottom
        decompose(p, a.lv[0].w, rows, g.n, rho, q1, inv_target, &a, &out->grid, kInvTmaWarps,
                  segq_fixed, res, 0, p->inv_seg_f);
        if (segq_fixed <= 0 && large > inv_target) {
            FusedArgs b = a;
            int grid_b = 0;
            decompose(p, a.lv[0].w, rows, g.n, rho, q1, large, &b, &grid_b, kInvTmaWarps, 0, res, sd,
                      p->inv_seg_f);
            if (b.segq >= p->large_segq) {
                a = b;
                out->grid = grid_b;
            }
        }
        out->path = 1;
        out->q1 = q1;
    } else {
        decompose(p, a.lv[0].w, (a.lv[0].h + 1) / 2, g.n, rho, 4, inv_target, &a, &out->grid, 4, 0,
                  8, 0, p->inv_seg_f);
        out->path = 2;
        out->q1 = 4;
    }
    return DWT2D_OK;
}

dwt2d_status run_fused(const dwt2d_plan_s* p, bool fwd, const void* src, int64_t sp, void* dst,
                       int64_t dp, void* ws, cudaStream_t st) {
    const int elem_kind = elem_kind_of(p->dtype);
    const int sch = base_scheme(p->scheme);
    char* wsb = reinterpret_cast<char*>(ws);
    int* err = reinterpret_cast<int*>(wsb);
    for (int k = 0; k < p->ngroups; ++k) {
        GroupLaunch gl;
        dwt2d_status s = build_group(p, fwd, k, src, sp / p->elem, dst, dp / p->elem, wsb, err,
                                     p->fwd_warps_target, p->inv_warps_target, &gl);
        if (s != DWT2D_OK) return s;
        gl.a.pdl = p->pdl;
        cudaError_t e;
        mark(p, k, 0, st);
        if (gl.path == 0)
            e = launch_fwd_fused(elem_kind, sch, gl.nl, gl.q1, gl.m[0], gl.a, gl.grid, st);
        else if (gl.path == 1)
            e = launch_inv_tma(elem_kind, sch, gl.nl, gl.q1, gl.m[0], gl.m[1], gl.m[2], gl.a, gl.grid,
                               st);
        else
            e = launch_inv_fused(elem_kind, sch, gl.nl, gl.a, gl.grid, st);
        if (e != cudaSuccess) return DWT2D_ERR_CUDA;
        mark(p, k, 1, st);
    }
    return DWT2D_OK;
}

// Steps of one level in forward order: (kind, coefficient).
int step_list(const dwt2d_plan_s* p, int* kinds, float* coefs) {
    const int sch = base_scheme(p->scheme);
    int n = 0;
    if (p->wavelet == DWT2D_CDF97) {
        const float pu[2][2] = {{-1.586134342059924f, -0.052980118572961f},
                                {0.882911075530934f, 0.443506852043971f}};
        for (int k = 0; k < 2; ++k) {
            if (sch == SCH_SEP) {
                kinds[n] = P_TH; coefs[n++] = pu[k][0];
                kinds[n] = P_TV; coefs[n++] = pu[k][0];
                kinds[n] = P_SH; coefs[n++] = pu[k][1];
                kinds[n] = P_SV; coefs[n++] = pu[k][1];
            } else {
                kinds[n] = sch == SCH_RED ? P_TR : P_T; coefs[n++] = pu[k][0];
                kinds[n] = sch == SCH_RED ? P_SR : P_S; coefs[n++] = pu[k][1];
            }
        }
    } else {
        if (sch == SCH_SEP) {
            kinds[n] = P_TH; coefs[n++] = 0.f;
            kinds[n] = P_TV; coefs[n++] = 0.f;
            kinds[n] = P_SH; coefs[n++] = 0.f;
            kinds[n] = P_SV; coefs[n++] = 0.f;
        } else {
            kinds[n] = P_T; coefs[n++] = 0.f;
            kinds[n] = P_S; coefs[n++] = 0.f;
        }
    }
    return n;
}

dwt2d_status run_multipass(const dwt2d_plan_s* p, bool fwd, const void* src, int64_t sp, void* dst,
                           int64_t dp, void* ws, cudaStream_t st) {
    const int elem_kind = elem_kind_of(p->dtype);
    char* wsb = reinterpret_cast<char*>(ws);
    void* X[2] = {wsb + p->off_x, wsb + p->off_y};
    void* LLb[2] = {wsb + p->off_a, wsb + p->off_b};
    const long long llp[2] = {p->pitch_a, p->pitch_b};
    const long long src_pe = sp / p->elem, dst_pe = dp / p->elem;
    int kinds[8];
    float coefs[8];
    const int nsteps = step_list(p, kinds, coefs);

    auto interleaved = [](const void* ptr, long long pitch) {
        Layout L;
        L.p = ptr;
        L.pitch = pitch;
        L.ll = nullptr;
        L.ll_pitch = 0;
        L.kind = 0;
        return L;
    };
    auto mallat = [](const void* ptr, long long pitch, const void* ll, long long llpitch) {
        Layout L;
        L.p = ptr;
        L.pitch = pitch;
        L.ll = ll;
        L.ll_pitch = llpitch;
        L.kind = 1;
        return L;
    };

    if (fwd) {
        Layout in = interleaved(src, src_pe);
        for (int l = 0; l < p->levels; ++l) {
            const int h = p->hs[l], w = p->ws[l];
            const bool lastlev = l == p->levels - 1;
            const void* llout = lastlev ? dst : LLb[l & 1];
            const long long llout_p = lastlev ? dst_pe : llp[l & 1];
            for (int k = 0; k < nsteps; ++k) {
                PassArgs a;
                memset(&a, 0, sizeof(a));
                a.h = h;
                a.w = w;
                a.src = k == 0 ? in : interleaved(X[(k - 1) & 1], p->pitch_x);
                const bool lastk = k == nsteps - 1;
                a.dst = lastk ? mallat(dst, dst_pe, llout, llout_p) : interleaved(X[k & 1], p->pitch_x);
                a.coef = coefs[k];
                if (lastk && p->wavelet == DWT2D_CDF97) {
                    level_scale(h, w, false, a.s);
                    a.scale_out = 1;
                }
                mark(p, l * nsteps + k, 0, st);
                if (launch_pass(elem_kind, kinds[k], true, a, st) != cudaSuccess) return DWT2D_ERR_CUDA;
                mark(p, l * nsteps + k, 1, st);
            }
            in = interleaved(llout, llout_p);
        }
        return DWT2D_OK;
    }
    const void* llin = src;
    long long llin_p = src_pe;
    for (int l = p->levels - 1, j = 0; l >= 0; --l, ++j) {
        const int h = p->hs[l], w = p->ws[l];
        const bool lastlev = l == 0;
        void* out = lastlev ? dst : LLb[j & 1];
        const long long out_p = lastlev ? dst_pe : llp[j & 1];
        for (int k = 0; k < nsteps; ++k) {
            const int step = nsteps - 1 - k;  // undo in reverse order
            PassArgs a;
            memset(&a, 0, sizeof(a));
            a.h = h;
            a.w = w;
            a.src = k == 0 ? mallat(src, src_pe, llin, llin_p) : interleaved(X[(k - 1) & 1], p->pitch_x);
            a.dst = k == nsteps - 1 ? interleaved(out, out_p) : interleaved(X[k & 1], p->pitch_x);
            a.coef = -coefs[step];
            if (k == 0 && p->wavelet == DWT2D_CDF97) {
                level_scale(h, w, true, a.s);
                a.scale_in = 1;
            }
            mark(p, j * nsteps + k, 0, st);
            if (launch_pass(elem_kind, kinds[step], false, a, st) != cudaSuccess) return DWT2D_ERR_CUDA;
            mark(p, j * nsteps + k, 1, st);
        }
        llin = out;
        llin_p = out_p;
    }
    return DWT2D_OK;
}

dwt2d_status run_conv_fwd(const dwt2d_plan_s* p, const void* src, int64_t sp, void* dst, int64_t dp,
                          void* ws, cudaStream_t st) {
    const int elem_kind = elem_kind_of(p->dtype);
    char* wsb = reinterpret_cast<char*>(ws);
    void* LLb[2] = {wsb + p->off_a, wsb + p->off_b};
    const long long llp[2] = {p->pitch_a, p->pitch_b};
    const long long src_pe = sp / p->elem, dst_pe = dp / p->elem;
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    cdf97_taps(a.h0, a.g0);
    const void* in = src;
    long long in_p = src_pe;
    for (int l = 0; l < p->levels; ++l) {
        a.h = p->hs[l];
        a.w = p->ws[l];
        a.src = in;
        a.src_pitch = in_p;
        a.dst = dst;
        a.dst_pitch = dst_pe;
        const bool last = l == p->levels - 1;
        a.ll = last ? dst : LLb[l & 1];
        a.ll_pitch = last ? dst_pe : llp[l & 1];
        mark(p, l, 0, st);
        if (launch_conv_fwd(elem_kind, a, st) != cudaSuccess) return DWT2D_ERR_CUDA;
        mark(p, l, 1, st);
        in = a.ll;
        in_p = a.ll_pitch;
    }
    return DWT2D_OK;
}

}  // namespace

size_t dwt::plan_workspace_bytes(dwt2d_plan_t p) { return p ? p->ws_bytes : 0; }

extern "C" {

static dwt2d_status plan_create(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                                dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                                dwt2d_dtype dtype, size_t* workspace_bytes, const dwt2d_tuning* tuning,
                                const dwt2d_plan_options* opts);

dwt2d_status dwt2d_plan(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                        dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                        dwt2d_dtype dtype, size_t* workspace_bytes) {
    return plan_create(out, height, width, levels, wavelet, scheme, boundary, dtype, workspace_bytes,
                       nullptr, nullptr);
}

dwt2d_status dwt2d_plan_ex(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                           dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                           dwt2d_dtype dtype, const dwt2d_plan_options* options,
                           size_t* workspace_bytes) {
    return plan_create(out, height, width, levels, wavelet, scheme, boundary, dtype, workspace_bytes,
                       nullptr, options);
}

}  // extern "C"

// An option field: its value, or dflt when it is 0.
static int opt(int v, int dflt) { return v != 0 ? v : dflt; }

// Options in range (0 = default everywhere).
static bool options_ok(const dwt2d_plan_options& o) {
    auto in = [](int v, int lo, int hi) { return v == 0 || (v >= lo && v <= hi); };
    auto sw = [](int v) { return v == 0 || v == 1 || v == -1; };
    return in(o.fuse_first, 1, kMaxFused) && in(o.fuse_max, 1, kMaxFused) &&
           in(o.fwd_warps_per_sm, 1, 1 << 16) && in(o.inv_warps_per_sm, 1, 1 << 16) &&
           (o.fwd_warps_per_sm_large == -1 || in(o.fwd_warps_per_sm_large, 1, 1 << 16)) &&
           (o.inv_warps_per_sm_large == -1 || in(o.inv_warps_per_sm_large, 1, 1 << 16)) &&
           in(o.large_segment, 1, 1 << 16) && in(o.min_segment, 1, 1 << 16) &&
           in(o.fwd_seg_interleave, 1, 1 << 16) &&
           (o.inv_seg_interleave == -1 || in(o.inv_seg_interleave, 1, 1 << 16)) &&
           (o.fwd_cols_per_lane == 0 || o.fwd_cols_per_lane == 2 || o.fwd_cols_per_lane == 4) &&
           (o.inv_cols_per_lane == 0 || o.inv_cols_per_lane == 2 || o.inv_cols_per_lane == 4) &&
           sw(o.programmatic_launch) && in(o.host_bands, 1, kMaxHostBands) && sw(o.host_pipeline) &&
           (o.fwd_short_tail == -1 || in(o.fwd_short_tail, 2, 64)) &&
           (o.inv_short_tail == -1 || in(o.inv_short_tail, 2, 64));
}

static dwt2d_status plan_create(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                                dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                                dwt2d_dtype dtype, size_t* workspace_bytes, const dwt2d_tuning* tuning,
                                const dwt2d_plan_options* opts) {
    if (!out || !workspace_bytes) return DWT2D_ERR_INVALID;
    *out = nullptr;
    dwt2d_plan_options o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (!options_ok(o)) return DWT2D_ERR_INVALID;
    if (height < 1 || width < 1 || height > 65536 || width > 65536) return DWT2D_ERR_INVALID;
    if (levels < 1 || levels > 16) return DWT2D_ERR_INVALID;
    if (boundary != DWT2D_SYMMETRIC_WHOLE) return DWT2D_ERR_UNSUPPORTED;
    if (scheme < DWT2D_SEPARABLE || scheme > DWT2D_SEPARABLE_CONVOLUTION) return DWT2D_ERR_INVALID;
    if (convolution(scheme) && wavelet != DWT2D_CDF97) return DWT2D_ERR_UNSUPPORTED;
    const bool half = dtype == DWT2D_F16 || dtype == DWT2D_BF16;
    if (!((wavelet == DWT2D_CDF97 && (dtype == DWT2D_F32 || half)) ||
          (wavelet == DWT2D_LEGALL53 && dtype == DWT2D_I32)))
        return DWT2D_ERR_UNSUPPORTED;
    if (half && multipass(scheme)) return DWT2D_ERR_UNSUPPORTED;
    dwt2d_plan_s* p = (dwt2d_plan_s*)calloc(1, sizeof(dwt2d_plan_s));
    if (!p) return DWT2D_ERR_NOMEM;
    p->H = height;
    p->W = width;
    p->levels = levels;
    p->wavelet = wavelet;
    p->scheme = scheme;
    p->dtype = dtype;
    p->elem = half ? 2 : 4;
    int h = height, w = width;
    for (int l = 0; l < levels; ++l) {
        p->hs[l] = h;
        p->ws[l] = w;
        h = (h + 1) / 2;
        w = (w + 1) / 2;
    }
    // level groups: the first launch fuses fuse_first levels (default 2), later
    // launches up to fuse_max (default 2; 3 needs 4 columns per lane, which
    // measured slower) each; the shorter group comes last (5 levels: 2 + 2 + 1
    // measured faster than 2 + 1 + 2 both ways)
    int maxf = tuning && tuning->fuse_max > 0 ? tuning->fuse_max : opt(o.fuse_max, 2);
    if (maxf < 1) maxf = 1;
    if (maxf > kMaxFused) maxf = kMaxFused;
    if (half && maxf > 2) maxf = 2;  // 16-bit storage runs 2 columns per lane: up to 2 levels
    int first = tuning && tuning->fuse_first > 0 ? tuning->fuse_first
                                                 : opt(o.fuse_first, maxf < 2 ? maxf : 2);
    if (first < 1) first = 1;
    if (first > maxf) first = maxf;
    p->ngroups = 0;
    for (int l = 0; l < levels;) {
        const int cap = p->ngroups == 0 ? first : maxf;
        const int n = levels - l < cap ? levels - l : cap;
        p->groups[p->ngroups].first = l;
        p->groups[p->ngroups].n = n;
        ++p->ngroups;
        l += n;
    }
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    p->sm_count = sms;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2 = 0;
    cudaGetLastError();
    p->l2_bytes = l2;
    p->fwd_warps_target = sms * (tuning && tuning->warps_per_sm > 0 ? tuning->warps_per_sm
                                                                    : opt(o.fwd_warps_per_sm, 16));
    p->inv_warps_target = sms * (tuning && tuning->warps_per_sm > 0 ? tuning->warps_per_sm
                                                                    : opt(o.inv_warps_per_sm, 12));
    p->min_segq = tuning && tuning->min_segment > 0 ? tuning->min_segment : opt(o.min_segment, 2);
    // measured at 8192^2: the first forward launch is fastest at 48 warps
    // per SM (3 waves of 16) for CDF 9/7 and at 44 for LeGall 5/3 (its
    // shorter halo) with 2 columns per lane, at 24 (2 waves of 12) with 4;
    // the small later ones at one wave
    const int fwl = opt(o.fwd_warps_per_sm_large, wavelet == DWT2D_CDF97 ? 48 : 44);
    p->fwd_warps_large = (tuning && tuning->warps_per_sm > 0) || fwl < 0 ? 0 : sms * fwl;
    const int fwl4 = opt(o.fwd_warps_per_sm_large, 24);
    p->fwd_warps_large4 = (tuning && tuning->warps_per_sm > 0) || fwl4 < 0 ? 0 : sms * fwl4;
    p->large_segq = opt(o.large_segment, 16);
    // the finest inverse launch: 64 warps per SM (4 waves of 16)
    const int iwl = opt(o.inv_warps_per_sm_large, 64);
    p->inv_warps_large = (tuning && tuning->warps_per_sm > 0) || iwl < 0 ? 0 : sms * iwl;
    p->fwd_q1 = o.fwd_cols_per_lane;  // 0: automatic
    p->pdl = opt(o.programmatic_launch, 1) > 0;
    p->fwd_seg_f = o.fwd_seg_interleave;
    p->inv_seg_f = o.inv_seg_interleave < 0 ? 0 : opt(o.inv_seg_interleave, 1);
    // short last-wave segments: measured 3 % (forward, 3 at 2 columns per
    // lane, 4 at 4) and 2 % (inverse, 4) faster at 8192^2
    p->fwd_short = o.fwd_short_tail < 0 ? 0 : opt(o.fwd_short_tail, 3);
    p->fwd_short4 = o.fwd_short_tail < 0 ? 0 : opt(o.fwd_short_tail, 4);
    p->inv_short = o.inv_short_tail < 0 ? 0 : opt(o.inv_short_tail, 4);
    p->host_bands = opt(o.host_bands, 8);
    p->host_pipeline = opt(o.host_pipeline, 1) > 0;
    p->inv_q1 = o.inv_cols_per_lane == 4 ? 4 : 2;
    const int iwl4 = opt(o.inv_warps_per_sm_large, 24);
    p->inv_warps_large4 = (tuning && tuning->warps_per_sm > 0) || iwl4 < 0 ? 0 : sms * iwl4;

    // workspace: header | LL buffer A | LL buffer B | (multipass) X | Y
    size_t off = kHeader;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    long long pa = 1, pb = 1;
    size_t ba = 0, bb = 0;
    if (multipass(scheme) || convolution(scheme)) {
        // LLs alternate between A and B in both directions; size both for LL of level 1
        if (levels > 1) {
            const int lh = (p->hs[0] + 1) / 2, lw = (p->ws[0] + 1) / 2;
            pa = pb = round_pitch(lw, p->elem);
            ba = bb = (size_t)pa * lh * p->elem;
        }
    } else {
        for (int gi = 0; gi + 1 < p->ngroups; ++gi) {
            const Group g = p->groups[gi];
            const int last = g.first + g.n - 1;
            const int lh = (p->hs[last] + 1) / 2, lw = (p->ws[last] + 1) / 2;
            const long long pp = round_pitch(lw, p->elem);
            const size_t b = (size_t)pp * lh * p->elem;
            // forward writes group gi's LL to buffer gi & 1; the inverse uses the
            // same buffers for the LL it produces, which have the same sizes
            if ((gi & 1) == 0) { if (b > ba) { ba = b; pa = pp; } }
            else { if (b > bb) { bb = b; pb = pp; } }
        }
        // inverse order: launch k writes buffer k & 1; launch k produces the LL
        // that group (ngroups - 2 - k) produced in the forward direction
        for (int k = 0; k + 1 < p->ngroups; ++k) {
            const Group g = p->groups[p->ngroups - 2 - k];
            const int last = g.first + g.n - 1;
            const int lh = (p->hs[last] + 1) / 2, lw = (p->ws[last] + 1) / 2;
            const long long pp = round_pitch(lw, p->elem);
            const size_t b = (size_t)pp * lh * p->elem;
            if ((k & 1) == 0) { if (b > ba) { ba = b; pa = pp; } }
            else { if (b > bb) { bb = b; pb = pp; } }
        }
    }
    p->off_a = take(ba);
    p->pitch_a = pa;
    p->size_a = ba;
    p->off_b = take(bb);
    p->pitch_b = pb;
    p->size_b = bb;
    if (multipass(scheme)) {
        const long long px = round_pitch(width + (width & 1), p->elem);
        const size_t bx = (size_t)px * (height + (height & 1)) * p->elem;
        p->off_x = take(bx);
        p->off_y = take(bx);
        p->pitch_x = px;
    }
    p->ws_bytes = off;
    *workspace_bytes = off;
    *out = p;
    return DWT2D_OK;
}

extern "C" {

// 16-bit storage: stored value = value / scale for image and coefficients
// alike.  The transform is linear, so the coefficients of the stored image are
// the stored coefficients and the kernels never apply the scale; it is only
// checked here.
static bool scale_ok(const dwt2d_plan_s* p, float scale) {
    if (p->elem != 2) return true;
    return scale > 0.0f && scale < 3.0e38f;
}

}  // extern "C"

dwt2d_status dwt::check_transform_args(dwt2d_plan_t p, const void* src, int64_t sp, const void* dst,
                                       int64_t dp, const void* ws, float scale) {
    dwt2d_status s = check_buffers(p, src, sp, dst, dp, ws);
    if (s == DWT2D_OK && !scale_ok(p, scale)) s = DWT2D_ERR_INVALID;
    if (s == DWT2D_OK && src == dst) s = DWT2D_ERR_INVALID;
    return s;
}

extern "C" {

dwt2d_status dwt2d_forward(dwt2d_plan_t p, const void* d_src, int64_t sp, void* d_dst, int64_t dp,
                           void* d_ws, float scale, void* stream) {
    const dwt2d_status s = dwt::check_transform_args(p, d_src, sp, d_dst, dp, d_ws, scale);
    if (s != DWT2D_OK) return s;
    if (convolution(p->scheme)) return run_conv_fwd(p, d_src, sp, d_dst, dp, d_ws, as_stream(stream));
    return multipass(p->scheme) ? run_multipass(p, true, d_src, sp, d_dst, dp, d_ws, as_stream(stream))
                                : run_fused(p, true, d_src, sp, d_dst, dp, d_ws, as_stream(stream));
}

dwt2d_status dwt2d_inverse(dwt2d_plan_t p, const void* d_src, int64_t sp, void* d_dst, int64_t dp,
                           void* d_ws, float scale, void* stream) {
    const dwt2d_status s = dwt::check_transform_args(p, d_src, sp, d_dst, dp, d_ws, scale);
    if (s != DWT2D_OK) return s;
    return multipass(p->scheme) ? run_multipass(p, false, d_src, sp, d_dst, dp, d_ws, as_stream(stream))
                                : run_fused(p, false, d_src, sp, d_dst, dp, d_ws, as_stream(stream));
}


static bool host_resources(dwt2d_plan_s* p) {
    if (p->host_ready) return true;
    if (cudaStreamCreateWithFlags(&p->host_in, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamCreateWithFlags(&p->host_out, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (auto& e : p->host_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    p->host_ready = true;
    return true;
}

// Rows of the first group's input that row segment s reads (its TMA boxes),
// as the forward kernel computes them: [0, end).
static int seg_input_end(const dwt2d_plan_s* p, const FusedArgs& a, int nl, int q1, int rho, int s) {
    const int neN = (a.lv[nl - 1].h + 1) >> 1;
    const int R0 = s * a.segq, R1 = std::min(R0 + a.segq, neN);
    int f = R0, e = R1 - 1;
    for (int l = nl; l >= 1; --l) {
        f -= rho;
        e += rho;
        if (l > 1) {
            f *= 2;
            e = 2 * e + 1;
        }
    }
    const int rows = fwd_slot_rows(nl, q1), sr = rows / 2;  // image / quadruple rows per slot
    const int qstart = std::max(f, 0) & ~(sr - 1), qend = e + 1;
    const int nslots = (qend - qstart + sr - 1) / sr;
    return std::min(2 * qstart + rows * nslots, p->H);
}

// Host image -> host coefficients with the copies overlapped with the
// transform.  The image goes in as row bands on one stream; the first level
// group runs as one launch per run of row segments whose input rows have
// arrived; the detail bands those segments finish go out on a second stream
// while later bands still come in; the top-left region the later groups
// write goes out last.  The link carries about 200 GB/s each way and about
// 330 GB/s both ways at once, so overlapping the two directions is the gain.
static dwt2d_status run_host_fwd_pipelined(dwt2d_plan_s* p, const void* h_src, int64_t hsp,
                                           void* h_dst, int64_t hdp, void* d_in, void* d_out,
                                           int64_t dpitch, void* d_ws, cudaStream_t st) {
    const int64_t es = p->elem;
    const int64_t row = (int64_t)p->W * es;
    const char* hs = reinterpret_cast<const char*>(h_src);
    char* hd = reinterpret_cast<char*>(h_dst);
    char* din = reinterpret_cast<char*>(d_in);
    char* dout = reinterpret_cast<char*>(d_out);
    char* wsb = reinterpret_cast<char*>(d_ws);
    int* err = reinterpret_cast<int*>(wsb);
    const int B = p->host_bands;
    cudaEvent_t* ev = p->host_ev;  // [0] start, then per band: arrived, launched; end, out
    auto ev_in = [&](int c) { return ev[1 + c]; };
    auto ev_run = [&](int c) { return ev[1 + kMaxHostBands + c]; };
    cudaEvent_t ev_end = ev[1 + 2 * kMaxHostBands], ev_out = ev[2 + 2 * kMaxHostBands];
    auto copy2d = [](char* dst, int64_t dp, const char* src, int64_t sp, int64_t w, int64_t rows,
                     cudaMemcpyKind kind, cudaStream_t s) {
        if (rows <= 0 || w <= 0) return cudaSuccess;
        if (dp == w && sp == w) return cudaMemcpyAsync(dst, src, (size_t)(w * rows), kind, s);
        return cudaMemcpy2DAsync(dst, dp, src, sp, w, rows, kind, s);
    };
    // begin after the caller's earlier work on st (it may still use the buffers)
    if (cudaEventRecord(ev[0], st) != cudaSuccess || cudaStreamWaitEvent(p->host_in, ev[0], 0) ||
        cudaStreamWaitEvent(p->host_out, ev[0], 0))
        return DWT2D_ERR_CUDA;
    const int rb = (p->H + B - 1) / B;
    for (int c = 0; c < B; ++c) {
        const int r0 = std::min(c * rb, p->H), r1 = std::min(r0 + rb, p->H);
        if (copy2d(din + r0 * dpitch, dpitch, hs + r0 * hsp, hsp, row, r1 - r0, cudaMemcpyHostToDevice,
                   p->host_in) != cudaSuccess ||
            cudaEventRecord(ev_in(c), p->host_in) != cudaSuccess)
            return DWT2D_ERR_CUDA;
    }
    const int elem_kind = elem_kind_of(p->dtype);
    const int sch = base_scheme(p->scheme);
    const int rho = p->wavelet == DWT2D_CDF97 ? 2 : 1;
    GroupLaunch g0;
    dwt2d_status s = build_group(p, true, 0, d_in, dpitch / es, d_out, dpitch / es, wsb, err,
                                 p->fwd_warps_target, p->inv_warps_target, &g0, 0, true);
    if (s != DWT2D_OK) return s;
    const int nl0 = g0.nl;
    FusedArgs base = g0.a;
    base.seg_f = 1;
    int next = 0;  // first segment not launched yet
    for (int c = 0; c < B && next < base.nsegs; ++c) {
        const int avail = std::min((c + 1) * rb, p->H);
        int end = next;
        while (end < base.nsegs && (c == B - 1 || seg_input_end(p, base, nl0, g0.q1, rho, end) <= avail))
            ++end;
        if (end == next) continue;
        FusedArgs a = base;
        a.seg_lo = next;
        a.nsegs = a.nbig = end - next;
        const int grid = (a.nstrips * a.nsegs + kFwdWarps - 1) / kFwdWarps;
        if (cudaStreamWaitEvent(st, ev_in(c), 0) != cudaSuccess ||
            launch_fwd_fused(elem_kind, sch, nl0, g0.q1, g0.m[0], a, grid, st) != cudaSuccess ||
            cudaEventRecord(ev_run(c), st) != cudaSuccess ||
            cudaStreamWaitEvent(p->host_out, ev_run(c), 0) != cudaSuccess)
            return DWT2D_ERR_CUDA;
        // the detail bands of levels 1..nl0 in these segments' rows are final
        for (int l = 0; l < nl0; ++l) {
            const int h = a.lv[l].h, w = a.lv[l].w;
            const int ne_r = (h + 1) >> 1, no_r = h >> 1, ne_c = (w + 1) >> 1;
            const int sh = nl0 - 1 - l;
            const int neN = (a.lv[nl0 - 1].h + 1) >> 1;
            const int q0 = (next * a.segq) << sh;
            const int q1 = std::min(std::min(end * a.segq, neN) << sh, ne_r);
            if (q1 <= q0) continue;
            // HL: rows [q0, q1), columns [ne_c, w)
            if (copy2d(hd + q0 * hdp + ne_c * es, hdp, dout + q0 * dpitch + ne_c * es, dpitch,
                       (int64_t)(w - ne_c) * es, q1 - q0, cudaMemcpyDeviceToHost, p->host_out) != cudaSuccess)
                return DWT2D_ERR_CUDA;
            // LH and HH: rows [ne_r + q0, ne_r + min(q1, no_r)), columns [0, w)
            const int r1 = std::min(q1, no_r);
            if (r1 > q0 && copy2d(hd + (ne_r + q0) * hdp, hdp, dout + (ne_r + q0) * dpitch, dpitch,
                                  (int64_t)w * es, r1 - q0, cudaMemcpyDeviceToHost, p->host_out) != cudaSuccess)
                return DWT2D_ERR_CUDA;
        }
        next = end;
    }
    // every band has arrived before the call returns (the input buffer is free)
    if (cudaStreamWaitEvent(st, ev_in(B - 1), 0) != cudaSuccess) return DWT2D_ERR_CUDA;
    for (int k = 1; k < p->ngroups; ++k) {
        GroupLaunch gl;
        s = build_group(p, true, k, d_in, dpitch / es, d_out, dpitch / es, wsb, err, p->fwd_warps_target,
                        p->inv_warps_target, &gl);
        if (s != DWT2D_OK) return s;
        if (launch_fwd_fused(elem_kind, sch, gl.nl, gl.q1, gl.m[0], gl.a, gl.grid, st) != cudaSuccess)
            return DWT2D_ERR_CUDA;
    }
    // the region of the later levels (and the last LL): rows [0, ne_r), columns [0, ne_c)
    const int hl = base.lv[nl0 - 1].h, wl = base.lv[nl0 - 1].w;
    const int ner = (hl + 1) >> 1, nec = (wl + 1) >> 1;
    if (cudaEventRecord(ev_end, st) != cudaSuccess || cudaStreamWaitEvent(p->host_out, ev_end, 0) ||
        copy2d(hd, hdp, dout, dpitch, (int64_t)nec * es, ner, cudaMemcpyDeviceToHost, p->host_out) !=
            cudaSuccess ||
        cudaEventRecord(ev_out, p->host_out) != cudaSuccess || cudaStreamWaitEvent(st, ev_out, 0))
        return DWT2D_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? DWT2D_OK : DWT2D_ERR_CUDA;
}

// Host coefficients -> host image, the inverse counterpart: the top-left
// region of the coarse levels goes in first and the coarse groups run on it;
// the detail bands of the finest group's levels go in by row bands, that
// group runs as launches over the row segments whose inputs have arrived, and
// each launch's finished image rows go out while later bands come in.
static dwt2d_status run_host_inv_pipelined(dwt2d_plan_s* p, const void* h_src, int64_t hsp,
                                           void* h_dst, int64_t hdp, void* d_in, void* d_out,
                                           int64_t dpitch, void* d_ws, cudaStream_t st) {
    const int64_t es = p->elem;
    const char* hs = reinterpret_cast<const char*>(h_src);
    char* hd = reinterpret_cast<char*>(h_dst);
    char* din = reinterpret_cast<char*>(d_in);
    char* dout = reinterpret_cast<char*>(d_out);
    char* wsb = reinterpret_cast<char*>(d_ws);
    int* err = reinterpret_cast<int*>(wsb);
    const int B = p->host_bands;
    cudaEvent_t* ev = p->host_ev;  // [0] start, then per band: arrived, launched; end
    auto ev_in = [&](int c) { return ev[1 + c]; };
    auto ev_run = [&](int c) { return ev[1 + kMaxHostBands + c]; };
    cudaEvent_t ev_end = ev[1 + 2 * kMaxHostBands];
    auto copy2d = [](char* dst, int64_t dp, const char* src, int64_t sp, int64_t w, int64_t rows,
                     cudaMemcpyKind kind, cudaStream_t s) {
        if (rows <= 0 || w <= 0) return cudaSuccess;
        if (dp == w && sp == w) return cudaMemcpyAsync(dst, src, (size_t)(w * rows), kind, s);
        return cudaMemcpy2DAsync(dst, dp, src, sp, w, rows, kind, s);
    };
    auto in_rows = [&](int r0, int r1, int c0, int c1) {  // coefficient rectangle, host -> device
        return copy2d(din + r0 * dpitch + c0 * es, dpitch, hs + r0 * hsp + c0 * es, hsp,
                      (int64_t)(c1 - c0) * es, r1 - r0, cudaMemcpyHostToDevice, p->host_in);
    };
    if (cudaEventRecord(ev[0], st) != cudaSuccess || cudaStreamWaitEvent(p->host_in, ev[0], 0) ||
        cudaStreamWaitEvent(p->host_out, ev[0], 0))
        return DWT2D_ERR_CUDA;
    const int n0 = p->groups[0].n;  // levels of the finest group
    const int hN = p->hs[n0 - 1], wN = p->ws[n0 - 1];
    // the coarse region: levels > n0 and the last LL
    if (in_rows(0, (hN + 1) / 2, 0, (wN + 1) / 2) != cudaSuccess) return DWT2D_ERR_CUDA;
    // the finest group's detail bands by row bands of level-1 quadruple rows
    const int ne_r1 = (p->hs[0] + 1) / 2;
    const int unit = 1 << (n0 - 1);
    const int rb = ((ne_r1 + B - 1) / B + unit - 1) / unit * unit;
    for (int c = 0; c < B; ++c) {
        for (int l = 0; l < n0; ++l) {
            const int h = p->hs[l], w = p->ws[l];
            const int ne_r = (h + 1) >> 1, no_r = h >> 1, ne_c = (w + 1) >> 1;
            const int q0 = std::min((c * rb) >> l, ne_r);
            const int q1 = c == B - 1 ? ne_r : std::min(((c + 1) * rb) >> l, ne_r);
            if (q1 <= q0) continue;
            if (in_rows(q0, q1, ne_c, w) != cudaSuccess) return DWT2D_ERR_CUDA;  // HL
            const int r1 = std::min(q1, no_r);
            if (r1 > q0 && in_rows(ne_r + q0, ne_r + r1, 0, w) != cudaSuccess) return DWT2D_ERR_CUDA;
        }
        if (cudaEventRecord(ev_in(c), p->host_in) != cudaSuccess) return DWT2D_ERR_CUDA;
    }
    const int elem_kind = elem_kind_of(p->dtype);
    const int sch = base_scheme(p->scheme);
    const int G = p->ngroups;
    // coarse groups: their input (the coarse region) went in first
    if (G > 1 && cudaStreamWaitEvent(st, ev_in(0), 0) != cudaSuccess) return DWT2D_ERR_CUDA;
    for (int k = 0; k + 1 < G; ++k) {
        GroupLaunch gl;
        dwt2d_status s = build_group(p, false, k, d_in, dpitch / es, d_out, dpitch / es, wsb, err,
                                     p->fwd_warps_target, p->inv_warps_target, &gl);
        if (s != DWT2D_OK) return s;
        const cudaError_t e = gl.path == 1 ? launch_inv_tma(elem_kind, sch, gl.nl, gl.q1, gl.m[0], gl.m[1],
                                                            gl.m[2], gl.a, gl.grid, st)
                                           : launch_inv_fused(elem_kind, sch, gl.nl, gl.a, gl.grid, st);
        if (e != cudaSuccess) return DWT2D_ERR_CUDA;
    }
    GroupLaunch gf;
    dwt2d_status s = build_group(p, false, G - 1, d_in, dpitch / es, d_out, dpitch / es, wsb, err,
                                 p->fwd_warps_target, p->inv_warps_target, &gf, 0, true);
    if (s != DWT2D_OK) return s;
    if (gf.path != 1) return DWT2D_ERR_INVALID;
    FusedArgs base = gf.a;
    base.seg_f = 1;
    const int lag = p->wavelet == DWT2D_CDF97 ? 2 : 1;
    const int ne_r2 = n0 == 2 ? (p->hs[1] + 1) / 2 : 0;
    const int sr = inv_slot_rows(gf.q1), spro = n0 == 2 ? 2 * lag / (sr / 2) : 0;
    auto ready = [&](int seg, int c) {  // rows segment `seg` reads are all in after band c
        if (c == B - 1) return true;
        const int A0 = seg * base.segq, A1 = std::min(A0 + base.segq, ne_r1);
        const int qstart = std::max(A0 - lag, 0) & ~(sr - 1);
        const int nmain = (A1 + lag - qstart + sr - 1) / sr;
        const int end1 = std::min(qstart + sr * nmain, ne_r1);
        if (end1 > std::min((c + 1) * rb, ne_r1)) return false;
        if (n0 == 2) {
            const int qlast = qstart - sr * spro + sr * (nmain + spro - 1);
            const int end2 = std::min(qlast / 2 + lag + sr / 2, ne_r2);
            if (end2 > std::min(((c + 1) * rb) >> 1, ne_r2)) return false;
        }
        return true;
    };
    int next = 0;
    for (int c = 0; c < B && next < base.nsegs; ++c) {
        int end = next;
        while (end < base.nsegs && ready(end, c)) ++end;
        if (end == next) continue;
        FusedArgs a = base;
        a.seg_lo = next;
        a.nsegs = a.nbig = end - next;
        const int grid = (a.nstrips * a.nsegs + kInvTmaWarps - 1) / kInvTmaWarps;
        if (cudaStreamWaitEvent(st, ev_in(c), 0) != cudaSuccess ||
            launch_inv_tma(elem_kind, sch, gf.nl, gf.q1, gf.m[0], gf.m[1], gf.m[2], a, grid, st) !=
                cudaSuccess ||
            cudaEventRecord(ev_run(c), st) != cudaSuccess ||
            cudaStreamWaitEvent(p->host_out, ev_run(c), 0) != cudaSuccess)
            return DWT2D_ERR_CUDA;
        const int y0 = std::min(2 * next * base.segq, p->H);
        const int y1 = std::min(2 * std::min(end * base.segq, ne_r1), p->H);
        if (copy2d(hd + y0 * hdp, hdp, dout + y0 * dpitch, dpitch, (int64_t)p->W * es, y1 - y0,
                   cudaMemcpyDeviceToHost, p->host_out) != cudaSuccess)
            return DWT2D_ERR_CUDA;
        next = end;
    }
    if (cudaStreamWaitEvent(st, ev_in(B - 1), 0) != cudaSuccess ||
        cudaEventRecord(ev_end, p->host_out) != cudaSuccess || cudaStreamWaitEvent(st, ev_end, 0))
        return DWT2D_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? DWT2D_OK : DWT2D_ERR_CUDA;
}

static dwt2d_status run_host(dwt2d_plan_t p, bool fwd, const void* h_src, int64_t hsp, void* h_dst,
                             int64_t hdp, void* d_in, void* d_out, int64_t dpitch, void* d_ws,
                             float scale, void* stream) {
    if (!p || !h_src || !h_dst) return DWT2D_ERR_INVALID;
    const int64_t row = (int64_t)p->W * p->elem;
    if (hsp < row || hdp < row) return DWT2D_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    if (fwd && p->H >= 1024 && !multipass(p->scheme) && !convolution(p->scheme) &&
        p->host_pipeline && check_buffers(p, d_in, dpitch, d_out, dpitch, d_ws) == DWT2D_OK &&
        p->groups[0].n <= 2 && scale_ok(p, scale) && host_resources(p))
        return run_host_fwd_pipelined(p, h_src, hsp, h_dst, hdp, d_in, d_out, dpitch, d_ws, st);
    if (!fwd && p->H >= 1024 && !multipass(p->scheme) && p->host_pipeline &&
        check_buffers(p, d_in, dpitch, d_out, dpitch, d_ws) == DWT2D_OK && p->groups[0].n <= 2 &&
        scale_ok(p, scale) && host_resources(p))
        return run_host_inv_pipelined(p, h_src, hsp, h_dst, hdp, d_in, d_out, dpitch, d_ws, st);
    // one linear copy when both sides are unpadded (faster than a 2-D copy)
    auto copy = [&](void* dst, int64_t dp, const void* src, int64_t sp, cudaMemcpyKind kind) {
        if (dp == row && sp == row)
            return cudaMemcpyAsync(dst, src, (size_t)row * p->H, kind, st);
        return cudaMemcpy2DAsync(dst, dp, src, sp, row, p->H, kind, st);
    };
    if (copy(d_in, dpitch, h_src, hsp, cudaMemcpyHostToDevice) != cudaSuccess) return DWT2D_ERR_CUDA;
    dwt2d_status s = fwd ? dwt2d_forward(p, d_in, dpitch, d_out, dpitch, d_ws, scale, stream)
                         : dwt2d_inverse(p, d_in, dpitch, d_out, dpitch, d_ws, scale, stream);
    if (s != DWT2D_OK) return s;
    if (copy(h_dst, hdp, d_out, dpitch, cudaMemcpyDeviceToHost) != cudaSuccess) return DWT2D_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? DWT2D_OK : DWT2D_ERR_CUDA;
}

dwt2d_status dwt2d_forward_host(dwt2d_plan_t p, const void* h_src, int64_t hsp, void* h_dst,
                                int64_t hdp, void* d_in, void* d_out, int64_t dpitch, void* d_ws,
                                float scale, void* stream) {
    return run_host(p, true, h_src, hsp, h_dst, hdp, d_in, d_out, dpitch, d_ws, scale, stream);
}

dwt2d_status dwt2d_inverse_host(dwt2d_plan_t p, const void* h_src, int64_t hsp, void* h_dst,
                                int64_t hdp, void* d_in, void* d_out, int64_t dpitch, void* d_ws,
                                float scale, void* stream) {
    return run_host(p, false, h_src, hsp, h_dst, hdp, d_in, d_out, dpitch, d_ws, scale, stream);
}

dwt2d_status dwt2d_workspace_init(void* d_ws, void* stream) {
    if (!d_ws) return DWT2D_ERR_INVALID;
    if (!aligned16(d_ws)) return DWT2D_ERR_ALIGN;
    // the whole header (its first word is the status word)
    return cudaMemsetAsync(d_ws, 0, kHeader, as_stream(stream)) == cudaSuccess ? DWT2D_OK
                                                                               : DWT2D_ERR_CUDA;
}

dwt2d_status dwt2d_workspace_status(void* d_ws, void* stream) {
    if (!d_ws) return DWT2D_ERR_INVALID;
    int h = 0;
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(&h, d_ws, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DWT2D_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DWT2D_ERR_CUDA;
    if (h != 0) {
        // clear the header for the next call
        if (cudaMemsetAsync(d_ws, 0, kHeader, st) != cudaSuccess) return DWT2D_ERR_CUDA;
        return (dwt2d_status)h;
    }
    return DWT2D_OK;
}

dwt2d_status dwt2d_plan_info(dwt2d_plan_t p, int32_t* launches, int32_t* fused, int32_t* n_groups) {
    if (!p) return DWT2D_ERR_INVALID;
    if (convolution(p->scheme)) {
        if (launches) *launches = p->levels;
        if (n_groups) *n_groups = p->levels;
        if (fused)
            for (int l = 0; l < p->levels; ++l) fused[l] = 1;
        return DWT2D_OK;
    }
    if (multipass(p->scheme)) {
        int kinds[8];
        float coefs[8];
        const int n = step_list(p, kinds, coefs);
        if (launches) *launches = n * p->levels;
        if (n_groups) *n_groups = p->levels;
        if (fused)
            for (int l = 0; l < p->levels; ++l) fused[l] = 1;
        return DWT2D_OK;
    }
    if (launches) *launches = p->ngroups;
    if (n_groups) *n_groups = p->ngroups;
    if (fused)
        for (int g = 0; g < p->ngroups; ++g) fused[g] = p->groups[g].n;
    return DWT2D_OK;
}

dwt2d_status dwt2d_plan_launch_info(dwt2d_plan_t p, int32_t inverse, int32_t i, int32_t* fused,
                                     int32_t* cols_per_lane, int32_t* warps) {
    if (!p || i < 0 || (inverse != 0 && inverse != 1)) return DWT2D_ERR_INVALID;
    if (multipass(p->scheme) || (convolution(p->scheme) && !inverse)) return DWT2D_ERR_UNSUPPORTED;
    if (i >= p->ngroups) return DWT2D_ERR_INVALID;
    GroupLaunch gl;
    const dwt2d_status s = build_group(p, !inverse, i, nullptr, 1, nullptr, 1, nullptr, nullptr,
                                       p->fwd_warps_target, p->inv_warps_target, &gl, 0, false, true);
    if (s != DWT2D_OK) return s;
    if (fused) *fused = gl.nl;
    if (cols_per_lane) *cols_per_lane = gl.q1;
    if (warps) *warps = gl.a.nstrips * gl.a.nsegs;
    return DWT2D_OK;
}

dwt2d_status dwt2d_plan_set_launch_events(dwt2d_plan_t p, void** events, int32_t count) {
    if (!p || count < 0) return DWT2D_ERR_INVALID;
    p->events = events ? reinterpret_cast<cudaEvent_t*>(events) : nullptr;
    p->nevents = events ? count : 0;
    return DWT2D_OK;
}

void dwt2d_plan_destroy(dwt2d_plan_t p) {
    if (p && p->host_ready) {
        cudaStreamDestroy(p->host_in);
        cudaStreamDestroy(p->host_out);
        for (auto& e : p->host_ev) cudaEventDestroy(e);
    }
    free(p);
}

dwt2d_status dwt2d_batch_create(dwt2d_batch_t* out, const dwt2d_batch_item* items, int32_t n,
                                dwt2d_scheme scheme, const dwt2d_tuning* tuning,
                                size_t* workspace_bytes) {
    if (!out || !workspace_bytes || (n > 0 && !items) || n < 0) return DWT2D_ERR_INVALID;
    *out = nullptr;
    if (scheme != DWT2D_SEPARABLE && scheme != DWT2D_NONSEP && scheme != DWT2D_NONSEP_REDUCED)
        return DWT2D_ERR_UNSUPPORTED;
    dwt2d_tuning tun = {0, 0, 0, 0};
    if (tuning) tun = *tuning;
    // the batched kernels run 2 or 4 quadruple columns per lane and fuse up to 2 levels
    if (tun.fuse_max > 2 || tun.fuse_first > 2) return DWT2D_ERR_UNSUPPORTED;
    if (tun.cols_per_lane != 0 && tun.cols_per_lane != 2 && tun.cols_per_lane != 4)
        return DWT2D_ERR_INVALID;
    const int q1 = tun.cols_per_lane == 4 ? 4 : 2;
    if (tun.fuse_max <= 0) tun.fuse_max = 2;
    const int wps = tun.warps_per_sm;
    tun.warps_per_sm = 0;  // the per-image share is set below
    dwt2d_batch_s* b = new (std::nothrow) dwt2d_batch_s();
    if (!b) return DWT2D_ERR_NOMEM;
    b->scheme = scheme;
    b->pdl = tun.programmatic_launch > 0;  // default off: measured neutral to 1 % slower for batches
    b->queue = tun.persistent > 0;
    b->q1 = q1;
    b->items.assign(items, items + n);
    size_t off = kHeader;
    b->table_off = off;
    for (int i = 0; i < n; ++i) {
        const dwt2d_batch_item& it = items[i];
        dwt2d_plan_t p = nullptr;
        size_t wsb = 0;
        dwt2d_status s = plan_create(&p, it.height, it.width, it.levels, it.wavelet, scheme,
                                     DWT2D_SYMMETRIC_WHOLE, it.dtype, &wsb, &tun, nullptr);
        if (s == DWT2D_OK && (it.inverse != 0 && it.inverse != 1)) s = DWT2D_ERR_INVALID;
        if (s == DWT2D_OK) s = check_buffers(p, it.d_src, it.src_pitch_bytes, it.d_dst,
                                             it.dst_pitch_bytes, it.d_src);
        if (s == DWT2D_OK && it.d_src == it.d_dst) s = DWT2D_ERR_INVALID;
        if (s != DWT2D_OK) {
            free(p);
            delete b;
            return s;
        }
        p->fwd_q1 = p->inv_q1 = q1;
        b->plans.push_back(p);
    }
    // Launch list: phase k, then direction, storage type, fusion depth.  One
    // launch spreads its rows evenly: every warp streams the same number of
    // rows (segq), chosen so that the launch has about warps_per_sm warps per
    // SM (default 48: four waves of the 12 resident, which evens out images
    // whose border strips run the slower edge path).
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    int max_groups = 0;
    for (auto* p : b->plans) max_groups = std::max(max_groups, p->ngroups);
    b->warps = 0;
    for (int k = 0; k < max_groups; ++k) {
        for (int fwd = 1; fwd >= 0; --fwd) {
            for (int ek = 0; ek < 4; ++ek) {
                for (int nl = 1; nl <= 2; ++nl) {
                    dwt2d_batch_s::Launch L = {fwd, ek, nl, (int)b->refs.size(), 0, 0};
                    struct Cand { int i, w0, rows, rho, nstrips; };
                    std::vector<Cand> cand;
                    long long work = 0;  // strips x rows over the launch
                    int min_segq = 1;
                    for (int i = 0; i < n; ++i) {
                        const dwt2d_plan_s* p = b->plans[i];
                        if ((items[i].inverse == 0) != (fwd == 1) || elem_kind_of(p->dtype) != ek ||
                            k >= p->ngroups)
                            continue;
                        const int gi = fwd ? k : p->ngroups - 1 - k;
                        const Group g = p->groups[gi];
                        if (g.n != nl) continue;
                        Cand c;
                        c.i = i;
                        c.rho = p->wavelet == DWT2D_CDF97 ? 2 : 1;
                        c.w0 = p->ws[g.first];
                        c.rows = fwd ? (p->hs[g.first + g.n - 1] + 1) / 2 : (p->hs[g.first] + 1) / 2;
                        FusedArgs a;
                        memset(&a, 0, sizeof(a));
                        int grid = 0;
                        decompose(p, c.w0, c.rows, nl, c.rho, q1, 1, &a, &grid, 4);
                        c.nstrips = a.nstrips;
                        work += (long long)c.nstrips * c.rows;
                        min_segq = std::max(min_segq, p->min_segq);
                        cand.push_back(c);
                    }
                    if (cand.empty()) continue;
                    const long long target = (long long)sms * (wps > 0 ? wps : 48);
                    const int segq = (int)std::max<long long>(min_segq, (work + target - 1) / target);
                    long long warps = 0;
                    for (const Cand& c : cand) {
                        const dwt2d_plan_s* p = b->plans[c.i];
                        FusedArgs a;
                        memset(&a, 0, sizeof(a));
                        int grid = 0;
                        decompose(p, c.w0, c.rows, nl, c.rho, q1, 1, &a, &grid, 4, segq);
                        b->refs.push_back({c.i, k});
                        b->segq.push_back(segq);
                        warps += (long long)a.nstrips * a.nsegs;
                        ++L.count;
                    }
                    if (warps > (1LL << 30)) {
                        delete b;
                        return DWT2D_ERR_INVALID;
                    }
                    const int per_cta = fwd ? kFwdWarps : kInvTmaWarps;
                    L.grid = (int)((warps + per_cta - 1) / per_cta);
                    b->warps += warps;
                    b->launches.push_back(L);
                }
            }
        }
    }
    off += (b->refs.size() * sizeof(BatchEntry) + 255) / 256 * 256;
    b->max_groups = max_groups;
    b->sms = sms;
    // queues: the launches of one (direction, storage type), in launch order
    // (level group by level group)
    for (int fwd = 1; fwd >= 0; --fwd) {
        for (int ek = 0; ek < 4; ++ek) {
            dwt2d_batch_s::Queue q = {fwd, ek, (int)b->qorder.size(), 0, 0};
            for (const auto& L : b->launches) {
                if (L.fwd != fwd || L.elem_kind != ek) continue;
                for (int j = L.first; j < L.first + L.count; ++j) b->qorder.push_back(j);
            }
            q.count = (int)b->qorder.size() - q.first;
            if (q.count > 0) b->queues.push_back(q);
        }
    }
    b->qtable_off = off;
    off += (b->qorder.size() * sizeof(BatchEntry) + 255) / 256 * 256;
    b->counters_off = off;
    b->counters_bytes = (size_t)(8 + n * std::max(max_groups, 1)) * sizeof(int);
    off += (b->counters_bytes + 255) / 256 * 256;
    for (int i = 0; i < n; ++i) {
        b->region.push_back(off);
        off += (b->plans[i]->ws_bytes + 255) / 256 * 256;
    }
    b->ws_bytes = off;
    *workspace_bytes = off;
    *out = b;
    return DWT2D_OK;
}

static dwt2d_status batch_upload(dwt2d_batch_t b, void* d_ws, void* h_staging, size_t staging_bytes,
                                 void* stream);

dwt2d_status dwt2d_batch_upload(dwt2d_batch_t b, void* d_ws, void* stream) {
    return batch_upload(b, d_ws, nullptr, 0, stream);
}

dwt2d_status dwt2d_batch_staging_bytes(dwt2d_batch_t b, size_t* bytes) {
    if (!b || !bytes) return DWT2D_ERR_INVALID;
    *bytes = (b->refs.size() + b->qorder.size()) * sizeof(BatchEntry);
    return DWT2D_OK;
}

dwt2d_status dwt2d_batch_upload_staged(dwt2d_batch_t b, void* d_ws, void* h_staging, size_t bytes,
                                       void* stream) {
    if (!b || !h_staging) return DWT2D_ERR_INVALID;
    size_t need = 0;
    dwt2d_batch_staging_bytes(b, &need);
    if (bytes < need || ((uintptr_t)h_staging & 15u)) return DWT2D_ERR_INVALID;
    return batch_upload(b, d_ws, h_staging, bytes, stream);
}

static dwt2d_status batch_upload(dwt2d_batch_t b, void* d_ws, void* h_staging, size_t staging_bytes,
                                 void* stream) {
    (void)staging_bytes;
    if (!b || !d_ws) return DWT2D_ERR_INVALID;
    if (!aligned16(d_ws) || ((uintptr_t)d_ws & 255u)) return DWT2D_ERR_ALIGN;
    cudaStream_t st = as_stream(stream);
    char* wsb = reinterpret_cast<char*>(d_ws);
    int* err = reinterpret_cast<int*>(wsb);
    b->table.assign(b->refs.size(), BatchEntry{});
    for (const auto& L : b->launches) {
        int first_warp = 0;
        for (int j = L.first; j < L.first + L.count; ++j) {
            const int i = b->refs[j].first, k = b->refs[j].second;
            const dwt2d_batch_item& it = b->items[i];
            const dwt2d_plan_s* p = b->plans[i];
            GroupLaunch gl;
            dwt2d_status s = build_group(p, it.inverse == 0, k, it.d_src, it.src_pitch_bytes / p->elem,
                                         it.d_dst, it.dst_pitch_bytes / p->elem, wsb + b->region[i],
                                         err, 1, 1, &gl, b->segq[j]);
            if (s != DWT2D_OK) return s;
            if (gl.path == 2 || gl.nl != L.nl || gl.q1 != b->q1) return DWT2D_ERR_INVALID;  // planned otherwise
            BatchEntry& e = b->table[j];
            memcpy(e.m, gl.m, sizeof(e.m));
            e.args = gl.a;
            // the images of a batch share the L2: no evict-last LL (measured 1 % slower)
            e.args.ll_keep = 0;
            e.first_warp = first_warp;
            first_warp += gl.a.nstrips * gl.a.nsegs;
        }
        // kernel attributes once, outside any capture
        const int sch = base_scheme(b->scheme);
        const cudaError_t e =
            L.fwd ? launch_fwd_batched(L.elem_kind, sch, L.nl, b->q1, nullptr, 0, 0, st, false)
                  : launch_inv_batched(L.elem_kind, sch, L.nl, b->q1, nullptr, 0, 0, st, false);
        if (e != cudaSuccess) return DWT2D_ERR_CUDA;
    }
    // the tables go up from the caller's pinned staging buffer when given one
    // (a copy from pageable memory may wait for the stream to drain)
    auto upload = [&](size_t dev_off, const std::vector<BatchEntry>& v, size_t stage_off) {
        if (v.empty()) return cudaSuccess;
        const size_t bytes = v.size() * sizeof(BatchEntry);
        const void* srcp = v.data();
        if (h_staging) {
            memcpy(static_cast<char*>(h_staging) + stage_off, v.data(), bytes);
            srcp = static_cast<char*>(h_staging) + stage_off;
        }
        return cudaMemcpyAsync(wsb + dev_off, srcp, bytes, cudaMemcpyHostToDevice, st);
    };
    if (upload(b->table_off, b->table, 0) != cudaSuccess) return DWT2D_ERR_CUDA;
    // queue mode: the same entries queue by queue, numbered within their
    // queue, with their done counters and the group each depends on
    b->qtable.clear();
    std::vector<long long> items_of((size_t)b->items.size() * std::max(b->max_groups, 1), 0);
    for (size_t j = 0; j < b->table.size(); ++j) {
        const int i = b->refs[j].first, k = b->refs[j].second;
        items_of[(size_t)i * b->max_groups + k] =
            (long long)b->table[j].args.nstrips * b->table[j].args.nsegs;
    }
    for (auto& q : b->queues) {
        long long first = 0;
        for (int t = q.first; t < q.first + q.count; ++t) {
            const int j = b->qorder[t];
            const int i = b->refs[j].first, k = b->refs[j].second;
            BatchEntry e = b->table[j];
            e.first_warp = (int)first;
            e.self = i * b->max_groups + k;
            e.dep = k > 0 ? i * b->max_groups + (k - 1) : -1;
            e.dep_items = k > 0 ? (int)items_of[(size_t)i * b->max_groups + (k - 1)] : 0;
            for (const auto& L : b->launches)
                if (j >= L.first && j < L.first + L.count) e.nl = L.nl;
            first += (long long)e.args.nstrips * e.args.nsegs;
            b->qtable.push_back(e);
        }
        q.items = first;
        if (first > (1LL << 30)) return DWT2D_ERR_INVALID;
        const int sch = base_scheme(b->scheme);
        const cudaError_t e = q.fwd ? launch_fwd_queue(q.elem_kind, sch, b->q1, nullptr, 0, 0, nullptr,
                                                       nullptr, nullptr, 0, st)
                                    : launch_inv_queue(q.elem_kind, sch, b->q1, nullptr, 0, 0, nullptr,
                                                       nullptr, nullptr, 0, st);
        if (e != cudaSuccess) return DWT2D_ERR_CUDA;
    }
    if (upload(b->qtable_off, b->qtable, b->table.size() * sizeof(BatchEntry)) != cudaSuccess)
        return DWT2D_ERR_CUDA;
    if (cudaMemsetAsync(d_ws, 0, sizeof(int), st) != cudaSuccess) return DWT2D_ERR_CUDA;
    return DWT2D_OK;
}

dwt2d_status dwt2d_batch_launch(dwt2d_batch_t b, void* d_ws, void* stream) {
    if (!b || !d_ws) return DWT2D_ERR_INVALID;
    if ((uintptr_t)d_ws & 255u) return DWT2D_ERR_ALIGN;
    if (b->table.size() != b->refs.size()) return DWT2D_ERR_INVALID;  // not uploaded
    cudaStream_t st = as_stream(stream);
    const BatchEntry* table =
        reinterpret_cast<const BatchEntry*>(reinterpret_cast<char*>(d_ws) + b->table_off);
    const int sch = base_scheme(b->scheme);
    if (b->queue) {
        char* wsb = reinterpret_cast<char*>(d_ws);
        int* err = reinterpret_cast<int*>(wsb);
        int* heads = reinterpret_cast<int*>(wsb + b->counters_off);
        int* done = heads + 8;
        // counters start at zero on every launch (a memset node in a captured graph)
        if (cudaMemsetAsync(heads, 0, b->counters_bytes, st) != cudaSuccess) return DWT2D_ERR_CUDA;
        const BatchEntry* qt = reinterpret_cast<const BatchEntry*>(wsb + b->qtable_off);
        for (size_t qi = 0; qi < b->queues.size(); ++qi) {
            const auto& q = b->queues[qi];
            // one wave: the warps the queue kernel's register budget keeps resident
            const long long resident =
                (long long)b->sms * (q.fwd ? fwd_queue_resident(b->q1) : inv_queue_resident(b->q1));
            const int grid = (int)std::min<long long>(q.items, resident);
            const cudaError_t e =
                q.fwd ? launch_fwd_queue(q.elem_kind, sch, b->q1, qt + q.first, q.count, (int)q.items,
                                         heads + qi, done, err, grid, st)
                      : launch_inv_queue(q.elem_kind, sch, b->q1, qt + q.first, q.count, (int)q.items,
                                         heads + qi, done, err, grid, st);
            if (e != cudaSuccess) return DWT2D_ERR_CUDA;
        }
        return DWT2D_OK;
    }
    for (const auto& L : b->launches) {
        const cudaError_t e =
            L.fwd ? launch_fwd_batched(L.elem_kind, sch, L.nl, b->q1, table + L.first, L.count, L.grid,
                                       st, b->pdl)
                  : launch_inv_batched(L.elem_kind, sch, L.nl, b->q1, table + L.first, L.count, L.grid,
                                       st, b->pdl);
        if (e != cudaSuccess) return DWT2D_ERR_CUDA;
    }
    return DWT2D_OK;
}

dwt2d_status dwt2d_batch_info(dwt2d_batch_t b, int32_t* launches, int64_t* warps) {
    if (!b) return DWT2D_ERR_INVALID;
    if (launches) *launches = (int32_t)(b->queue ? b->queues.size() : b->launches.size());
    if (warps) *warps = b->warps;
    return DWT2D_OK;
}

void dwt2d_batch_destroy(dwt2d_batch_t b) { delete b; }

const char* dwt2d_status_string(dwt2d_status s) {
    switch (s) {
        case DWT2D_OK: return "ok";
        case DWT2D_ERR_INVALID: return "invalid argument";
        case DWT2D_ERR_UNSUPPORTED: return "unsupported wavelet/dtype/scheme";
        case DWT2D_ERR_ALIGN: return "pointer or pitch not 16-byte aligned";
        case DWT2D_ERR_NOMEM: return "host allocation failed";
        case DWT2D_ERR_CUDA: return "CUDA error";
        case DWT2D_ERR_TIMEOUT: return "kernel wait timed out";
        case DWT2D_ERR_BOUNDS: return "store out of bounds (bounds-checked build)";
    }
    return "unknown status";
}

}  // extern "C"
