// Host/device argument blocks shared by the C ABI and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dwt2d.h"

namespace dwt {

constexpr int kMaxFused = 3;  // levels fused in one streaming launch

// Lifting schemes: separable (Sec. 2), non-separable and its reduced form (Sec. 3).
enum Scheme { SCH_SEP = 0, SCH_NONSEP = 1, SCH_RED = 2 };

// Geometry of one warp-streaming launch (forward or inverse, 1..3 levels).
struct LevelArgs {
    int h, w;     // extent this level transforms (image or LL of the level before)
    float s[4];   // forward: scale of LL, HL, LH, HH; inverse: its reciprocal
};

struct FusedArgs {
    LevelArgs lv[kMaxFused];
    // Mallat coefficient array (forward: written; inverse: read), element pitch
    void* mallat;
    long long mallat_pitch;
    // forward: LL of the last fused level is written here;
    // inverse: LL of the coarsest fused level is read from here
    void* ll;
    long long ll_pitch;
    // inverse only: the reconstructed image (or LL of the finest fused level - 1)
    void* out;
    long long out_pitch;
    int nstrips, nsegs, segq;        // warp work items = nstrips * nsegs
    int seg_f;                       // segment order interleave (<= 1: top to bottom)
    int seg_lo;                      // first row segment of this launch (launches over a subset)
    // segments [0, nbig) have segq rows (taken in seg_f interleaved groups);
    // segments [nbig, nsegs) are shorter, segq2 rows each, below them, taken
    // last and top to bottom (nbig == nsegs: every segment has segq rows)
    int nbig, segq2;
    long long mallat_elems, ll_elems, out_elems;  // buffer extents (elements) for checked builds
    int valid_px, xoff;              // strip width in input pixels and left halo offset
    int lane_lo, lane_hi;            // lanes that store
    int* err;                        // device status word (0 = ok)
    int pdl;                         // host: launch with programmatic stream serialization
    int ll_keep;                     // forward: store the LL with an L2 evict-last policy
};


// Where a multipass kernel reads or writes a level's coefficients.
struct Layout {
    const void* p;       // kind 0: interleaved image layout; kind 1: Mallat array (details)
    long long pitch;     // elements
    const void* ll;      // kind 1: the LL band (may be inside p)
    long long ll_pitch;  // elements
    int kind;
};

// One pass of the multipass (off-chip exchange) scheme.
struct PassArgs {
    int h, w;          // extent of the level
    Layout src, dst;
    float s[4];        // per-component scale applied on load (scale_in) or store (scale_out)
    float coef;        // float lifting coefficient of this step, sign included
    int scale_in, scale_out;
};

// One image (one level group) of a batched launch, in device memory.  The
// tensor maps (128-byte aligned) come first.  The forward uses m[0];
// the inverse m[0] (Mallat, level-1 box), m[1] (Mallat, level-2 box), m[2]
// (LL source).
struct BatchEntry {
    CUtensorMap m[3];
    FusedArgs args;
    int first_warp;  // first global warp of this entry in the launch (queue mode: in its queue)
    // queue mode: the entry's fusion depth, its done counter (image, level
    // group) and the counter of the group it consumes (-1: none) with the
    // number of work items that group has
    int nl, self, dep, dep_items;
};

// Persistent batched kernels (queue mode): `grid` one-warp CTAs take the
// `total` work items of a queue (entries of one direction and storage type,
// every level group, ordered by group) through the counter `head`; an item of
// a later group first waits (bounded) until done[dep] reaches dep_items.
// q1: quadruple columns per lane (2 or 4) of every item in the queue.
// Warps per SM that the queue kernels' register budget keeps resident.
__host__ __device__ constexpr int fwd_queue_resident(int q1) { return q1 >= 4 ? 8 : 12; }
__host__ __device__ constexpr int inv_queue_resident(int q1) { return q1 >= 4 ? 8 : 12; }
cudaError_t launch_fwd_queue(int elem, int scheme, int q1, const BatchEntry* table, int n, int total,
                             int* head, int* done, int* err, int grid, cudaStream_t st);
cudaError_t launch_inv_queue(int elem, int scheme, int q1, const BatchEntry* table, int n, int total,
                             int* head, int* done, int* err, int grid, cudaStream_t st);

// Kernel-geometry constants of the streaming forward kernel.
// warps per CTA: each warp is independent, so one-warp CTAs let the CTA
// scheduler refill an SM warp by warp (measured 1-4 % faster than 4)
constexpr int kFwdWarps = 1;
constexpr int kFwdSlots = 3;        // TMA ring depth per warp
constexpr int kFwdSlotRows = 8;     // image rows per TMA box (4 quadruple rows) with 2 columns per lane

// Image rows per TMA box of the forward kernel: 8, or 4 with 4 quadruple
// columns per lane and at most 2 fused levels.
int fwd_slot_rows(int nl, int q1);
size_t fwd_smem_bytes(int elem_bytes, int nl, int q1);

// Batched forward / inverse: entries of one element type, scheme, fusion
// depth (1 or 2) and quadruple columns per lane q1 (2 or 4); `grid` CTAs of
// kFwdWarps (forward) or kInvTmaWarps (inverse) warps.
// grid == 0 only sets the kernel's shared-memory attribute (done once, before
// any stream capture), so a launch itself is a plain kernel launch.
cudaError_t launch_fwd_batched(int elem, int scheme, int nl, int q1, const BatchEntry* table, int n,
                               int grid, cudaStream_t st, bool pdl);
cudaError_t launch_inv_batched(int elem, int scheme, int nl, int q1, const BatchEntry* table, int n,
                               int grid, cudaStream_t st, bool pdl);

// Launch `kernel` on `st`; with `pdl` the grid is launched with programmatic
// stream serialization (it may be scheduled while the previous kernel in the
// stream drains, and waits in griddepcontrol.wait before its first global
// access).  Only kernels that issue that wait may be launched with `pdl`.
template <class... P, class... A>
cudaError_t launch_kernel(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t st,
                          bool pdl, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// q1: quadruple columns per lane at the first fused level (2 or 4; 3 fused levels need 4)
cudaError_t launch_fwd_fused(int elem, int scheme, int nl, int q1, const CUtensorMap& map,
                             const FusedArgs& a, int grid, cudaStream_t st);
cudaError_t launch_inv_fused(int elem, int scheme, int nl, const FusedArgs& a, int grid,
                             cudaStream_t st);

// TMA-fed inverse for 1 or 2 fused levels: m1 / m2 map the Mallat array with
// boxes {32 q1 + 4, 4} and {16 q1 + 4, 2}; ml maps the LL source with the
// level-1 box (1 level) or the level-2 box (2 levels).
cudaError_t launch_inv_tma(int elem, int scheme, int nl, int q1, const CUtensorMap& m1,
                           const CUtensorMap& m2, const CUtensorMap& ml, const FusedArgs& a,
                           int grid, cudaStream_t st);
size_t inv_tma_smem_bytes(int elem_bytes, int nl, int q1);
// Level-1 quadruple rows per slot of the TMA inverse: 4, or 2 with 4 columns per lane.
int inv_slot_rows(int q1);
constexpr int kInvTmaWarps = 1;  // one-warp CTAs, as the forward

// One level of the separable convolution scheme (Sec. 2, Eq. 1).
struct ConvArgs {
    int h, w;
    const void* src;   // the level's input (image or LL), element pitch
    long long src_pitch;
    void* dst;         // Mallat array (detail bands of this level)
    long long dst_pitch;
    void* ll;          // LL output of this level
    long long ll_pitch;
    float h0[9];       // analysis low pass, centred (k = -4 .. 4)
    float g0[7];       // analysis high pass, centred (k = -3 .. 3)
};
cudaError_t launch_conv_fwd(int elem, const ConvArgs& a, cudaStream_t st);

// elem: 0 = float32, 1 = int32.  kind: the step (see dwt_multipass.cu).
cudaError_t launch_pass(int elem, int kind, bool fwd, const PassArgs& a, cudaStream_t st);

enum PassKind { P_TH = 0, P_TV, P_SH, P_SV, P_T, P_S, P_TR, P_SR };

// Workspace bytes a plan needs (0 for a null plan).
size_t plan_workspace_bytes(dwt2d_plan_t p);

// The argument checks of dwt2d_forward / dwt2d_inverse (buffers, alignment,
// pitches, 16-bit scale, src != dst), without any GPU work.
dwt2d_status check_transform_args(dwt2d_plan_t p, const void* src, int64_t src_pitch_bytes,
                                  const void* dst, int64_t dst_pitch_bytes, const void* ws,
                                  float scale);

}  // namespace dwt
