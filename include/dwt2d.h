/*
 * dwt2d.h -- C ABI of a GB300 (sm_103a) library for the multilevel 2-D discrete
 * wavelet transform computed by lifting, in the separable and non-separable
 * forms of Barina et al., "Accelerating Discrete Wavelet Transforms on GPUs"
 * (arXiv 1705.08266).
 *
 * What is computed
 * ----------------
 * One level splits an H x W image into four bands (Sec. 2: the 2-D transform
 * is the tensor product of 1-D transforms and yields a quadruple of
 * coefficients).  With quadruple (r, c) = (x[2r][2c], x[2r][2c+1],
 * x[2r+1][2c], x[2r+1][2c+1]) = (c0, c1, c2, c3):
 *   c0 -> LL, c1 -> HL (high pass along rows), c2 -> LH, c3 -> HH.
 * Bands are stored in the Mallat layout: LL is the top-left ceil(H/2) x
 * ceil(W/2) block, HL top-right, LH bottom-left, HH bottom-right.  Level l+1
 * transforms the LL of level l (multi-scale Mallat recursion; the paper
 * treats one scale and names more as future work, Sec. 5).
 *
 * Lifting (Sec. 2, Eq. 2): per (predict P, update U) pair, the separable
 * scheme runs T_P^H, T_P^V, S_U^H, S_U^V (four barrier steps); the
 * non-separable scheme (Sec. 3) runs the spatial predict T_P and the spatial
 * update S_U (two steps); the reduced form (Sec. 3, P = P0 + P1, U = U0 + U1)
 * computes the same two steps with fewer multiply-accumulates.  CDF 9/7 uses
 * two pairs and a final scaling low / K, high * K per axis
 * (K = 1.230174104914001); reversible LeGall 5/3 uses one integer pair
 * d = x_odd - floor((e_i + e_{i+1})/2), s = x_even + floor((d_{i-1} + d_i + 2)/4),
 * applied in the order T^H, T^V, S^H, S^V, which every scheme reproduces
 * bit for bit.  Borders use whole-sample symmetric extension; an axis of
 * length 1 is left unchanged.
 *
 * Schemes ending in _MULTIPASS run every lifting step as its own kernel that
 * exchanges all coefficients through HBM: the GB300 restatement of the paper's
 * pixel-shader mapping, in which results are exchanged through off-chip
 * textures and nothing stays in registers (Sec. 3, last paragraphs).  The
 * other schemes keep a level's data on chip: tiles staged by TMA, lifting in
 * registers with warp shuffles, several levels fused per launch.
 *
 * Conventions
 * -----------
 * - Every pointer named d_* is a device pointer of the current device; the
 *   caller allocates and owns all device memory and the stream.  The library
 *   never allocates device memory, never synchronizes a stream (except the
 *   *_host calls and dwt2d_workspace_status, which say so), never prints and
 *   never aborts.
 * - Pitches are in bytes, must be multiples of 16 and at least width *
 *   element size; device base pointers must be 16-byte aligned
 *   (DWT2D_ERR_ALIGN otherwise).
 * - Element types: DWT2D_F32 (CDF 9/7), DWT2D_I32 (LeGall 5/3),
 *   DWT2D_F16 / DWT2D_BF16 (CDF 9/7 with 16-bit storage, FP32 arithmetic,
 *   stored value = coefficient / scale).  Other pairs: DWT2D_ERR_UNSUPPORTED.
 * - src and dst must not overlap.  Launch errors return DWT2D_ERR_CUDA; a
 *   kernel that gives up waiting on a copy (bounded waits) records
 *   DWT2D_ERR_TIMEOUT in the workspace, read by dwt2d_workspace_status.
 */
#ifndef DWT2D_H
#define DWT2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwt2d_plan_s* dwt2d_plan_t; /* opaque, host memory, owned by the caller */

typedef enum { DWT2D_CDF97 = 0, DWT2D_LEGALL53 = 1 } dwt2d_wavelet;

typedef enum {
    DWT2D_SEPARABLE = 0,            /* S_U^V | S_U^H | T_P^V | T_P^H per pair (Sec. 2) */
    DWT2D_NONSEP = 1,               /* S_U | T_P, plain matrices (Sec. 3)              */
    DWT2D_NONSEP_REDUCED = 2,       /* S_U | T_P with P = P0 + P1, U = U0 + U1 (Sec. 3) */
    DWT2D_SEPARABLE_MULTIPASS = 3,  /* one HBM round trip per step (shader mapping)    */
    DWT2D_NONSEP_MULTIPASS = 4,
    DWT2D_NONSEP_REDUCED_MULTIPASS = 5,
    DWT2D_SEPARABLE_CONVOLUTION = 6 /* N^V | N^H: 9/7 filter bank per level (Sec. 2, Eq. 1);
                                       CDF 9/7 only; its inverse runs the reduced lifting */
} dwt2d_scheme;

typedef enum { DWT2D_F32 = 0, DWT2D_I32 = 1, DWT2D_F16 = 2, DWT2D_BF16 = 3 } dwt2d_dtype;

typedef enum { DWT2D_SYMMETRIC_WHOLE = 0 } dwt2d_boundary;

typedef enum {
    DWT2D_OK = 0,
    DWT2D_ERR_INVALID = -1,     /* bad argument (null pointer, size, level count) */
    DWT2D_ERR_UNSUPPORTED = -2, /* wavelet / dtype / scheme combination not offered */
    DWT2D_ERR_ALIGN = -3,       /* pointer or pitch alignment */
    DWT2D_ERR_NOMEM = -4,       /* host allocation of the plan failed */
    DWT2D_ERR_CUDA = -5,        /* a CUDA call or launch failed */
    DWT2D_ERR_TIMEOUT = -6,     /* a kernel gave up a bounded wait */
    DWT2D_ERR_BOUNDS = -7       /* a bounds-checked build (DWT_BOUNDS_CHECK) caught a store
                                   outside its buffer (the store was skipped) */
} dwt2d_status;

/*
 * dwt2d_plan -- validate a transform description and build a host plan.
 *   Problem statement: Sec. 2 (single-scale 2-D DWT of an image by lifting,
 *   Eq. 2) and Sec. 3 (non-separable scheme); levels > 1 is the Mallat
 *   recursion on LL.
 *   out             receives the plan (free with dwt2d_plan_destroy).
 *   height, width   image size, >= 1 each, at most 65536 each.
 *   levels          1 .. 16.
 *   workspace_bytes receives the size of the device workspace that every
 *                   forward / inverse call on this plan needs (>= 256).  The
 *                   workspace must be zeroed once before first use
 *                   (dwt2d_workspace_init); one workspace must not be used by
 *                   two calls that run at the same time.
 *   Errors: DWT2D_ERR_INVALID, DWT2D_ERR_UNSUPPORTED, DWT2D_ERR_NOMEM.
 *   The plan is immutable; concurrent calls on different streams with
 *   different workspaces may share it.
 */
dwt2d_status dwt2d_plan(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                        dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                        dwt2d_dtype dtype, size_t* workspace_bytes);

/*
 * dwt2d_plan_options -- how a plan cuts its work into launches.  These knobs
 *   change the launch decomposition, not the arithmetic: every setting gives
 *   the same result bit for bit, except that with 16-bit storage the LL
 *   handed from one launch to the next is stored (rounded) in 16 bits, so
 *   fuse_first / fuse_max move those roundings (the result stays within the
 *   16-bit tolerance).  Every field 0 = the library default
 *   (measured fastest on GB300 at 8192 x 8192, 5 levels); switches take
 *   1 = on, -1 = off.  The library reads no environment variables.
 */
typedef struct {
    int32_t fuse_first;            /* levels fused in the first launch, 1-3 (default 2) */
    int32_t fuse_max;              /* at most per later launch, 1-3 (default 2; 3 runs 4 quadruple
                                      columns per lane; 16-bit storage caps both at 2) */
    int32_t fwd_warps_per_sm;      /* warps a forward launch is cut into, per SM (default 16) */
    int32_t inv_warps_per_sm;      /* the same for the inverse (default 12) */
    int32_t fwd_warps_per_sm_large;/* forward launches whose row segments stay at least
                                      large_segment rows long at this many warps per SM take it
                                      (default 48 for CDF 9/7, 44 for LeGall 5/3 at 2 columns per
                                      lane, 24 at 4; -1: never) */
    int32_t inv_warps_per_sm_large;/* the same for the inverse (default 64 at 2 columns per lane,
                                      24 at 4; -1: never) */
    int32_t large_segment;         /* that threshold, quadruple rows of the launch's last level
                                      (default 16) */
    int32_t min_segment;           /* shortest row segment of a warp (default 2) */
    int32_t fwd_seg_interleave;    /* forward segment order: taken in this many interleaved groups
                                      (default: the launch's waves of resident warps; 1: top to
                                      bottom) */
    int32_t inv_seg_interleave;    /* the same for the inverse (default 1; -1: the launch's waves) */
    int32_t fwd_cols_per_lane;     /* quadruple columns per lane, 2 or 4 (default: 4 for a float
                                      launch of at most 2 fused levels whose rows give long
                                      segments at 24 warps per SM, else 2) */
    int32_t inv_cols_per_lane;     /* the same for the inverse, 2 or 4 (default 2) */
    int32_t programmatic_launch;   /* device entry points launch with programmatic stream
                                      serialization (default on) */
    int32_t host_bands;            /* row bands of the *_host entry points, 1-64 (default 8) */
    int32_t host_pipeline;         /* *_host entry points overlap copies and transform (default on) */
    int32_t fwd_short_tail;        /* in a large launch, the rows one wave of warps takes last are
                                      cut into segments this many times shorter, 2-64, so that
                                      the launch drains quickly (default 3 at 2 columns per lane,
                                      4 at 4; -1: off) */
    int32_t inv_short_tail;        /* the same for the inverse (default 4) */
} dwt2d_plan_options;

/*
 * dwt2d_plan_ex -- dwt2d_plan with launch options (NULL = all defaults, which
 *   is what dwt2d_plan does).  Errors as dwt2d_plan, plus DWT2D_ERR_INVALID
 *   for an option out of its range.
 */
dwt2d_status dwt2d_plan_ex(dwt2d_plan_t* out, int32_t height, int32_t width, int32_t levels,
                           dwt2d_wavelet wavelet, dwt2d_scheme scheme, dwt2d_boundary boundary,
                           dwt2d_dtype dtype, const dwt2d_plan_options* options,
                           size_t* workspace_bytes);

/*
 * dwt2d_forward -- image -> Mallat-layout coefficients (Sec. 2 and Sec. 3).
 *   d_src           height x width elements of the plan's dtype, row pitch
 *                   src_pitch_bytes.  Not modified.
 *   d_dst           height x width coefficients, row pitch dst_pitch_bytes.
 *   d_workspace     workspace_bytes from dwt2d_plan (device, 16-byte aligned).
 *   scale           16-bit storage only: stored value = value / scale, for
 *                   input and coefficients alike (> 0); ignored otherwise.
 *   stream          a cudaStream_t (NULL = legacy default stream).
 *   Asynchronous on stream.  Errors: DWT2D_ERR_INVALID, DWT2D_ERR_ALIGN,
 *   DWT2D_ERR_CUDA.
 *   The streaming kernels are launched with programmatic stream
 *   serialization (environment DWT2D_PDL=0 at plan creation turns it off): a
 *   launch may become resident while the kernel before it on `stream` (the
 *   call's previous launch, or the caller's own kernel) drains, and every
 *   thread waits for that kernel's completion and memory before its first
 *   global access.  Stream order is unchanged for the caller.  An event
 *   recorded between two launches (dwt2d_plan_set_launch_events) suspends
 *   the overlap of those two.
 */
dwt2d_status dwt2d_forward(dwt2d_plan_t plan, const void* d_src, int64_t src_pitch_bytes,
                           void* d_dst, int64_t dst_pitch_bytes, void* d_workspace,
                           float scale, void* stream);

/*
 * dwt2d_inverse -- Mallat-layout coefficients -> image: the inverse of Eq. 2,
 *   every lifting step undone in reverse order (negated filters; the integer
 *   5/3 steps undone exactly), coarse levels first.  Arguments as
 *   dwt2d_forward, with d_src the coefficients and d_dst the image.
 */
dwt2d_status dwt2d_inverse(dwt2d_plan_t plan, const void* d_src, int64_t src_pitch_bytes,
                           void* d_dst, int64_t dst_pitch_bytes, void* d_workspace,
                           float scale, void* stream);

/*
 * dwt2d_forward_host / dwt2d_inverse_host -- the same transform on HOST
 *   buffers: copies h_src (host, pitch h_src_pitch_bytes; pinned memory for
 *   overlap) into d_stage_in, transforms into d_stage_out, copies d_stage_out
 *   back to h_dst, then synchronizes stream.  The forward of a fused-lifting
 *   plan with at least 1024 rows overlaps the three: the image goes in by row
 *   bands on an internal stream, the first level group runs on `stream` band
 *   by band as its input rows arrive, and the finished detail bands come back
 *   on a second internal stream while later bands still go in (the plan owns
 *   the two streams; a plan's _host calls must not overlap each other; the
 *   band count is the plan option host_bands, default 8).  The
 *   inverse does the same the other way round: the coarse levels' top-left
 *   region goes in first, the finest level group runs by row bands as their
 *   detail bands arrive, and finished image rows come back meanwhile.
 *   d_stage_in, d_stage_out: device buffers of height rows x d_pitch_bytes.
 *   Errors: as dwt2d_forward, plus DWT2D_ERR_CUDA for a failed copy.
 */
dwt2d_status dwt2d_forward_host(dwt2d_plan_t plan, const void* h_src, int64_t h_src_pitch_bytes,
                                void* h_dst, int64_t h_dst_pitch_bytes, void* d_stage_in,
                                void* d_stage_out, int64_t d_pitch_bytes, void* d_workspace,
                                float scale, void* stream);
dwt2d_status dwt2d_inverse_host(dwt2d_plan_t plan, const void* h_src, int64_t h_src_pitch_bytes,
                                void* h_dst, int64_t h_dst_pitch_bytes, void* d_stage_in,
                                void* d_stage_out, int64_t d_pitch_bytes, void* d_workspace,
                                float scale, void* stream);

/*
 * dwt2d_workspace_init -- zero the 256-byte header of a workspace (its first
 *   word is the status word; asynchronous on stream).  Call once after
 *   allocating a workspace.
 * dwt2d_workspace_status -- copy the status word to the host (synchronizes
 *   stream) and return DWT2D_OK or the recorded error (DWT2D_ERR_TIMEOUT);
 *   after an error it zeroes the header again.
 */
dwt2d_status dwt2d_workspace_init(void* d_workspace, void* stream);
dwt2d_status dwt2d_workspace_status(void* d_workspace, void* stream);

/*
 * dwt2d_plan_info -- kernel launches one forward call makes (for launch
 *   accounting), and the number of levels fused per launch, in launch order.
 *   fused: array of at least 16 entries (may be NULL).
 */
dwt2d_status dwt2d_plan_info(dwt2d_plan_t plan, int32_t* launches_per_call, int32_t* fused,
                             int32_t* n_groups);

/*
 * dwt2d_plan_launch_info -- the shape of launch i (in launch order) of a
 *   forward (inverse = 0) or inverse (inverse = 1) call: levels fused,
 *   quadruple columns per lane and warps.  Any output may be NULL.  Streaming
 *   schemes only (DWT2D_ERR_UNSUPPORTED for the multipass schemes and the
 *   convolution forward); needs no GPU.
 */
dwt2d_status dwt2d_plan_launch_info(dwt2d_plan_t plan, int32_t inverse, int32_t i, int32_t* fused,
                                    int32_t* cols_per_lane, int32_t* warps);

/*
 * dwt2d_plan_set_launch_events -- profiling hook.  With events != NULL, every
 *   later forward / inverse call on this plan records events[2i] (a
 *   cudaEvent_t) on its stream just before its i-th kernel launch and
 *   events[2i+1] just after it, for i < count.  NULL turns the hook off.  The
 *   caller owns the events.  Not safe while another call uses the plan.
 */
dwt2d_status dwt2d_plan_set_launch_events(dwt2d_plan_t plan, void** events, int32_t count);

/*
 * dwt2d_forward_noalloc -- dwt2d_forward for callers that cannot allocate
 *   device memory.  (The paper has no counterpart: this is a library service.)
 *
 *   Some callers never get to call cudaMalloc: a plugin inside a host
 *   application that owns every byte of device memory and hands the plugin
 *   only its input and output buffers, code on a latency-critical path where
 *   an allocation (which may synchronize the device) is not acceptable, or a
 *   service that must not be able to fail with out-of-memory in the middle of
 *   a request.  This entry point needs no workspace argument: the scratch the
 *   multilevel forward transform uses between its launches (and the status
 *   word of its bounded waits) lives in one fixed array of
 *   DWT2D_NOALLOC_SCRATCH_BYTES in the library's device memory, which every
 *   GPU that loads the library holds until the process exits.  The caller
 *   still passes the image and the coefficient buffer, exactly as for
 *   dwt2d_forward, and gets the same coefficients.
 *
 *   - Every call looks up the current device's address of the array
 *     (cudaGetSymbolAddress) with the caller's device current.  The first
 *     call on a device may load the library's device code there; make that
 *     first call before any stream capture.
 *   - A plan whose workspace_bytes exceeds DWT2D_NOALLOC_SCRATCH_BYTES is
 *     rejected with DWT2D_ERR_INVALID before any GPU work (for example an
 *     8192 x 8192 float image with 5 levels fits, 16384 x 16384 with 6 levels
 *     or any multipass scheme of a large image does not).
 *   - All calls on a device share the one array, and it keeps whatever the
 *     last call left in it.  Each call clears the status word first; the rest
 *     is written before it is read.  Calls whose kernels overlap on the GPU
 *     (two streams, or a second call before the first has finished on another
 *     stream) race on the array and corrupt each other's results: serialise
 *     them, for example on one stream.
 *   - Nothing here calls cudaMalloc, cudaFree or an allocating library
 *     routine.  The arguments are checked as dwt2d_forward checks them, and
 *     a call that is refused puts nothing on the stream.  Kernel errors
 *     (a bounded wait that gave up) land in the array's status word, which
 *     the caller has no address for: read them with dwt2d_noalloc_status.
 *
 * dwt2d_noalloc_status -- dwt2d_workspace_status for the array above:
 *   synchronizes stream, returns DWT2D_OK or the error the kernels of the
 *   calls so far recorded (DWT2D_ERR_TIMEOUT, or DWT2D_ERR_BOUNDS in a
 *   bounds-checked build), and resets the status word to zero.  The next
 *   dwt2d_forward_noalloc clears it too, so read it before that call.
 */
#define DWT2D_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
dwt2d_status dwt2d_forward_noalloc(dwt2d_plan_t plan, const void* d_src, int64_t src_pitch_bytes,
                                   void* d_dst, int64_t dst_pitch_bytes, float scale, void* stream);
dwt2d_status dwt2d_noalloc_status(void* stream);

/*
 * Batched transforms -- many images of different sizes, level counts,
 * wavelets, storage types and directions in a few launches.  (The paper
 * transforms one image at a time; this is a library service for workloads of
 * many small images, where per-image launches are latency-bound.)
 *
 * Images are processed in phases: phase k runs level group k of every forward
 * image (fine to coarse) and level group (groups - 1 - k) of every inverse
 * image (coarse to fine).  Within a phase, one launch covers every image of
 * the same direction, storage type and fusion depth: its warps walk a table of
 * per-image descriptors (geometry and TMA tensor maps) in device memory.
 */
typedef struct dwt2d_batch_s* dwt2d_batch_t;

typedef struct {
    int32_t height, width, levels;
    dwt2d_wavelet wavelet;
    dwt2d_dtype dtype;
    int32_t inverse;          /* 0: image -> coefficients, 1: coefficients -> image */
    const void* d_src;        /* device, 16-byte aligned, pitch a multiple of 16 */
    int64_t src_pitch_bytes;
    void* d_dst;              /* device, must not overlap d_src */
    int64_t dst_pitch_bytes;
} dwt2d_batch_item;

/* Tuning knobs (0 = library default): levels fused in the first launch of an
 * image (1 or 2; default 2), at most per later launch (1 or 2; default 2),
 * warps per SM that the rows of one launch are cut into (default 48; the
 * batched kernels keep 12 warps per SM resident, 8 for the persistent form
 * at 4 columns per lane, so 48 is four or six waves), the
 * smallest row segment of a warp (quadruple rows of the last fused level;
 * default 2), and whether the batch's launches use programmatic stream
 * serialization (1 on, -1 or 0 off: measured neutral to 1 % slower for
 * batches).  Every warp of a launch streams the same number of rows.
 * cols_per_lane: quadruple columns per lane at the first level of a launch
 * (0 or 2: 2, a 128-pixel strip per warp; 4: a 256-pixel strip with half the
 * strips' halo overlap; any other value is DWT2D_ERR_INVALID). */
typedef struct {
    int32_t fuse_first, fuse_max, warps_per_sm, min_segment;
    int32_t programmatic_launch;
    int32_t persistent;  /* 1: one persistent launch per direction and storage type over a
                            queue of every level group's work items (warps take items from a
                            counter; an item waits, bounded, until the level group it reads
                            is done); otherwise one launch per level group, direction,
                            storage type and fusion depth */
    int32_t cols_per_lane;
} dwt2d_tuning;

/*
 * dwt2d_batch_create -- validate n items (each as dwt2d_plan would, plus its
 *   buffers as dwt2d_forward would) for one lifting scheme (DWT2D_SEPARABLE,
 *   DWT2D_NONSEP or DWT2D_NONSEP_REDUCED) and plan the launches.  The items
 *   are copied; their buffers must stay valid while the batch is used.
 *   tuning may be NULL.  workspace_bytes receives the device workspace the
 *   batch needs (descriptor tables + inter-launch LL buffers + status word).
 * dwt2d_batch_upload -- write the descriptor tables into d_workspace
 *   (asynchronous on stream; not capturable: call it before any capture).
 *   Zeroes the status word.
 * dwt2d_batch_launch -- launch every kernel of the batch on stream (in the
 *   persistent form, after one memset of the queue counters); nothing else,
 *   so it can be captured in a CUDA graph and replayed.  The workspace must
 *   have been uploaded for this batch.
 * dwt2d_batch_info -- kernel launches per dwt2d_batch_launch and warps in all.
 */
dwt2d_status dwt2d_batch_create(dwt2d_batch_t* out, const dwt2d_batch_item* items, int32_t n,
                                dwt2d_scheme scheme, const dwt2d_tuning* tuning,
                                size_t* workspace_bytes);
dwt2d_status dwt2d_batch_upload(dwt2d_batch_t batch, void* d_workspace, void* stream);

/*
 * dwt2d_batch_staging_bytes -- host bytes of the batch's descriptor tables.
 * dwt2d_batch_upload_staged -- dwt2d_batch_upload, copying the tables from
 *   h_staging: pinned host memory (cudaHostAlloc or registered), 16-byte
 *   aligned, at least dwt2d_batch_staging_bytes long, owned by the caller and
 *   left untouched until the stream has passed the upload.  A copy from
 *   pageable memory may make the host wait until the stream drains; from
 *   pinned memory it is queued at once, so a serving loop can queue a new
 *   batch on another stream while earlier batches run.
 */
dwt2d_status dwt2d_batch_staging_bytes(dwt2d_batch_t batch, size_t* bytes);
dwt2d_status dwt2d_batch_upload_staged(dwt2d_batch_t batch, void* d_workspace, void* h_staging,
                                       size_t staging_bytes, void* stream);
dwt2d_status dwt2d_batch_launch(dwt2d_batch_t batch, void* d_workspace, void* stream);
dwt2d_status dwt2d_batch_info(dwt2d_batch_t batch, int32_t* launches, int64_t* warps);
void dwt2d_batch_destroy(dwt2d_batch_t batch);

void dwt2d_plan_destroy(dwt2d_plan_t plan);
const char* dwt2d_status_string(dwt2d_status status);

#ifdef __cplusplus
}
#endif

#endif /* DWT2D_H */
