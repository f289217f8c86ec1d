// dwt2d_forward_noalloc: the forward transform for callers that cannot
// allocate device memory.
//
// A plugin living inside a host application that owns all device memory, or
// code on a path where an allocation (and the device synchronisation it may
// bring) is not allowed, still has to hand the multilevel transform some
// scratch: the LL band that one fused launch leaves for the next, and the
// status word of the kernels' bounded waits.  Here that scratch is one fixed
// array in the library's own device memory, sized DWT2D_NOALLOC_SCRATCH_BYTES
// (8 MiB), which exists on every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address: the
// address is looked up on every call, with the caller's device current, and
// passed to the kernels like any caller-owned workspace.  (Looking it up each
// time costs little once the module is loaded, and stays right if the
// device's context is ever torn down and created again.)
#include <cuda_runtime.h>

#include "dwt2d.h"
#include "dwt_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[DWT2D_NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device.
dwt2d_status scratch_address(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DWT2D_ERR_CUDA;
    *out = p;
    return DWT2D_OK;
}

}  // namespace

extern "C" dwt2d_status dwt2d_forward_noalloc(dwt2d_plan_t plan, const void* d_src,
                                              int64_t src_pitch_bytes, void* d_dst,
                                              int64_t dst_pitch_bytes, float scale, void* stream) {
    if (!plan) return DWT2D_ERR_INVALID;
    if (dwt::plan_workspace_bytes(plan) > DWT2D_NOALLOC_SCRATCH_BYTES) return DWT2D_ERR_INVALID;
    void* scratch = nullptr;
    dwt2d_status s = scratch_address(&scratch);
    if (s != DWT2D_OK) return s;
    // every check dwt2d_forward makes, before anything goes on the stream
    s = dwt::check_transform_args(plan, d_src, src_pitch_bytes, d_dst, dst_pitch_bytes, scratch, scale);
    if (s != DWT2D_OK) return s;
    // the header (its first word is the status word) must start at zero;
    // everything else is written before it is read
    if (cudaMemsetAsync(scratch, 0, 256, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return DWT2D_ERR_CUDA;
    return dwt2d_forward(plan, d_src, src_pitch_bytes, d_dst, dst_pitch_bytes, scratch, scale, stream);
}

extern "C" dwt2d_status dwt2d_noalloc_status(void* stream) {
    void* scratch = nullptr;
    const dwt2d_status s = scratch_address(&scratch);
    if (s != DWT2D_OK) return s;
    return dwt2d_workspace_status(scratch, stream);
}
