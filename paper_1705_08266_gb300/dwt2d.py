"""Python binding of libdwt2d.so: argument marshalling only.

Every step of the transform runs in the library's CUDA kernels; PyTorch only
provides device memory and streams.  The names follow the C ABI in
include/dwt2d.h: Plan wraps dwt2d_plan, Plan.forward / Plan.inverse wrap
dwt2d_forward / dwt2d_inverse, Plan.forward_host / inverse_host the host-buffer
entry points, Batch the dwt2d_batch_* calls.  There is no CPU fallback: if the
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DWT2D_LIBRARY selects another build of the same library (the bounds-checked
# one in tests)
LIB_PATH = os.environ.get("DWT2D_LIBRARY") or os.path.join(_HERE, "libdwt2d.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dwt2d.h")

WAVELETS = {"cdf97": 0, "legall53": 1}
SCHEMES = {
    "separable": 0,
    "nonsep": 1,
    "nonsep_reduced": 2,
    "separable_multipass": 3,
    "nonsep_multipass": 4,
    "nonsep_reduced_multipass": 5,
    "separable_convolution": 6,
}
DTYPES = {torch.float32: 0, torch.int32: 1, torch.float16: 2, torch.bfloat16: 3}
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported", -3: "alignment", -4: "no memory",
          -5: "CUDA error", -6: "timeout", -7: "store out of bounds (checked build)"}

_lib = None


class BatchItem(ctypes.Structure):
    """dwt2d_batch_item."""
    _fields_ = [("height", ctypes.c_int32), ("width", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("wavelet", ctypes.c_int), ("dtype", ctypes.c_int), ("inverse", ctypes.c_int32),
                ("d_src", ctypes.c_void_p), ("src_pitch_bytes", ctypes.c_int64),
                ("d_dst", ctypes.c_void_p), ("dst_pitch_bytes", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    """dwt2d_tuning (0 = library default)."""
    _fields_ = [("fuse_first", ctypes.c_int32), ("fuse_max", ctypes.c_int32),
                ("warps_per_sm", ctypes.c_int32), ("min_segment", ctypes.c_int32),
                ("programmatic_launch", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("cols_per_lane", ctypes.c_int32)]


class PlanOptions(ctypes.Structure):
    """dwt2d_plan_options (0 = library default; switches 1 on, -1 off)."""
    _fields_ = [(n, ctypes.c_int32) for n in (
        "fuse_first", "fuse_max", "fwd_warps_per_sm", "inv_warps_per_sm", "fwd_warps_per_sm_large",
        "inv_warps_per_sm_large", "large_segment", "min_segment", "fwd_seg_interleave",
        "inv_seg_interleave", "fwd_cols_per_lane", "inv_cols_per_lane", "programmatic_launch",
        "host_bands", "host_pipeline", "fwd_short_tail", "inv_short_tail")]


def plan_options(**kw) -> PlanOptions:
    """A dwt2d_plan_options with the named fields set (unknown names raise)."""
    o = PlanOptions()
    names = {f[0] for f in PlanOptions._fields_}
    for k, v in kw.items():
        if k not in names:
            raise KeyError(f"unknown plan option {k!r}")
        setattr(o, k, int(v))
    return o


class DwtError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: dwt2d status {status} ({STATUS.get(status, '?')})")


def lib() -> ctypes.CDLL:
    """Load libdwt2d.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1705_08266_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    L.dwt2d_plan.argtypes = [ctypes.POINTER(vp), i32, i32, i32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, ctypes.POINTER(sz)]
    L.dwt2d_plan_ex.argtypes = [ctypes.POINTER(vp), i32, i32, i32, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.POINTER(PlanOptions), ctypes.POINTER(sz)]
    L.dwt2d_noalloc_status.argtypes = [vp]
    for name in ("dwt2d_forward", "dwt2d_inverse"):
        getattr(L, name).argtypes = [vp, vp, i64, vp, i64, vp, f32, vp]
    for name in ("dwt2d_forward_host", "dwt2d_inverse_host"):
        getattr(L, name).argtypes = [vp, vp, i64, vp, i64, vp, vp, i64, vp, f32, vp]
    L.dwt2d_workspace_init.argtypes = [vp, vp]
    L.dwt2d_workspace_status.argtypes = [vp, vp]
    L.dwt2d_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.dwt2d_plan_launch_info.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)]
    L.dwt2d_plan_launch_info.restype = ctypes.c_int
    L.dwt2d_plan_set_launch_events.argtypes = [vp, ctypes.POINTER(vp), i32]
    L.dwt2d_plan_set_launch_events.restype = ctypes.c_int
    L.dwt2d_plan_destroy.argtypes = [vp]
    L.dwt2d_plan_destroy.restype = None
    L.dwt2d_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(BatchItem), i32, ctypes.c_int,
                                     ctypes.POINTER(Tuning), ctypes.POINTER(sz)]
    L.dwt2d_batch_upload.argtypes = [vp, vp, vp]
    L.dwt2d_batch_staging_bytes.argtypes = [vp, ctypes.POINTER(sz)]
    L.dwt2d_batch_staging_bytes.restype = ctypes.c_int
    L.dwt2d_batch_upload_staged.argtypes = [vp, vp, vp, sz, vp]
    L.dwt2d_batch_upload_staged.restype = ctypes.c_int
    L.dwt2d_batch_launch.argtypes = [vp, vp, vp]
    L.dwt2d_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.dwt2d_batch_destroy.argtypes = [vp]
    L.dwt2d_batch_destroy.restype = None
    L.dwt2d_status_string.argtypes = [ctypes.c_int]
    L.dwt2d_status_string.restype = ctypes.c_char_p
    for name in ("dwt2d_plan", "dwt2d_plan_ex", "dwt2d_noalloc_status", "dwt2d_forward",
                 "dwt2d_inverse", "dwt2d_forward_host",
                 "dwt2d_inverse_host", "dwt2d_workspace_init", "dwt2d_workspace_status",
                 "dwt2d_plan_info", "dwt2d_batch_create", "dwt2d_batch_upload",
                 "dwt2d_batch_launch", "dwt2d_batch_info"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def header_functions() -> list:
    """Names of the functions that include/dwt2d.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dwt2d_\w+)\s*\(", text)))


def _check(status: int, what: str):
    if status != 0:
        raise DwtError(status, what)


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def pitch_elems(width: int, dtype: torch.dtype) -> int:
    """Row pitch (elements) that makes every row start on a 16-byte boundary."""
    es = dtype.itemsize
    return ((width * es + 15) // 16 * 16) // es


def empty_image(height: int, width: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    """An (height, width) view with a 16-byte-aligned row pitch."""
    buf = torch.empty((height, pitch_elems(width, dtype)), dtype=dtype, device=device)
    return buf[:, :width]


def as_pitched(t: torch.Tensor) -> torch.Tensor:
    """t itself if its rows are 16-byte aligned and unit-stride, else a pitched copy."""
    es = t.element_size()
    if t.dim() == 2 and t.stride(1) == 1 and (t.stride(0) * es) % 16 == 0 and t.data_ptr() % 16 == 0:
        return t
    out = empty_image(t.shape[0], t.shape[1], t.dtype, t.device)
    out.copy_(t)
    return out


def workspace_bytes(height: int, width: int, levels: int, wavelet: str = "cdf97",
                    scheme: str = "nonsep_reduced", dtype: Optional[torch.dtype] = None) -> int:
    """Device workspace a default plan of this transform needs (dwt2d_plan,
    then dwt2d_plan_destroy; no Python plan object)."""
    L = lib()
    if dtype is None:
        dtype = torch.int32 if wavelet == "legall53" else torch.float32
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check(L.dwt2d_plan(ctypes.byref(h), height, width, levels, WAVELETS[wavelet], SCHEMES[scheme], 0,
                        DTYPES[dtype], ctypes.byref(ws)), "dwt2d_plan")
    L.dwt2d_plan_destroy(h)
    return ws.value


class Plan:
    """A transform description (dwt2d_plan) plus convenience wrappers."""

    def __init__(self, height: int, width: int, levels: int, wavelet: str = "cdf97",
                 scheme: str = "nonsep_reduced", dtype: Optional[torch.dtype] = None,
                 options: Optional[dict] = None):
        """options: dwt2d_plan_options fields by name (launch decomposition only)."""
        L = lib()
        if dtype is None:
            dtype = torch.int32 if wavelet == "legall53" else torch.float32
        self.height, self.width, self.levels = height, width, levels
        self.wavelet, self.scheme, self.dtype = wavelet, scheme, dtype
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        opts = ctypes.byref(plan_options(**options)) if options else None
        _check(L.dwt2d_plan_ex(ctypes.byref(self._h), height, width, levels, WAVELETS[wavelet],
                               SCHEMES[scheme], 0, DTYPES[dtype], opts, ctypes.byref(ws)),
               "dwt2d_plan_ex")
        self.workspace_bytes = ws.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.dwt2d_plan_destroy(h)
            self._h = None

    def info(self):
        """(launches per call, fused levels per launch)."""
        n, ng = ctypes.c_int32(), ctypes.c_int32()
        fused = (ctypes.c_int32 * 16)()
        _check(lib().dwt2d_plan_info(self._h, ctypes.byref(n), fused, ctypes.byref(ng)), "plan_info")
        return n.value, [fused[i] for i in range(ng.value)]

    def launch_info(self, inverse: bool = False):
        """[(levels fused, columns per lane, warps)] of each launch of a call, in launch order."""
        out = []
        n = self.info()[0]
        for i in range(n):
            f, q, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            _check(lib().dwt2d_plan_launch_info(self._h, int(inverse), i, ctypes.byref(f), ctypes.byref(q),
                                                ctypes.byref(w)), "plan_launch_info")
            out.append((f.value, q.value, w.value))
        return out

    def set_launch_events(self, events):
        """Record events[2i] / events[2i+1] (torch.cuda.Event) around launch i of later calls."""
        if not events:
            self._ev_keep = None
            _check(lib().dwt2d_plan_set_launch_events(self._h, None, 0), "set_launch_events")
            return
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        self._ev_keep = (arr, events)
        _check(lib().dwt2d_plan_set_launch_events(self._h, arr, len(events) // 2), "set_launch_events")

    def workspace(self, device="cuda", stream=None) -> torch.Tensor:
        ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
        _check(lib().dwt2d_workspace_init(ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)),
               "workspace_init")
        return ws

    def status(self, workspace: torch.Tensor, stream=None) -> int:
        return lib().dwt2d_workspace_status(ctypes.c_void_p(workspace.data_ptr()), _stream_ptr(stream))

    def _run(self, name, src, dst, workspace, scale, stream):
        src = as_pitched(src)
        if dst is None:
            dst = empty_image(self.height, self.width, self.dtype, src.device)
        own_ws = workspace is None
        if own_ws:
            workspace = self.workspace(src.device, stream)
        es = src.element_size()
        st = getattr(lib(), name)(self._h, ctypes.c_void_p(src.data_ptr()), src.stride(0) * es,
                                  ctypes.c_void_p(dst.data_ptr()), dst.stride(0) * es,
                                  ctypes.c_void_p(workspace.data_ptr()), float(scale),
                                  _stream_ptr(stream))
        _check(st, name)
        if own_ws:
            # nobody else can read the status word of a workspace made here:
            # read it now (synchronizes the stream) so kernel errors surface
            _check(self.status(workspace, stream), name + " (kernel status)")
        return dst

    def forward(self, src: torch.Tensor, dst: Optional[torch.Tensor] = None,
                workspace: Optional[torch.Tensor] = None, scale: float = 1.0, stream=None):
        """Image (H, W) on the device -> Mallat coefficients (H, W)."""
        return self._run("dwt2d_forward", src, dst, workspace, scale, stream)

    def inverse(self, src: torch.Tensor, dst: Optional[torch.Tensor] = None,
                workspace: Optional[torch.Tensor] = None, scale: float = 1.0, stream=None):
        """Mallat coefficients (H, W) on the device -> image (H, W)."""
        return self._run("dwt2d_inverse", src, dst, workspace, scale, stream)

    def _run_host(self, name, h_src, h_dst, d_in, d_out, workspace, scale, stream):
        es = h_src.element_size()
        assert d_in.stride(0) == d_out.stride(0)
        st = getattr(lib(), name)(self._h, ctypes.c_void_p(h_src.data_ptr()), h_src.stride(0) * es,
                                  ctypes.c_void_p(h_dst.data_ptr()), h_dst.stride(0) * es,
                                  ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                  d_in.stride(0) * es, ctypes.c_void_p(workspace.data_ptr()),
                                  float(scale), _stream_ptr(stream))
        _check(st, name)
        return h_dst

    def forward_host(self, h_src, h_dst, d_in, d_out, workspace, scale=1.0, stream=None):
        """Host image -> host coefficients through device staging buffers (synchronous)."""
        return self._run_host("dwt2d_forward_host", h_src, h_dst, d_in, d_out, workspace, scale, stream)

    def inverse_host(self, h_src, h_dst, d_in, d_out, workspace, scale=1.0, stream=None):
        return self._run_host("dwt2d_inverse_host", h_src, h_dst, d_in, d_out, workspace, scale, stream)


class Batch:
    """Many transforms in a few launches (dwt2d_batch_*).

    jobs: sequence of (src, dst, levels, wavelet, inverse) with src / dst device
    tensors of the same shape and dtype (16-byte-aligned rows; see empty_image).
    The tensors are referenced, not copied: they must stay alive and in place
    while the batch is used.  upload() writes the descriptor tables into the
    workspace; launch() only launches kernels (capturable in a CUDA graph).
    """

    def __init__(self, jobs, scheme: str = "nonsep_reduced", tuning=None):
        L = lib()
        self.jobs = list(jobs)
        self.scheme = scheme
        arr = (BatchItem * max(1, len(self.jobs)))()
        for i, (src, dst, levels, wavelet, inverse) in enumerate(self.jobs):
            if src.shape != dst.shape or src.dtype != dst.dtype or src.dim() != 2:
                raise ValueError("src and dst must be 2-D tensors of one shape and dtype")
            es = src.element_size()
            arr[i] = BatchItem(src.shape[0], src.shape[1], levels, WAVELETS[wavelet], DTYPES[src.dtype],
                               int(bool(inverse)), src.data_ptr(), src.stride(0) * es, dst.data_ptr(),
                               dst.stride(0) * es)
        tun = None
        if tuning is not None:
            tun = ctypes.byref(Tuning(*[int(tuning.get(k, 0)) for k, _t in Tuning._fields_]))
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        _check(L.dwt2d_batch_create(ctypes.byref(self._h), arr, len(self.jobs), SCHEMES[scheme], tun,
                                    ctypes.byref(ws)), "dwt2d_batch_create")
        self.workspace_bytes = ws.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.dwt2d_batch_destroy(h)
            self._h = None

    def info(self):
        """(kernel launches per launch(), warp work items in all)."""
        n, w = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().dwt2d_batch_info(self._h, ctypes.byref(n), ctypes.byref(w)), "batch_info")
        return n.value, w.value

    def workspace(self, device="cuda") -> torch.Tensor:
        # 256-byte aligned (the caching allocator's blocks are)
        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def staging_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().dwt2d_batch_staging_bytes(self._h, ctypes.byref(n)), "batch_staging_bytes")
        return n.value

    def upload(self, workspace: torch.Tensor, stream=None, staging: Optional[torch.Tensor] = None):
        """Write the descriptor tables into the workspace.  With `staging` (a
        pinned uint8 host tensor of at least staging_bytes(), kept alive until
        the stream has passed the upload) the copy is queued without waiting
        for the stream."""
        if staging is not None:
            _check(lib().dwt2d_batch_upload_staged(self._h, ctypes.c_void_p(workspace.data_ptr()),
                                                   ctypes.c_void_p(staging.data_ptr()),
                                                   staging.numel() * staging.element_size(),
                                                   _stream_ptr(stream)), "dwt2d_batch_upload_staged")
            return
        _check(lib().dwt2d_batch_upload(self._h, ctypes.c_void_p(workspace.data_ptr()),
                                        _stream_ptr(stream)), "dwt2d_batch_upload")

    def launch(self, workspace: torch.Tensor, stream=None):
        _check(lib().dwt2d_batch_launch(self._h, ctypes.c_void_p(workspace.data_ptr()),
                                        _stream_ptr(stream)), "dwt2d_batch_launch")

    def status(self, workspace: torch.Tensor, stream=None) -> int:
        return lib().dwt2d_workspace_status(ctypes.c_void_p(workspace.data_ptr()), _stream_ptr(stream))


def forward(x: torch.Tensor, levels: int, wavelet: str = "cdf97", scheme: str = "nonsep_reduced"):
    """One-shot forward transform of a device image."""
    return Plan(x.shape[0], x.shape[1], levels, wavelet, scheme, x.dtype).forward(x)


def inverse(c: torch.Tensor, levels: int, wavelet: str = "cdf97", scheme: str = "nonsep_reduced"):
    """One-shot inverse transform of device coefficients."""
    return Plan(c.shape[0], c.shape[1], levels, wavelet, scheme, c.dtype).inverse(c)
