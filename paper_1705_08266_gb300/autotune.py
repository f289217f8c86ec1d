"""Autotuner for batched transforms (dwt2d_batch_*).

A batch's launch shape has six knobs (dwt2d_tuning): levels fused in an
image's first launch, levels fused per later launch (with the wavelet, this
sets the halo each strip and segment recomputes), warps targeted per SM (how
finely the rows are cut into warp segments, i.e. how many waves or queue
items), the smallest segment, the launch form (one launch per level group
and kind, or one persistent launch per direction and storage type over a
queue of work items) and the tile width (2 or 4 quadruple columns per lane:
128- or 256-pixel strips, the wider with half the halo overlap per pixel but
fewer strips to spread).  The best setting depends on the mix of
image sizes and level counts, so the tuner times a small set of candidates on
the batch itself (CUDA events, on the caller's buffers: the outputs are
overwritten) and keeps the fastest.  Results are cached in a JSON file keyed
by a signature of the batch (per job its storage type, wavelet, direction,
level count and the power-of-two class of each side) and by the device and
library build it was measured on.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Iterable, Optional

KNOBS = ("fuse_first", "fuse_max", "warps_per_sm", "min_segment", "persistent", "cols_per_lane")

CANDIDATES = [
    {"fuse_first": ff, "fuse_max": 2, "warps_per_sm": w, "min_segment": m, "persistent": 0,
     "cols_per_lane": 2}
    for ff in (2, 1) for w in (12, 24, 32, 48) for m in (2, 8)
] + [
    {"fuse_first": 2, "fuse_max": 2, "warps_per_sm": w, "min_segment": 2, "persistent": 0,
     "cols_per_lane": 4}
    for w in (12, 24, 48)
] + [
    {"fuse_first": 2, "fuse_max": 2, "warps_per_sm": w, "min_segment": m, "persistent": 1,
     "cols_per_lane": q}
    for q in (2, 4) for w in (24, 48, 96) for m in (2, 8)
]


def default_cache_path() -> str:
    return os.environ.get("DWT2D_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "dwt2d", "autotune.json")


def _size_class(n: int) -> int:
    return max(0, int(n).bit_length() - 1)


def signature(descs: Iterable) -> str:
    """descs: (height, width, levels, wavelet, dtype_name, inverse) per job.
    Order-independent; images whose sides fall in the same power-of-two class
    share a signature."""
    keys = sorted(f"{dt}/{wav}/{int(bool(inv))}/L{lv}/{_size_class(h)}x{_size_class(w)}"
                  for h, w, lv, wav, dt, inv in descs)
    counts = {}
    for k in keys:
        counts[k] = counts.get(k, 0) + 1
    text = ";".join(f"{k}*{c}" for k, c in sorted(counts.items()))
    return hashlib.sha1(text.encode()).hexdigest()[:16]


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(sig: str, measure: Callable[[dict], float], candidates=None, cache_path: Optional[str] = None,
         scheme: str = "nonsep_reduced", context: str = "") -> dict:
    """The fastest candidate for signature `sig` (cached).  measure(tuning)
    returns milliseconds, or None when the candidate does not apply.
    `context` (the device and library build) is part of the cache key, so a
    tuning measured elsewhere is not reused."""
    key = f"{scheme}:{context}:{sig}" if context else f"{scheme}:{sig}"
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache and "tuning" in cache[key]:
        return dict(cache[key]["tuning"])
    best, best_ms, tried = None, float("inf"), []
    for cand in candidates or CANDIDATES:
        ms = measure(dict(cand))
        if ms is None:
            continue
        tried.append({"tuning": cand, "ms": ms})
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    if best is None:
        raise RuntimeError("no tuning candidate applies to this batch")
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"tuning": best, "ms": best_ms, "tried": tried}
        save_cache(cache_path, cache)
    return best


def tune(jobs, scheme: str = "nonsep_reduced", cache_path: Optional[str] = None, iters: int = 5,
         warmup: int = 2, stream=None, candidates=None) -> dict:
    """Time the candidates on `jobs` (as for dwt2d.Batch) and return the best
    tuning dict.  Overwrites the jobs' outputs."""
    import torch

    from . import dwt2d as D

    descs = [(s.shape[0], s.shape[1], lv, wav, str(s.dtype).replace("torch.", ""), inv)
             for s, _d, lv, wav, inv in jobs]
    st = stream if stream is not None else torch.cuda.current_stream()

    def measure(tuning):
        try:
            b = D.Batch(jobs, scheme, tuning)
        except D.DwtError:
            return None
        ws = b.workspace(jobs[0][0].device)
        b.upload(ws, stream=st)
        for _ in range(warmup):
            b.launch(ws, stream=st)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(iters):
            b.launch(ws, stream=st)
        e1.record(st)
        e1.synchronize()
        # a candidate whose kernels recorded an error (a wait that gave up,
        # a caught store) is not a valid timing: reject it
        if b.status(ws, stream=st) != 0:
            return None
        return e0.elapsed_time(e1) / iters

    dev = jobs[0][0].device
    props = torch.cuda.get_device_properties(dev)
    st_lib = os.stat(D.LIB_PATH)
    context = f"{props.name}/{props.multi_processor_count}sm/lib{st_lib.st_size}.{st_lib.st_mtime_ns}"
    return pick(signature(descs), measure, candidates, cache_path, scheme, context)
