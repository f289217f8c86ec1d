"""Serving loop: continuous batching of transform requests under a device
memory budget.

Requests (an image to transform forward, or Mallat coefficients to transform
back) are queued as they arrive.  Each call of Server.poll() retires the
batches whose kernels have finished and admits queued requests, in arrival
order, while their device memory fits the budget, into one new batch
(dwt2d_batch_*: a few kernel launches for any mix of sizes, level counts,
wavelets, storage types and directions).  Several batches are in flight at
once, each on its own stream of the executor's pool, so a batch admitted while
others run starts on the device at once and its kernels share the SMs with
theirs (the work of concurrently admitted requests overlaps), while the host
prepares the next batch.

Memory: a request reserves its output (kept resident on the device until the
client calls release()), its share of the batch workspace, and a device copy of
its input when the input is on the host or not pitched for the kernels.  A
request that can never fit is rejected at submit; the others wait (back
pressure) until earlier results are released.

Failures stay with the request that caused them: a malformed request is
rejected at submit, a refused allocation fails that request only, a cancelled
request is dropped (or its result discarded), and a slow input loader runs on a
worker thread while the queue moves on.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import contextlib
import itertools
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch

QUEUED, LOADING, RUNNING, DONE, FAILED, CANCELLED, REJECTED = (
    "queued", "loading", "running", "done", "failed", "cancelled", "rejected")

VALID_TYPES = {("cdf97", torch.float32), ("cdf97", torch.float16), ("cdf97", torch.bfloat16),
               ("legall53", torch.int32)}
TABLE_ENTRY_BYTES = 1024  # descriptor table bytes reserved per request and launch


@dataclass
class Request:
    """One transform: `data` (H, W) on the host or the device, or a `loader`
    that returns it (run on a worker thread)."""
    height: int
    width: int
    levels: int
    wavelet: str = "cdf97"
    dtype: torch.dtype = torch.float32
    inverse: bool = False
    data: Optional[torch.Tensor] = None
    loader: Optional[Callable[[], torch.Tensor]] = None


@dataclass
class Ticket:
    id: int
    request: Request
    state: str = QUEUED
    error: str = ""
    result: Optional[torch.Tensor] = None
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    reserved: int = 0          # bytes counted against the budget
    reserved_out: int = 0      # the part that stays resident with the result
    _src: Optional[torch.Tensor] = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    def finished(self) -> bool:
        return self.state in (DONE, FAILED, CANCELLED, REJECTED)


def validate(req: Request) -> str:
    """'' if the request is well formed, else the reason."""
    if not isinstance(req, Request):
        return "not a Request"
    for name in ("height", "width", "levels"):
        if not isinstance(getattr(req, name), int):
            return f"{name} must be an int"
    if not (1 <= req.height <= 65536 and 1 <= req.width <= 65536):
        return "height and width must be in 1..65536"
    if not 1 <= req.levels <= 16:
        return "levels must be in 1..16"
    if (req.wavelet, req.dtype) not in VALID_TYPES:
        return f"unsupported wavelet / storage type {req.wavelet} / {req.dtype}"
    if (req.data is None) == (req.loader is None):
        return "exactly one of data and loader is needed"
    if req.data is not None:
        return check_data(req, req.data)
    return ""


def check_data(req: Request, t) -> str:
    if not isinstance(t, torch.Tensor):
        return "data is not a tensor"
    if t.dim() != 2 or tuple(t.shape) != (req.height, req.width):
        return f"data shape {tuple(t.shape)} != ({req.height}, {req.width})"
    if t.dtype != req.dtype:
        return f"data dtype {t.dtype} != {req.dtype}"
    return ""


class GpuExecutor:
    """Runs batches with the library's batched kernels on a pool of streams.

    Batch k goes to stream k mod `streams`: the staging copies and the
    allocations of the batch being formed use that stream too, so every batch
    is ordered only after its own inputs, and batches on different streams run
    concurrently.  `timing=True` records CUDA events (with timestamps) around
    every batch, for measuring how they overlap."""

    def __init__(self, device="cuda", scheme="nonsep_reduced", tuning=None, stream=None,
                 streams: int = 4, timing: bool = False):
        from . import dwt2d as D

        self.D = D
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.scheme = scheme
        self.tuning = tuning
        if stream is not None:
            self.streams = [stream]
        else:
            self.streams = [torch.cuda.Stream(self.device) for _ in range(max(1, int(streams)))]
        self.timing = timing
        self._next = 0
        self._ws_cache = {}

    @property
    def stream(self):
        """The stream of the batch being formed."""
        return self.streams[self._next]

    def workspace_bytes(self, req: Request) -> int:
        # one plan per distinct transform description (admission runs per request)
        key = (req.height, req.width, req.levels, req.wavelet, req.dtype)
        n = self._ws_cache.get(key)
        if n is None:
            n = self.D.workspace_bytes(req.height, req.width, req.levels, req.wavelet, self.scheme,
                                       req.dtype)
            if len(self._ws_cache) > 65536:
                self._ws_cache.clear()
            self._ws_cache[key] = n
        return n

    def allocating(self):
        """Context for the allocations of the batch being formed: blocks owned
        by its stream (entered once per batch, not per allocation)."""
        return torch.cuda.stream(self.stream)

    def empty(self, h, w, dtype):
        # called inside allocating(): the current stream is the batch's
        return self.D.empty_image(h, w, dtype, self.device)

    def pitched(self, t: torch.Tensor) -> bool:
        es = t.element_size()
        return (t.device == self.device and t.stride(1) == 1 and (t.stride(0) * es) % 16 == 0
                and t.data_ptr() % 16 == 0)

    def copy_in(self, dst: torch.Tensor, src: torch.Tensor):
        with torch.cuda.stream(self.stream):
            dst.copy_(src, non_blocking=True)

    def launch(self, jobs):
        st = self.stream
        batch = self.D.Batch(jobs, self.scheme, self.tuning)
        with torch.cuda.stream(st):
            ws = batch.workspace(self.device)
        # pinned staging: queuing the table copy does not wait for the stream,
        # so this batch is queued while earlier ones still run; the handle
        # keeps the staging alive until the batch retires
        staging = torch.empty(max(batch.staging_bytes(), 16), dtype=torch.uint8, pin_memory=True)
        batch.upload(ws, stream=st, staging=staging)
        ev0 = None
        if self.timing:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(st)
        batch.launch(ws, stream=st)
        ev = torch.cuda.Event(enable_timing=self.timing)
        ev.record(st)
        self._next = (self._next + 1) % len(self.streams)
        return (batch, ws, ev, st, ev0, staging)

    def done(self, handle) -> bool:
        return handle[2].query()

    def status(self, handle) -> int:
        batch, ws, _ev, st = handle[:4]
        return batch.status(ws, stream=st)

    def span(self, handle):
        """(start, end) events of a batch launched with timing=True."""
        return handle[4], handle[2]


class Server:
    """Continuous batching under `budget_bytes` of device memory."""

    def __init__(self, budget_bytes: int = 40 << 30, executor=None, max_batch: int = 256,
                 max_inflight: int = 4, allocator: Optional[Callable] = None, loader_threads: int = 4,
                 clock: Callable[[], float] = time.perf_counter, track_finished: bool = False,
                 **executor_args):
        self.budget = int(budget_bytes)
        self.ex = executor if executor is not None else GpuExecutor(**executor_args)
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.alloc = allocator if allocator is not None else (lambda t, h, w, dt: self.ex.empty(h, w, dt))
        self.clock = clock
        self.in_use = 0
        self.peak = 0
        self.queue = collections.deque()  # of Ticket, arrival order
        self.inflight = []  # (handle, [tickets])
        # finished requests are counted, not kept (the client holds its tickets)
        self.counts = {DONE: 0, FAILED: 0, CANCELLED: 0, REJECTED: 0}
        # tickets finished since take_finished() (kept only when asked for)
        self._finished = collections.deque() if track_finished else None
        self.latencies: List[float] = []
        self._ids = itertools.count()
        self._lock = threading.Lock()
        self._loaders = cf.ThreadPoolExecutor(max_workers=loader_threads)
        self._loading = 0
        self.batches = 0
        self.batch_sizes: List[int] = []  # requests per launched batch
        self.retired_handles = []  # (handle, requests) of retired batches when keep_handles is set
        self.keep_handles = False

    # ---- client side
    def submit(self, req: Request, t_arrival: Optional[float] = None) -> Ticket:
        """Queue a request (latency counts from t_arrival, default now)."""
        t = Ticket(next(self._ids), req, t_submit=self.clock() if t_arrival is None else t_arrival)
        why = validate(req)
        if not why:
            try:
                t.reserved_out, tmp = self._need(req)
                t.reserved = t.reserved_out + tmp
            except Exception as e:  # a plan the library refuses
                why = f"plan refused: {e}"
        if not why and t.reserved > self.budget:
            why = f"needs {t.reserved} bytes, budget {self.budget}"
        if why:
            self._finish(t, REJECTED, why)
            return t
        if req.loader is not None:
            t.state = LOADING
            with self._lock:
                self._loading += 1
            self._loaders.submit(self._load, t)
        else:
            t._src = req.data
            with self._lock:
                self.queue.append(t)
        return t

    def cancel(self, t: Ticket) -> bool:
        """Drop a request that has not finished; its result (if the kernels are
        already running) is discarded when they end."""
        with self._lock:
            if t.finished():
                return False
            if t in self.queue:
                self.queue.remove(t)
            if t.state == RUNNING:
                t.state = CANCELLED  # retire() releases its memory
                t.error = "cancelled while running"
                return True
        self._finish(t, CANCELLED, "cancelled")
        return True

    def take_finished(self) -> List[Ticket]:
        """The tickets that finished (any final state) since the last call, in
        the order they finished: a client releases results without scanning
        every ticket it holds."""
        if self._finished is None:
            raise RuntimeError("Server(track_finished=True) keeps the finished tickets")
        out = []
        with self._lock:
            while self._finished:
                out.append(self._finished.popleft())
        return out

    def release(self, t: Ticket) -> None:
        """The client is done with a resident result: return its memory."""
        if t.result is not None:
            t.result = None
            self._unreserve(t)

    def poll(self) -> int:
        """Retire finished batches, then admit and launch one new batch.
        Returns the number of requests that finished in this call."""
        n = self.retire()
        if len(self.inflight) < self.max_inflight:
            self.admit_and_launch()
        return n

    def run_until_idle(self, timeout: float = 60.0, sleep: float = 0.0) -> bool:
        t_end = self.clock() + timeout
        while self.clock() < t_end:
            self.poll()
            with self._lock:
                busy = self.queue or self.inflight or self._loading
            if not busy:
                return True
            if sleep:
                time.sleep(sleep)
        return False

    def result(self, t: Ticket, timeout: float = 60.0) -> torch.Tensor:
        """Drive the loop until `t` finishes; its resident result, or raise
        with the reason it did not complete."""
        t_end = self.clock() + timeout
        while not t.finished():
            if self.clock() >= t_end:
                raise TimeoutError(f"request {t.id} still {t.state} after {timeout} s")
            self.poll()
        if t.state != DONE:
            raise RuntimeError(f"request {t.id} {t.state}: {t.error}")
        return t.result

    def stats(self) -> dict:
        with self._lock:
            lat = sorted(self.latencies)
            c = dict(self.counts)

        def q(p):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]

        sizes = self.batch_sizes
        return {"completed": c[DONE], "failed": c[FAILED], "cancelled": c[CANCELLED],
                "rejected": c[REJECTED], "p50_s": q(0.50), "p99_s": q(0.99),
                "max_s": lat[-1] if lat else None, "batches": self.batches,
                "requests_per_batch": (sum(sizes) / len(sizes)) if sizes else None,
                "max_batch_seen": max(sizes) if sizes else 0,
                "peak_bytes": self.peak, "budget_bytes": self.budget}

    def reset_stats(self):
        """Forget the counts and latencies so far (e.g. after a warm-up)."""
        with self._lock:
            self.counts = {k: 0 for k in self.counts}
            self.latencies = []
            self.batches = 0
            self.batch_sizes = []
            self.peak = self.in_use

    def close(self):
        self._loaders.shutdown(wait=True)

    # ---- internals
    def _need(self, req: Request):
        """(resident output bytes, bytes held only while the kernels run)."""
        es = req.dtype.itemsize
        img = req.height * ((req.width * es + 15) // 16 * 16)
        tmp = self.ex.workspace_bytes(req) + 4 * TABLE_ENTRY_BYTES
        data = req.data
        if data is None or not self.ex.pitched(data):
            tmp += img  # device copy of the input
        return img, tmp

    def _load(self, t: Ticket):
        try:
            data = t.request.loader()
            why = check_data(t.request, data)
        except Exception as e:  # the loader's own failure
            data, why = None, f"loader failed: {e!r}"
        with self._lock:
            self._loading -= 1
            if t.state != LOADING:  # cancelled meanwhile
                return
            if why:
                t.state = FAILED
            else:
                t._src = data
                t.state = QUEUED
                self.queue.append(t)
        if why:
            self._finish(t, FAILED, why)

    def _reserve(self, n: int):
        self.in_use += n
        self.peak = max(self.peak, self.in_use)

    def _unreserve(self, t: Ticket, keep_out: bool = False):
        with self._lock:
            keep = t.reserved_out if keep_out else 0
            self.in_use -= t.reserved - keep
            t.reserved = keep

    def _finish(self, t: Ticket, state: str, error: str = ""):
        t.state = state
        t.error = error
        t.t_done = self.clock()
        if state != DONE:
            t.result = None
            t._src = None
        with self._lock:  # loader threads finish failed loads concurrently
            self.counts[state] = self.counts.get(state, 0) + 1
            if state == DONE:
                self.latencies.append(t.t_done - t.t_submit)
            if self._finished is not None:
                self._finished.append(t)

    def admit_and_launch(self):
        picked = []
        with self._lock:
            q = self.queue
            # arrival order: nobody overtakes a request waiting for memory
            while q and len(picked) < self.max_batch and self.in_use + q[0].reserved <= self.budget:
                t = q.popleft()
                self._reserve(t.reserved)
                picked.append(t)
        if not picked:
            return
        jobs, ok = [], []
        ctx = getattr(self.ex, "allocating", None)
        with (ctx() if ctx is not None else contextlib.nullcontext()):
            self._allocate(picked, jobs, ok)
        if not ok:
            return
        try:
            handle = self.ex.launch(jobs)
        except Exception as e:
            for t in ok:
                self._unreserve(t)
                self._finish(t, FAILED, f"launch failed: {e!r}")
            return
        self.batches += 1
        self.batch_sizes.append(len(ok))
        self.inflight.append((handle, ok))

    def _allocate(self, picked, jobs, ok):
        """Inputs (copied in if not resident and pitched) and outputs of the
        picked requests; a refused allocation fails that request only."""
        for t in picked:
            r = t.request
            try:
                src = t._src
                if not self.ex.pitched(src):
                    dev = self.alloc(t, r.height, r.width, r.dtype)
                    self.ex.copy_in(dev, src)
                    src = dev
                out = self.alloc(t, r.height, r.width, r.dtype)
            except Exception as e:  # allocation refused: this request only
                self._unreserve(t)
                self._finish(t, FAILED, f"allocation refused: {e!r}")
                continue
            t._src = src
            t.result = out
            t.state = RUNNING
            t.t_start = self.clock()
            jobs.append((src, out, r.levels, r.wavelet, int(r.inverse)))
            ok.append(t)

    def retire(self) -> int:
        n = 0
        still = []
        for handle, tickets in self.inflight:
            if not self.ex.done(handle):
                still.append((handle, tickets))
                continue
            status = self.ex.status(handle)
            for t in tickets:
                t._src = None
                if t.state == CANCELLED:
                    t.result = None
                    self._unreserve(t)
                    self._finish(t, CANCELLED, t.error)
                elif status != 0:
                    self._unreserve(t)
                    self._finish(t, FAILED, f"kernel status {status}")
                else:
                    self._unreserve(t, keep_out=True)  # the output stays resident
                    self._finish(t, DONE)
                n += 1
            if self.keep_handles:
                self.retired_handles.append((handle, len(tickets)))
        self.inflight = still
        return n
