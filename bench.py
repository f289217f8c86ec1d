#!/usr/bin/env python
"""Benchmark: multilevel 2-D DWT by non-separable lifting on GB300.

Workload (one step): CDF 9/7 forward transform of one 8192 x 8192 float32
image, 5 levels, non-separable lifting in its reduced form, through the C ABI
(dwt2d_forward), input resident in HBM.  The image (256 MiB) and the
coefficients (256 MiB) are both larger than L2, so no flush is needed between
steps.  Also measured in the same run and reported under "variants": every
scheme (separable, non-separable, reduced, and their multipass forms) forward
and inverse, and reversible LeGall 5/3 int32.

Prints ONE JSON line.  `--impl reference` times the FP64 oracle on the host
cores instead (a bounded sample of the same workload).
Multi-GPU: one process per GPU (torchrun); every rank transforms its own image
(replicas, no collective on the data path); value = all ranks' pixels / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
HBM_NOMINAL = 7900.0  # GB/s, GB300 HBM3e nominal
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "Gpixel/s and % HBM roofline, CDF 9/7 fwd 8192² 5 levels, non-sep vs separable"
UNIT = "Gpixel/s"
H = W = 8192
LEVELS = 5
HEADLINE_SCHEME = "nonsep_reduced"
WORKLOAD = ("CDF 9/7 forward, 8192x8192 float32, 5 levels, non-separable lifting (reduced form), "
            "input resident in HBM")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inverse-only", action="store_true",
                    help="time only the inverse of the headline workload (for profiling its kernels)")
    ap.add_argument("--size", type=int, default=8192,
                    help="image side (profiling runs use a smaller case; the metric is 8192)")
    ap.add_argument("--scheme", default=None,
                    help="time the workload with another lifting scheme (profiling runs; the metric "
                         "is non-separable reduced)")
    return ap.parse_args()


_REDUCE_DEVICE = "cuda"


def dist_setup():
    """One process per GPU (torchrun env); NCCL on GPUs, gloo without (host tests)."""
    global _REDUCE_DEVICE
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            _REDUCE_DEVICE = "cuda"
        else:
            dist.init_process_group("gloo")
            _REDUCE_DEVICE = "cpu"
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=_REDUCE_DEVICE)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash() -> str:
    """Short hash of the kernel sources (a profile taken on other sources is stale)."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1705_08266_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary.

    The summary line reads `traffic_bytes_per_launch: <bytes> <kernel tag> src=<hash>`;
    None if absent, for another kernel, or taken on different kernel sources.
    """
    path = os.path.join(ROOT, "profiles", "fwd_fused_cdf97_8192x8192_l5.md")
    try:
        with open(path) as f:
            for line in f:
                if not line.startswith("traffic_bytes_per_launch:"):
                    continue
                parts = line.split(":", 1)[1].split()
                if len(parts) >= 3 and parts[1] == kernel_tag and parts[2] == "src=" + kernel_source_hash():
                    return float(parts[0])
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled in the background."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.f = open(self.path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, t0: float, t1: float):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
                except (ValueError, IndexError):
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05] or rows[-3:]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def time_calls(fn, iters: int, stream) -> float:
    """Mean ms per call of fn() on `stream`, CUDA events, after the caller's warm-up."""
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(iters):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / iters


def cpu_baseline(seconds_hint: float = 15.0):
    """The FP64 oracle timed on this host on a bounded sample of the workload."""
    from oracle import lifting as L
    from paper_1705_08266_gb300 import synth

    n = H  # the full workload image: about 10-30 s of single-thread FP64 work
    x = synth.gradient_noise(n, n, synth.SEED_LARGE)
    t0 = time.perf_counter()
    runs = 0
    while True:
        L.forward(x, LEVELS, "cdf97")
        runs += 1
        if time.perf_counter() - t0 > seconds_hint or runs >= 3:
            break
    dt = (time.perf_counter() - t0) / runs
    return {"value": round(n * n / dt / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"CDF 9/7 forward, {n}x{n} of the same gradient+noise recipe, {LEVELS} levels, "
                      f"FP64 numpy separable lifting, single thread, mean of {runs} run(s)"}


_ORACLE_WORKER = """
import sys, time
from oracle import lifting as L
from paper_1705_08266_gb300 import synth
n, levels, runs, seed, start = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), float(sys.argv[5])
x = synth.gradient_noise(n, n, seed)
while time.time() < start:
    time.sleep(0.005)
t0 = time.time()
for _ in range(runs):
    L.forward(x, levels, "cdf97")
print(t0, time.time())
"""


def cpu_baseline_all_cores(n: int = 2048, runs: int = 3):
    """The unmodified FP64 oracle in one process per host core, each on its
    own n x n image of the workload's recipe, started together: the host's
    throughput with every core busy (memory bandwidth shared)."""
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    start = time.time() + 3.0 + 0.05 * cores
    procs = [subprocess.Popen([sys.executable, "-c", _ORACLE_WORKER, str(n), str(LEVELS), str(runs),
                               str(1000 + i), repr(start)], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for i in range(cores)]
    spans = []
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        if pr.returncode != 0:
            raise RuntimeError(f"oracle worker failed: {err[-500:]}")
        spans.append(tuple(float(v) for v in out.split()))
    wall = max(b for _, b in spans) - min(a for a, _ in spans)
    return {"value": round(cores * runs * n * n / wall / 1e9, 6), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} processes (one per host core), each {runs} CDF 9/7 forward transforms of "
                      f"its own {n}x{n} image of the same recipe, {LEVELS} levels, FP64 numpy; "
                      f"rate over the common wall time"}


def run_reference(args, ws, rank):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only."""
    if rank != 0:
        return
    from oracle import lifting as L
    from paper_1705_08266_gb300 import synth

    n = 2048  # 1/16 of the workload's pixels per step, so K steps end within minutes
    x = synth.gradient_noise(n, n, synth.SEED_LARGE)
    for _ in range(min(max(args.warmup, 0), 3)):
        L.forward(x, LEVELS, "cdf97")
    steps = max(args.steps, 1)
    budget = 150.0
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        L.forward(x, LEVELS, "cdf97")
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = (time.perf_counter() - t0) / done
    v = n * n / dt / 1e9
    sample = (f"CDF 9/7 forward of a {n}x{n} crop-size image of the same recipe, {LEVELS} levels, "
              f"FP64 numpy oracle, single thread; {done} timed step(s)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": args.gpus,
        "steps": done, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "image": [8192, 8192], "levels": LEVELS, "wavelet": "cdf97",
                   "scheme": HEADLINE_SCHEME,
                   "sample": f"each step transforms a {n}x{n} image of the same recipe (1/16 of the "
                             f"pixels); the rate is per pixel",
                   "parallelism": "host, 1 thread"},
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    global H, W, HEADLINE_SCHEME
    args = parse()
    H = W = args.size
    if args.scheme:
        HEADLINE_SCHEME = args.scheme
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    from paper_1705_08266_gb300 import dwt2d as D
    from paper_1705_08266_gb300 import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.inverse_only:
        inverse_only(args, D, synth, dev)
        return
    x_h = synth.gradient_noise(H, W, synth.SEED_LARGE)
    x = D.empty_image(H, W, torch.float32, dev)
    x.copy_(torch.from_numpy(x_h))
    dst = D.empty_image(H, W, torch.float32, dev)
    plan = D.Plan(H, W, LEVELS, "cdf97", HEADLINE_SCHEME)
    wsb = plan.workspace(dev)
    launches, fused = plan.info()
    shapes = plan.launch_info()  # (levels fused, columns per lane, warps) per launch
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()

    fwd = lambda: plan.forward(x, dst, wsb, stream=stream)  # noqa: E731
    for _ in range(max(args.warmup, 3)):
        fwd()
    torch.cuda.synchronize()

    # Two passes of K steps on the launching stream.  Pass 1 (plain steps) gives
    # the step time: the launches of a step run with programmatic stream
    # serialization, and an event recorded between two launches would suspend
    # that overlap.  Pass 2 brackets launch 0 (the dominant kernel) of every
    # step with events and gives that kernel's duration.
    K = max(args.steps, 1)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for row in evs:  # torch creates an event on its first record; the library re-records it
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    start.record(stream)
    for k in range(K):
        fwd()
    end.record(stream)
    end.synchronize()
    torch.cuda.synchronize()
    barrier(ws)
    for k in range(K):
        plan.set_launch_events(evs[k])
        fwd()
    torch.cuda.synchronize()
    t1 = time.time()
    barrier(ws)
    plan.set_launch_events(None)
    clocks = sampler.stop(t0, t1)
    ms_local = start.elapsed_time(end) / K
    ms = max_over_ranks(ws, ms_local)
    assert plan.status(wsb) == 0, "kernel reported a timeout"

    launch_ms = [statistics.mean(evs[k][0].elapsed_time(evs[k][1]) for k in range(K))]
    dom = 0
    value = ws * H * W / (ms / 1e3) / 1e9

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # dominant launch: fused levels 1..fused[0] of the full image: reads the image once and
    # writes every coefficient of those levels (details + LL) once = 2 * 4 * H * W bytes
    alg_bytes_dom = 2 * 4 * H * W if dom == 0 else None
    strict_bytes = 2 * 4 * H * W  # the whole transform: image read once, coefficients written once
    traffic = profiled_traffic(f"fused{fused[0]}") if H == 8192 else None
    achieved = alg_bytes_dom / (launch_ms[dom] / 1e3) / 1e9 if alg_bytes_dom else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 4) if achieved else None,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": f"fwd_fused_kernel<float, {HEADLINE_SCHEME}, {shapes[0][0]} levels, "
                          f"{shapes[0][1]} columns/lane> (launch {dom} of {launches}, {shapes[0][2]} warps)",
                "kernel_ms": round(launch_ms[dom], 5),
                "kernel_timing": "CUDA events around launch 0 of each step, second pass of K steps",
                "alg_bytes_per_launch": alg_bytes_dom,
                "whole_step": {"strict_bytes": strict_bytes,
                               "achieved": round(strict_bytes / (ms / 1e3) / 1e9, 1),
                               "frac": round(strict_bytes / (ms / 1e3) / 1e9 / hbm, 4),
                               "frac_of_nominal": round(strict_bytes / (ms / 1e3) / 1e9 / HBM_NOMINAL, 4)},
                # the same fractions against the nominal HBM3e bandwidth (context only)
                "nominal_peak": HBM_NOMINAL,
                "frac_of_nominal": round(achieved / HBM_NOMINAL, 4) if achieved else None}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "image": [H, W], "levels": LEVELS, "wavelet": "cdf97", "scheme": HEADLINE_SCHEME,
                   "launches_per_step": launches, "fused_levels_per_launch": fused,
                   "launch_shapes": [{"levels": f, "cols_per_lane": q, "warps": w} for f, q, w in shapes],
                   "l2": "inputs and outputs (256 MiB each) larger than L2; no flush",
                   "parallelism": f"replicas x{ws}"},
        # pass 1 (step time) and pass 2 (launch 0 bracketed by events)
        "gpu_launches": 2 * launches * K,
        "roofline": roofline,
        "clocks": clocks,
    }

    if not args.no_variants:
        out["variants"] = variants(D, synth, dev, stream, x, dst)
        out["precision_16384x16384_l6"] = precision_variants(D, synth, dev, stream)
        out["batch_256_mixed"] = batch_variants(D, synth, dev, stream)
        out["serving_poisson"] = serving_variant(D, synth, dev)
        # the same recipe at ten times the arrival rate: batches fill up
        out["serving_poisson_10x"] = serving_variant(D, synth, dev, seconds=3.0, rate=20000.0)

    if args.no_e2e:
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    # end to end through the host-buffer entry point (copies inside the timed region)
    hs = torch.from_numpy(x_h).pin_memory()
    hd = torch.empty_like(hs).pin_memory()
    din = D.empty_image(H, W, torch.float32, dev)
    for _ in range(2):
        plan.forward_host(hs, hd, din, dst, wsb, stream=stream)
    n_e2e = min(K, 30)
    barrier(ws)
    te = time.perf_counter()
    for _ in range(n_e2e):
        plan.forward_host(hs, hd, din, dst, wsb, stream=stream)
    e2e_s = max_over_ranks(ws, (time.perf_counter() - te) / n_e2e)
    out["e2e"] = {"value": round(ws * H * W / e2e_s / 1e9, 3), "unit": UNIT,
                  "h2d_bytes_per_step": 4 * H * W, "d2h_bytes_per_step": 4 * H * W,
                  "steps": n_e2e, "api": "dwt2d_forward_host (pinned host buffers)"}
    # a pipelined host-buffer call (1024 rows or more): one launch of the first
    # level group per row band (at 8192^2 every band completes some of its row
    # segments) plus one per later group; below that the plain launches
    bands = 8  # the default dwt2d_plan_options.host_bands
    per_call = bands + launches - 1 if H >= 1024 else launches
    out["e2e"]["gpu_launches_per_step"] = per_call
    out["gpu_launches"] += n_e2e * per_call

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def inverse_only(args, D, synth, dev):
    """The inverse of the headline workload alone: warm-up, then K timed steps
    (one line of JSON with the per-step time), for profiling its launches."""
    x = D.empty_image(H, W, torch.float32, dev)
    x.copy_(torch.from_numpy(synth.gradient_noise(H, W, synth.SEED_LARGE)))
    c = D.empty_image(H, W, torch.float32, dev)
    y = D.empty_image(H, W, torch.float32, dev)
    plan = D.Plan(H, W, LEVELS, "cdf97", HEADLINE_SCHEME)
    wsb = plan.workspace(dev)
    stream = torch.cuda.Stream(dev)
    plan.forward(x, c, wsb, stream=stream)
    inv = lambda: plan.inverse(c, y, wsb, stream=stream)  # noqa: E731
    for _ in range(max(args.warmup, 3)):
        inv()
    K = max(args.steps, 1)
    ms = time_calls(inv, K, stream)
    assert plan.status(wsb) == 0, "kernel reported a timeout"
    print(json.dumps({"inverse_ms_per_step": round(ms, 5), "image": [H, W], "levels": LEVELS,
                      "scheme": HEADLINE_SCHEME, "launches_per_step": plan.info()[0], "steps": K}),
          flush=True)


def variants(D, synth, dev, stream, x, dst):
    """Every scheme forward / inverse (9/7) and 5/3, same image size."""
    res = {}
    iters, warm = 20, 3
    strict = 2 * 4 * H * W
    hbm = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    c = D.empty_image(H, W, torch.float32, dev)
    for scheme in D.SCHEMES:  # CDF 9/7: every scheme, incl. the separable convolution
        plan = D.Plan(H, W, LEVELS, "cdf97", scheme)
        wsb = plan.workspace(dev)
        plan.forward(x, c, wsb, stream=stream)
        for direction, fn in (("fwd", lambda: plan.forward(x, c, wsb, stream=stream)),
                              ("inv", lambda: plan.inverse(c, dst, wsb, stream=stream))):
            for _ in range(warm):
                fn()
            ms = time_calls(fn, iters, stream)
            res[f"cdf97_f32_{scheme}_{direction}"] = {
                "ms": round(ms, 5), "gpx_s": round(H * W / ms / 1e6, 2),
                "strict_frac": round(strict / (ms / 1e3) / 1e9 / hbm, 4),
                "launches": plan.info()[0]}
        del wsb
    xi = D.empty_image(H, W, torch.int32, dev)
    xi.copy_(torch.from_numpy(synth.uniform_int(H, W, synth.SEED_LARGE)))
    ci = D.empty_image(H, W, torch.int32, dev)
    yi = D.empty_image(H, W, torch.int32, dev)
    for scheme in ("separable", "nonsep", "separable_multipass", "nonsep_multipass"):
        plan = D.Plan(H, W, LEVELS, "legall53", scheme)
        wsb = plan.workspace(dev)
        plan.forward(xi, ci, wsb, stream=stream)
        for direction, fn in (("fwd", lambda: plan.forward(xi, ci, wsb, stream=stream)),
                              ("inv", lambda: plan.inverse(ci, yi, wsb, stream=stream))):
            for _ in range(warm):
                fn()
            ms = time_calls(fn, iters, stream)
            res[f"legall53_i32_{scheme}_{direction}"] = {
                "ms": round(ms, 5), "gpx_s": round(H * W / ms / 1e6, 2),
                "strict_frac": round(strict / (ms / 1e3) / 1e9 / hbm, 4),
                "launches": plan.info()[0]}
    return res


def band_rects(h: int, w: int, levels: int):
    """{"L<l> <band>": (r0, r1, c0, c1)} of the Mallat layout (LL only at the last level)."""
    out = {}
    for lvl in range(1, levels + 1):
        he, we = (h + 1) // 2, (w + 1) // 2
        out[f"L{lvl} HL"] = (0, he, we, w)
        out[f"L{lvl} LH"] = (he, h, 0, we)
        out[f"L{lvl} HH"] = (he, h, we, w)
        if lvl == levels:
            out[f"L{lvl} LL"] = (0, he, 0, we)
        h, w = he, we
    return out


def precision_variants(D, synth, dev, stream):
    """CDF 9/7 non-separable reduced, 16384^2, 6 levels: FP32 vs FP16 vs BF16 storage.

    Error of the 16-bit coefficients per band and level, as a fraction of
    max|x|, over every coefficient: against the FP32-storage transform of the
    same dequantised 16-bit image (the parity tests hold that transform within
    1e-5 max|x| of the FP64 reference per level, so the figure is the error
    against FP64 to within 1e-5; the sampled FP64 comparison is in the GPU
    tests)."""
    n, levels, iters, warm = 16384, 6, 10, 3
    hbm = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    x32 = synth.gradient_noise(n, n, synth.SEED_PRECISION)
    scale = float(np.max(np.abs(x32)))
    rects = band_rects(n, n, levels)
    res = {}
    for name, dt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
        xs = torch.from_numpy(x32 if dt == torch.float32 else x32 / scale).to(dt)
        x = D.empty_image(n, n, dt, dev)
        x.copy_(xs)
        c = D.empty_image(n, n, dt, dev)
        y = D.empty_image(n, n, dt, dev)
        plan = D.Plan(n, n, levels, "cdf97", "nonsep_reduced", dt)
        wsb = plan.workspace(dev)
        sc = 1.0 if dt == torch.float32 else scale
        plan.forward(x, c, wsb, scale=sc, stream=stream)
        for direction, fn in (("fwd", lambda: plan.forward(x, c, wsb, scale=sc, stream=stream)),
                              ("inv", lambda: plan.inverse(c, y, wsb, scale=sc, stream=stream))):
            for _ in range(warm):
                fn()
            ms = time_calls(fn, iters, stream)
            strict = 2 * x.element_size() * n * n
            res[f"{name}_{direction}"] = {"ms": round(ms, 4), "gpx_s": round(n * n / ms / 1e6, 1),
                                          "strict_frac": round(strict / (ms / 1e3) / 1e9 / hbm, 4)}
        if dt != torch.float32:
            # reference: the FP32-storage transform of the dequantised 16-bit image
            plan32 = D.Plan(n, n, levels, "cdf97", "nonsep_reduced", torch.float32)
            xd = D.empty_image(n, n, torch.float32, dev)
            with torch.cuda.stream(stream):  # every step of the comparison on the one stream
                xd.copy_(x.to(torch.float32) * scale)
                r32 = plan32.forward(xd, stream=stream)
                plan.forward(x, c, wsb, scale=sc, stream=stream)
            torch.cuda.synchronize()
            maxabs = float(xd.abs().max())
            errs = {}
            for key, (r0, r1, c0, c1) in rects.items():
                d = (c[r0:r1, c0:c1].to(torch.float64) * scale - r32[r0:r1, c0:c1].to(torch.float64))
                errs[key] = round(float(d.abs().max()) / maxabs, 7) if d.numel() else 0.0
            tol = 2e-3 if dt == torch.float16 else 1.6e-2
            res[f"{name}_fwd"]["max_err_over_maxabs"] = errs
            res[f"{name}_fwd"]["tolerance"] = tol
            res[f"{name}_fwd"]["within_tolerance"] = max(errs.values()) <= tol
            res[f"{name}_fwd"]["error_reference"] = ("FP32-storage GPU transform of the dequantised "
                                                     "16-bit image (itself within 1e-5 max|x| of FP64)")
            del plan32, xd, r32
        del x, c, y, wsb
        torch.cuda.empty_cache()
    return res


def batch_variants(D, synth, dev, stream):
    """Batched forward transforms: 256 images, H and W uniform on 65..4096,
    levels uniform on 1..6, 75% CDF 9/7 float32 and 25% LeGall 5/3 int32
    (seed 2017).  One batch (eager and replayed from a CUDA graph, in the
    table and the persistent form and with the autotuned launch shape) against
    one dwt2d_forward call per image (eager and captured in one CUDA graph)."""
    from paper_1705_08266_gb300 import autotune

    rng = np.random.default_rng(2017)
    iters, warm = 10, 3
    base = {"cdf97": torch.from_numpy(synth.gradient_noise(4096, 4096, 2017)).to(dev),
            "legall53": torch.from_numpy(synth.uniform_int(4096, 4096, 2017)).to(dev)}
    jobs, plans, wss = [], [], []
    px = 0
    for i in range(256):
        h, w = int(rng.integers(65, 4097)), int(rng.integers(65, 4097))
        lv = int(rng.integers(1, 7))
        wav = "cdf97" if rng.random() < 0.75 else "legall53"
        dt = torch.float32 if wav == "cdf97" else torch.int32
        x = D.empty_image(h, w, dt, dev)
        x.copy_(base[wav][:h, :w])
        jobs.append((x, D.empty_image(h, w, dt, dev), lv, wav, 0))
        plans.append(D.Plan(h, w, lv, wav))
        wss.append(plans[-1].workspace(dev))
        px += h * w
    batch = D.Batch(jobs)
    bws = batch.workspace(dev)
    batch.upload(bws, stream=stream)
    res = {"workload": "256 images, H,W ~ U{65..4096}, levels ~ U{1..6}, 75% CDF 9/7 f32 / "
                       "25% LeGall 5/3 i32, forward, non-separable reduced lifting, seed 2017",
           "images": 256, "pixels": px, "batch_launches": batch.info()[0],
           "per_image_launches": sum(p.info()[0] for p in plans)}

    def per_image():
        for p, (s_, d_, _lv, _w, _i), w_ in zip(plans, jobs, wss):
            p.forward(s_, d_, w_, stream=stream)

    def batched():
        batch.launch(bws, stream=stream)

    for name, fn in (("per_image_eager", per_image), ("batch_eager", batched)):
        for _ in range(warm):
            fn()
        ms = time_calls(fn, iters, stream)
        res[name] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1)}
    for name, fn in (("per_image_graph", per_image), ("batch_graph", batched)):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        with torch.cuda.stream(stream):  # replay on the timed stream
            for _ in range(warm):
                g.replay()
            ms = time_calls(g.replay, iters, stream)
        res[name] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1)}
        del g
    # the persistent form: one launch per direction and storage type over a
    # queue of every level group's work items
    pb = D.Batch(jobs, tuning={"persistent": 1})
    pws = pb.workspace(dev)
    pb.upload(pws, stream=stream)
    fn = lambda: pb.launch(pws, stream=stream)  # noqa: E731
    for _ in range(warm):
        fn()
    ms = time_calls(fn, iters, stream)
    res["batch_persistent_eager"] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1),
                                     "launches": pb.info()[0]}
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    with torch.cuda.stream(stream):
        for _ in range(warm):
            g.replay()
        ms = time_calls(g.replay, iters, stream)
    res["batch_persistent_graph"] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1)}
    assert pb.status(pws, stream=stream) == 0
    del g
    with tempfile.TemporaryDirectory() as tmp:
        best = autotune.tune(jobs, cache_path=os.path.join(tmp, "tune.json"), stream=stream)
    tb = D.Batch(jobs, tuning=best)
    tws = tb.workspace(dev)
    tb.upload(tws, stream=stream)
    fn = lambda: tb.launch(tws, stream=stream)  # noqa: E731
    for _ in range(warm):
        fn()
    ms = time_calls(fn, iters, stream)
    res["batch_autotuned"] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1), "tuning": best,
                              "launches": tb.info()[0]}
    # the autotuned batch captured in a CUDA graph (its launches, and the
    # queue-counter memset of the persistent form, replayed as one graph)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    with torch.cuda.stream(stream):
        for _ in range(warm):
            g.replay()
        ms = time_calls(g.replay, iters, stream)
    res["batch_autotuned_graph"] = {"ms": round(ms, 4), "gpx_s": round(px / ms / 1e6, 1)}
    assert tb.status(tws, stream=stream) == 0
    del g
    torch.cuda.synchronize()
    return res


def serving_variant(D, synth, dev, seconds: float = 10.0, rate: float = 2000.0):
    """Open-loop serving: Poisson arrivals at `rate` per second for `seconds`;
    long side s log-uniform on [64, 8192], aspect a ~ U[1, 4] (short side
    max(16, s / a), orientation random), 70% forward / 30% inverse, levels
    U{1..6}, 50% CDF 9/7 float16 / 50% LeGall 5/3 int32, 40 GB budget, seed
    2026.  Inputs are device-resident views of one synthetic image per type;
    each result is released as soon as it completes.  Latency runs from the
    arrival time to the host seeing the batch's completion event."""
    from paper_1705_08266_gb300 import serve as S

    rng = np.random.default_rng(2026)
    n = int(rng.poisson(rate * seconds))
    arrivals = np.sort(rng.uniform(0.0, seconds, n))
    base = {torch.float16: torch.from_numpy(synth.gradient_noise(8192, 8192, 2026) / 256.0).to(
                dev, torch.float16),
            torch.int32: torch.from_numpy(synth.uniform_int(8192, 8192, 2026)).to(dev)}
    reqs, px = [], 0
    for _ in range(n):
        s_ = float(np.exp(rng.uniform(np.log(64), np.log(8192))))
        a = float(rng.uniform(1, 4))
        lg, sh = int(s_), max(16, int(s_ / a))
        h, w = (lg, sh) if rng.random() < 0.5 else (sh, lg)
        inv = bool(rng.random() < 0.3)
        lv = int(rng.integers(1, 7))
        wav, dt = ("cdf97", torch.float16) if rng.random() < 0.5 else ("legall53", torch.int32)
        reqs.append(S.Request(h, w, lv, wav, dt, inv, data=base[dt][:h, :w]))
        px += h * w
    import gc

    srv = S.Server(budget_bytes=40 << 30, device=dev, track_finished=True)
    # warm-up: module loading and kernel attributes outside the measurement
    warm = [srv.submit(r) for r in reqs[:32]]
    srv.run_until_idle(60)
    for t in warm:
        srv.release(t)
    srv.take_finished()
    srv.reset_stats()
    # no collector pauses inside the timed loop (a serving process would tune it too)
    gc.collect()
    gc.disable()
    t0 = time.perf_counter()
    i = 0
    outstanding = 0
    while i < n or outstanding:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            srv.submit(reqs[i], t_arrival=t0 + arrivals[i])
            outstanding += 1
            i += 1
        srv.poll()
        for t in srv.take_finished():  # release each result as soon as it completes
            srv.release(t)
            outstanding -= 1
    wall = time.perf_counter() - t0
    gc.enable()
    st = srv.stats()
    srv.close()
    return {"workload": f"Poisson {rate:.0f}/s for {seconds:g} s; s log-uniform [64, 8192], aspect U[1,4], "
                        "short side >= 16; 70% fwd / 30% inv; levels U{1..6}; 50% CDF 9/7 f16 / 50% "
                        "LeGall 5/3 i32; 40 GB budget; seed 2026; device-resident inputs; "
                        f"{len(srv.ex.streams)} streams",
            "requests": n, "pixels": px, "completed": st["completed"], "rejected": st["rejected"],
            "failed": st["failed"], "wall_s": round(wall, 3),
            "p50_ms": round(st["p50_s"] * 1e3, 3) if st["p50_s"] is not None else None,
            "p99_ms": round(st["p99_s"] * 1e3, 3) if st["p99_s"] is not None else None,
            "max_ms": round(st["max_s"] * 1e3, 3) if st["max_s"] is not None else None,
            "requests_per_s": round(st["completed"] / wall, 1), "gpx_s": round(px / wall / 1e9, 3),
            "batches": st["batches"],
            "requests_per_batch": round(st["requests_per_batch"], 2) if st["requests_per_batch"] else None,
            "max_requests_per_batch": st["max_batch_seen"],
            "peak_reserved_gb": round(st["peak_bytes"] / 1e9, 3)}


if __name__ == "__main__":
    main()
