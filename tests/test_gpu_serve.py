"""Serving loop on the GPU: a request's result alone equals its result in a
mixed stream (bit for bit) and the single-image call's; resident coefficients
feed inverse requests; host inputs are staged; a Poisson stream under a small
budget completes with the peak reservation inside the budget."""
import time

import numpy as np
import pytest
import torch

from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import serve as S
from paper_1705_08266_gb300 import synth
from tests.parity_util import TOL_F32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    D.lib()


def _data(h, w, wav, dt, seed):
    x = synth.image(wav, h, w, seed)
    if dt in (torch.float16, torch.bfloat16):
        x = x / max(1.0, float(np.abs(x).max()))
    t = D.empty_image(h, w, dt)
    t.copy_(torch.from_numpy(x).to(dt))
    return t


def _random_request(rng, seed):
    s = float(np.exp(rng.uniform(np.log(16), np.log(1500))))
    a = rng.uniform(1, 4)
    long_, short = int(s), max(16, int(s / a))
    h, w = (long_, short) if rng.random() < 0.5 else (short, long_)
    wav, dt = (("cdf97", torch.float16), ("legall53", torch.int32), ("cdf97", torch.float32))[
        int(rng.integers(0, 3))]
    return S.Request(h, w, int(rng.integers(1, 7)), wav, dt, bool(rng.random() < 0.3),
                     data=_data(h, w, wav, dt, seed))


TARGETS = [
    S.Request(300, 517, 4, "cdf97", torch.float16, False),
    S.Request(257, 96, 6, "legall53", torch.int32, True),
    S.Request(1030, 770, 5, "cdf97", torch.float32, False),
    S.Request(16, 900, 6, "cdf97", torch.float32, True),
]


def _with_data(r, seed):
    return S.Request(r.height, r.width, r.levels, r.wavelet, r.dtype, r.inverse,
                     data=_data(r.height, r.width, r.wavelet, r.dtype, seed))


def test_result_alone_equals_result_in_the_mix():
    targets = [_with_data(r, 50 + i) for i, r in enumerate(TARGETS)]
    alone = []
    for r in targets:
        srv = S.Server(budget_bytes=8 << 30)
        t = srv.submit(r)
        assert srv.run_until_idle(30)
        assert t.state == S.DONE, t.error
        alone.append(t.result.cpu())
    rng = np.random.default_rng(2026)
    mix = [_random_request(rng, 1000 + i) for i in range(60)]
    order = list(range(len(mix) + len(targets)))
    rng.shuffle(order)
    srv = S.Server(budget_bytes=8 << 30)
    tickets = {}
    for k in order:
        r = targets[k - len(mix)] if k >= len(mix) else mix[k]
        tickets[k] = srv.submit(r)
        if k % 7 == 0:
            srv.poll()
    assert srv.run_until_idle(60)
    assert srv.stats()["completed"] == len(order)
    for i, r in enumerate(targets):
        got = tickets[len(mix) + i].result.cpu()
        assert torch.equal(got, alone[i]), f"target {i} differs in the mix"
        plan = D.Plan(r.height, r.width, r.levels, r.wavelet, "nonsep_reduced", r.dtype)
        ref = plan.inverse(r.data) if r.inverse else plan.forward(r.data)
        assert torch.equal(got, ref.cpu()), f"target {i} differs from the single-image call"


def test_resident_coefficients_feed_the_inverse():
    srv = S.Server(budget_bytes=4 << 30)
    x = _data(700, 901, "cdf97", torch.float32, 3)
    xi = _data(333, 444, "legall53", torch.int32, 4)
    f = srv.submit(S.Request(700, 901, 5, data=x))
    fi = srv.submit(S.Request(333, 444, 3, "legall53", torch.int32, data=xi))
    assert srv.run_until_idle(30)
    b = srv.submit(S.Request(700, 901, 5, inverse=True, data=f.result))
    bi = srv.submit(S.Request(333, 444, 3, "legall53", torch.int32, True, data=fi.result))
    assert srv.run_until_idle(30)
    maxabs = float(x.abs().max())
    assert float((b.result - x).abs().max()) <= 2 * 5 * TOL_F32 * maxabs
    assert torch.equal(bi.result.cpu(), xi.cpu())


def test_host_input_is_staged():
    x = _data(120, 250, "cdf97", torch.float32, 9)
    host = x.cpu().pin_memory()
    srv = S.Server(budget_bytes=1 << 30)
    a = srv.submit(S.Request(120, 250, 3, data=x))
    b = srv.submit(S.Request(120, 250, 3, data=host))
    assert b.reserved > a.reserved  # the device copy of the input is counted
    assert srv.run_until_idle(30)
    assert torch.equal(a.result.cpu(), b.result.cpu())


def test_poisson_stream_under_small_budget():
    rng = np.random.default_rng(7)
    reqs = [_random_request(rng, 3000 + i) for i in range(150)]
    budget = 96 << 20
    srv = S.Server(budget_bytes=budget, max_batch=32)
    arrivals = np.cumsum(rng.exponential(1 / 2000.0, len(reqs)))
    t0 = time.perf_counter()
    tickets, i = [], 0
    while i < len(reqs) or any(not t.finished() for t in tickets):
        now = time.perf_counter() - t0
        while i < len(reqs) and arrivals[i] <= now:
            tickets.append(srv.submit(reqs[i], t_arrival=t0 + arrivals[i]))
            i += 1
        srv.poll()
        for t in tickets:
            if t.state == S.DONE and t.result is not None:
                srv.release(t)
        assert time.perf_counter() - t0 < 60
    st = srv.stats()
    assert st["completed"] + st["rejected"] == len(reqs)
    assert all(t.state == S.REJECTED and "budget" in t.error for t in tickets if t.state != S.DONE)
    assert st["peak_bytes"] <= budget
    assert st["p50_s"] > 0 and st["p99_s"] >= st["p50_s"]
    assert srv.in_use == 0


def _batch_jobs(seed, n=48):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        h, w = int(rng.integers(100, 700)), int(rng.integers(100, 700))
        wav, dt = ("cdf97", torch.float32) if i % 3 else ("legall53", torch.int32)
        src = _data(h, w, wav, dt, seed * 100 + i)
        jobs.append((src, D.empty_image(h, w, dt), int(rng.integers(1, 6)), wav, 0))
    return jobs


def _run_gated(ex, batches):
    """Launch `batches` (job lists) through the executor, every stream held at
    one gate that opens after all of them are queued: their device work
    starts together whatever the host's launch latency.  Returns the handles
    and the gate event."""
    gate = torch.cuda.Event(enable_timing=True)
    opener = torch.cuda.Stream()
    with torch.cuda.stream(opener):
        # the gate is recorded behind about 10 ms of spinning: every launch
        # below is queued before it opens
        torch.cuda._sleep(20_000_000)
        gate.record(opener)
    handles = []
    for jobs in batches:
        ex.stream.wait_event(gate)
        handles.append(ex.launch(jobs))
    torch.cuda.synchronize()
    for h in handles:
        assert ex.status(h) == 0
    return handles, gate


def test_batches_in_flight_overlap_on_the_device():
    """Two batches admitted one after the other run on two streams of the
    executor: on the device they overlap (the second starts before the first
    ends, and together they take clearly less than the two alone), and each
    gives the same bits as when it runs alone."""
    jobs_a, jobs_b = _batch_jobs(1), _batch_jobs(2)
    solo = []
    outs_alone = []
    for jobs in (jobs_a, jobs_b):
        ex1 = S.GpuExecutor(streams=1, timing=True)
        (h,), gate = _run_gated(ex1, [jobs])
        e0, e1 = ex1.span(h)
        solo.append(e0.elapsed_time(e1))
        outs_alone.append([d.clone() for (_s, d, _l, _w, _i) in jobs])
    ex2 = S.GpuExecutor(streams=2, timing=True)
    (ha, hb), gate = _run_gated(ex2, [jobs_a, jobs_b])
    assert ha[3] is not hb[3]  # two streams
    a0, a1 = ex2.span(ha)
    b0, b1 = ex2.span(hb)
    t = lambda e: gate.elapsed_time(e)  # noqa: E731  ms after the gate opened
    assert t(b0) < t(a1) and t(a0) < t(b1), (t(a0), t(a1), t(b0), t(b1))
    together = max(t(a1), t(b1)) - min(t(a0), t(b0))
    assert together < 0.85 * (solo[0] + solo[1]), (together, solo)
    for jobs, ref in zip((jobs_a, jobs_b), outs_alone):
        for (_s, d, _l, _w, _i), r in zip(jobs, ref):
            assert torch.equal(d, r)


def test_server_spreads_batches_over_streams():
    """With several batches in flight, the server has them on different streams."""
    ex = S.GpuExecutor(streams=3)
    srv = S.Server(budget_bytes=4 << 30, executor=ex, max_batch=4, max_inflight=3)
    srv.keep_handles = True
    tickets = [srv.submit(_with_data(S.Request(700, 900, 4, "cdf97", torch.float32, False), 9 + i))
               for i in range(12)]
    assert srv.run_until_idle(60)
    assert all(t.state == S.DONE for t in tickets)
    streams = {id(h[3]) for h, _n in srv.retired_handles}
    assert len(streams) == 3
    assert srv.stats()["requests_per_batch"] == pytest.approx(4.0)
