"""Serving loop host logic on the CPU, with a stand-in executor: admission in
arrival order under the memory budget, back pressure, and the failure paths
(malformed request, oversize request, refused allocation, cancellation, slow
or failing loader, failed kernel status), each isolated to its own request."""
import time

import pytest
import torch

from paper_1705_08266_gb300 import serve as S


class FakeExecutor:
    """out = 2 * src (forward) or -src (inverse); a batch is 'running' for
    `lag` polls; `bad_batches` get a nonzero kernel status."""

    def __init__(self, lag=0, bad_batches=()):
        self.lag = lag
        self.bad = set(bad_batches)
        self.launched = []

    def workspace_bytes(self, req):
        return 1000

    def empty(self, h, w, dt):
        return torch.empty(h, w, dtype=dt)

    def pitched(self, t):
        return t.is_contiguous()

    def copy_in(self, dst, src):
        dst.copy_(src)

    def launch(self, jobs):
        idx = len(self.launched)
        self.launched.append(len(jobs))
        for src, out, lv, wav, inv in jobs:
            out.copy_(-src if inv else 2 * src)
        return {"polls": self.lag, "idx": idx}

    def done(self, h):
        if h["polls"] > 0:
            h["polls"] -= 1
            return False
        return True

    def status(self, h):
        return -6 if h["idx"] in self.bad else 0


def req(h=8, w=8, lv=2, inv=False, fill=1.0, dtype=torch.float32, wav="cdf97"):
    return S.Request(h, w, lv, wav, dtype, inv, data=torch.full((h, w), fill, dtype=dtype))


def img_bytes(h, w, es=4):
    return h * ((w * es + 15) // 16 * 16)


NEED = img_bytes(8, 8) + 1000 + 4 * S.TABLE_ENTRY_BYTES  # one 8x8 float request


def test_all_complete_with_results_and_stats():
    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor())
    ts = [srv.submit(req(fill=float(i), inv=i % 3 == 0)) for i in range(20)]
    assert srv.run_until_idle(5)
    for i, t in enumerate(ts):
        assert t.state == S.DONE, t.error
        want = -float(i) if i % 3 == 0 else 2.0 * i
        assert torch.all(t.result == want)
    st = srv.stats()
    assert st["completed"] == 20 and st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    # resident outputs stay counted until released
    assert srv.in_use == 20 * img_bytes(8, 8)
    for t in ts:
        srv.release(t)
    assert srv.in_use == 0


@pytest.mark.parametrize("bad", [
    S.Request(0, 8, 1, data=torch.zeros(0, 8)),
    S.Request(8, 8, 0, data=torch.zeros(8, 8)),
    S.Request(8, 8, 17, data=torch.zeros(8, 8)),
    S.Request(8, 8, 2, "cdf97", torch.int32, data=torch.zeros(8, 8, dtype=torch.int32)),
    S.Request(8, 8, 2, "legall53", torch.float32, data=torch.zeros(8, 8)),
    S.Request(8, 8, 2, data=torch.zeros(8, 9)),
    S.Request(8, 8, 2, data=torch.zeros(8, 8, dtype=torch.float64)),
    S.Request(8, 8, 2),
    S.Request(8, 8, 2, data=[[0.0] * 8] * 8),
    S.Request(8.0, 8, 2, data=torch.zeros(8, 8)),
])
def test_malformed_request_is_rejected_alone(bad):
    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor())
    a = srv.submit(req(fill=3.0))
    b = srv.submit(bad)
    c = srv.submit(req(fill=4.0))
    assert b.state == S.REJECTED and b.error
    assert srv.run_until_idle(5)
    assert a.state == c.state == S.DONE
    assert torch.all(a.result == 6.0) and torch.all(c.result == 8.0)


def test_oversize_request_rejected_others_run():
    srv = S.Server(budget_bytes=3 * NEED, executor=FakeExecutor())
    big = srv.submit(req(h=64, w=64))
    small = srv.submit(req())
    assert big.state == S.REJECTED and "budget" in big.error
    assert srv.run_until_idle(5) and small.state == S.DONE


def test_back_pressure_until_release_and_peak_within_budget():
    need = img_bytes(64, 64) + 1000 + 4 * S.TABLE_ENTRY_BYTES
    srv = S.Server(budget_bytes=2 * need + 10, executor=FakeExecutor())
    ts = [srv.submit(req(64, 64, fill=float(i))) for i in range(6)]
    for _ in range(10):
        srv.poll()
    # two fit; their outputs stay resident and leave no room for a third
    assert [t.state for t in ts] == [S.DONE] * 2 + [S.QUEUED] * 4
    assert srv.peak <= srv.budget
    while not all(t.state == S.DONE for t in ts):
        for t in ts:
            if t.state == S.DONE:
                srv.release(t)
        srv.poll()
    assert srv.peak <= srv.budget
    for t in ts:
        srv.release(t)
    assert srv.in_use == 0


def test_refused_allocation_fails_that_request_only():
    victim = {}

    def alloc(t, h, w, dt):
        if t.id == victim.get("id"):
            raise MemoryError("injected refusal")
        return torch.empty(h, w, dtype=dt)

    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor(), allocator=alloc)
    a = srv.submit(req(fill=1.0))
    b = srv.submit(req(fill=2.0))
    victim["id"] = b.id
    c = srv.submit(req(fill=3.0))
    assert srv.run_until_idle(5)
    assert b.state == S.FAILED and "allocation refused" in b.error and b.result is None
    assert a.state == c.state == S.DONE and torch.all(c.result == 6.0)
    assert srv.in_use == 2 * img_bytes(8, 8)


def test_cancel_queued_and_running():
    ex = FakeExecutor(lag=3)
    srv = S.Server(budget_bytes=1 << 30, executor=ex, max_inflight=1)
    a = srv.submit(req(fill=1.0))
    srv.poll()                       # a is running (3 polls)
    b = srv.submit(req(fill=2.0))    # queued behind the one batch in flight
    assert a.state == S.RUNNING and b.state == S.QUEUED
    assert srv.cancel(b) and b.state == S.CANCELLED
    assert srv.cancel(a)
    assert srv.run_until_idle(5)
    assert a.state == S.CANCELLED and a.result is None
    assert ex.launched == [1]        # b never launched
    assert srv.in_use == 0
    assert not srv.cancel(a)         # already finished


def test_slow_loader_does_not_hold_the_queue():
    def slow():
        time.sleep(0.3)
        return torch.full((8, 8), 5.0)

    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor())
    s = srv.submit(S.Request(8, 8, 2, loader=slow))
    fast = [srv.submit(req(fill=float(i))) for i in range(5)]
    t0 = time.perf_counter()
    while not all(t.state == S.DONE for t in fast):
        srv.poll()
        assert time.perf_counter() - t0 < 0.25, "fast requests waited for the slow loader"
    assert s.state == S.LOADING
    assert srv.run_until_idle(5)
    assert s.state == S.DONE and torch.all(s.result == 10.0)
    assert max(t.t_done for t in fast) < s.t_done


def test_failing_loader_and_bad_loaded_data():
    def boom():
        raise IOError("disk gone")

    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor())
    a = srv.submit(S.Request(8, 8, 2, loader=boom))
    b = srv.submit(S.Request(8, 8, 2, loader=lambda: torch.zeros(4, 4)))
    c = srv.submit(req(fill=1.0))
    assert srv.run_until_idle(5)
    assert a.state == S.FAILED and "loader failed" in a.error
    assert b.state == S.FAILED and "shape" in b.error
    assert c.state == S.DONE


def test_failed_kernel_status_fails_its_batch_only():
    ex = FakeExecutor(bad_batches={0})
    srv = S.Server(budget_bytes=1 << 30, executor=ex)
    a = srv.submit(req(fill=1.0))
    srv.poll()                       # batch 0 = [a]
    b = srv.submit(req(fill=2.0))
    assert srv.run_until_idle(5)
    assert a.state == S.FAILED and "status -6" in a.error
    assert b.state == S.DONE and torch.all(b.result == 4.0)
    assert srv.in_use == img_bytes(8, 8)


def test_non_pitched_input_is_copied_and_counted():
    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor())
    x = torch.arange(64.0).reshape(8, 8).t()  # not contiguous -> device copy
    t = srv.submit(S.Request(8, 8, 1, data=x))
    assert t.reserved == NEED + img_bytes(8, 8)
    assert srv.run_until_idle(5)
    assert torch.equal(t.result, 2 * x)
    assert srv.in_use == img_bytes(8, 8)


def test_result_drives_the_loop_and_reports_failures():
    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor(lag=2))
    t = srv.submit(req(fill=2.0))
    assert torch.all(srv.result(t, timeout=5) == 4.0)
    bad = srv.submit(S.Request(8, 8, 0, data=torch.zeros(8, 8)))
    with pytest.raises(RuntimeError, match="rejected"):
        srv.result(bad, timeout=5)
    slow = srv.submit(S.Request(8, 8, 2, loader=lambda: (time.sleep(0.5), torch.zeros(8, 8))[1]))
    with pytest.raises(TimeoutError):
        srv.result(slow, timeout=0.05)
    assert torch.all(srv.result(slow, timeout=5) == 0.0)


def test_counts_exact_with_concurrent_loader_failures():
    """Loader threads finish failed loads while the polling thread finishes
    completed batches: every request is counted exactly once."""
    def boom():
        time.sleep(0.001)
        raise IOError("gone")

    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor(), loader_threads=8)
    bad = [srv.submit(S.Request(8, 8, 1, loader=boom)) for _ in range(150)]
    good = [srv.submit(req(fill=float(i))) for i in range(150)]
    assert srv.run_until_idle(10)
    st = srv.stats()
    assert st["failed"] == 150 and st["completed"] == 150
    assert all(t.state == S.FAILED for t in bad) and all(t.state == S.DONE for t in good)
    srv.reset_stats()
    st = srv.stats()
    assert st["completed"] == 0 and st["p99_s"] is None
    srv.close()


def test_take_finished_hands_each_ticket_out_once():
    """Finished tickets (done, rejected) come out of take_finished once each,
    in the order they finished; without tracking the call is refused."""
    srv = S.Server(budget_bytes=1 << 30, executor=FakeExecutor(lag=1), track_finished=True)
    bad = srv.submit(req(h=0))  # malformed: rejected at submit
    ts = [srv.submit(req(fill=float(i))) for i in range(6)]
    got = srv.take_finished()
    assert got == [bad] and bad.state == S.REJECTED
    seen = []
    for _ in range(50):
        srv.poll()
        seen += srv.take_finished()
        if len(seen) == len(ts):
            break
    assert sorted(t.id for t in seen) == sorted(t.id for t in ts)
    assert all(t.state == S.DONE for t in seen)
    assert [t.t_done for t in seen] == sorted(t.t_done for t in seen)
    assert srv.take_finished() == []
    for t in seen:
        srv.release(t)
    assert srv.in_use == 0
    with pytest.raises(RuntimeError):
        S.Server(budget_bytes=1 << 30, executor=FakeExecutor()).take_finished()


def test_queue_admits_in_arrival_order_under_backlog():
    """A backlog longer than one batch drains in arrival order, max_batch at a time."""
    ex = FakeExecutor()
    srv = S.Server(budget_bytes=1 << 30, executor=ex, max_batch=4, max_inflight=1)
    ts = [srv.submit(req(fill=float(i))) for i in range(10)]
    assert srv.run_until_idle(5)
    assert ex.launched == [4, 4, 2]
    assert [t.t_start for t in ts] == sorted(t.t_start for t in ts)
