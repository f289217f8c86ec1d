"""Batched transforms: many images of different sizes, level counts, wavelets,
storage types and directions in a few launches.

Each image of a batch must come out bit for bit as the single-image entry
point computes it (same lifting arithmetic, only the warp-to-work mapping
differs), and within the oracle's tolerance.  A batch captured in a CUDA graph
and replayed on new input contents gives the same results again.
"""
import numpy as np
import pytest
import torch

from oracle import lifting as L
from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import synth
from tests.parity_util import TOL_F32, assert_forward_matches, device_image

pytestmark = pytest.mark.gpu

# (height, width, levels, wavelet, dtype, inverse)
MIXED = [
    (96, 130, 3, "cdf97", torch.float32, 0),
    (1, 5, 1, "cdf97", torch.float32, 0),
    (3, 3, 2, "cdf97", torch.float32, 1),
    (257, 511, 5, "cdf97", torch.float32, 0),
    (64, 64, 1, "cdf97", torch.float32, 1),
    (200, 33, 4, "legall53", torch.int32, 0),
    (130, 96, 3, "legall53", torch.int32, 1),
    (77, 1030, 2, "cdf97", torch.float16, 0),
    (512, 300, 6, "cdf97", torch.bfloat16, 1),
    (1030, 770, 5, "cdf97", torch.float32, 1),
    (17, 2, 3, "legall53", torch.int32, 0),
    (640, 480, 3, "cdf97", torch.float32, 0),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    D.lib()


def _input(h, w, levels, wavelet, dtype, inverse, seed):
    """The host array a job starts from (image, or coefficients of one)."""
    x = synth.image(wavelet, h, w, seed)
    if dtype in (torch.float16, torch.bfloat16):
        x = (x / max(1.0, float(np.max(np.abs(x))))).astype(np.float32)
    if inverse:
        c = L.forward(x.astype(np.int64 if wavelet == "legall53" else np.float64), levels, wavelet)
        x = c.astype(np.int32) if wavelet == "legall53" else c.astype(np.float32)
    return torch.from_numpy(x).to(dtype)


def _jobs(spec, seed0, scheme="nonsep_reduced"):
    jobs, hosts = [], []
    for i, (h, w, lv, wav, dt, inv) in enumerate(spec):
        xh = _input(h, w, lv, wav, dt, inv, seed0 + i)
        src = D.empty_image(h, w, dt)
        src.copy_(xh)
        dst = D.empty_image(h, w, dt)
        dst.fill_(0)
        jobs.append((src, dst, lv, wav, inv))
        hosts.append(xh)
    return jobs, hosts


def _single(src, levels, wavelet, inverse, scheme):
    plan = D.Plan(src.shape[0], src.shape[1], levels, wavelet, scheme, src.dtype)
    out = plan.inverse(src) if inverse else plan.forward(src)
    return out


def _assert_same_as_single(jobs, scheme, what):
    for i, (src, dst, lv, wav, inv) in enumerate(jobs):
        ref = _single(src, lv, wav, inv, scheme)
        torch.cuda.synchronize()
        a, b = dst.cpu(), ref.cpu()
        if not torch.equal(a, b):
            d = (a.to(torch.float64) - b.to(torch.float64)).abs().max().item()
            raise AssertionError(f"{what} item {i} {tuple(src.shape)} L{lv} {wav} inv={inv}: "
                                 f"differs from the single-image call, max |diff| {d:.3g}")


@pytest.mark.parametrize("scheme", ["nonsep_reduced", "separable", "nonsep"])
def test_mixed_batch_equals_single_image_calls(scheme):
    jobs, hosts = _jobs(MIXED, 2026, scheme)
    batch = D.Batch(jobs, scheme)
    ws = batch.workspace()
    batch.upload(ws)
    batch.launch(ws)
    torch.cuda.synchronize()
    assert batch.status(ws) == 0
    launches, warps = batch.info()
    assert 1 <= launches <= 3 * 2 * 4 * 2  # phases x directions x types x depths
    _assert_same_as_single(jobs, scheme, scheme)


def test_mixed_batch_against_oracle():
    jobs, hosts = _jobs(MIXED, 4242)
    batch = D.Batch(jobs)
    ws = batch.workspace()
    batch.upload(ws)
    batch.launch(ws)
    torch.cuda.synchronize()
    for (src, dst, lv, wav, inv), xh in zip(jobs, hosts):
        if xh.dtype in (torch.float16, torch.bfloat16):
            continue  # 16-bit storage has its own tolerance tests
        got = dst.cpu().numpy()
        if inv:
            ref = L.inverse(xh.numpy().astype(np.float64) if wav == "cdf97" else xh.numpy().astype(np.int64),
                            lv, wav)
            if wav == "legall53":
                assert np.array_equal(got.astype(np.int64), ref)
            else:
                maxabs = float(np.max(np.abs(ref)))
                assert float(np.max(np.abs(got - ref))) <= TOL_F32 * max(maxabs, 1.0)
        else:
            assert_forward_matches(got, xh.numpy(), lv, wav, f"{tuple(xh.shape)} L{lv}")


def test_many_small_images_one_launch_per_bucket():
    rng = np.random.default_rng(1705)
    spec = []
    for _ in range(256):
        h, w = int(rng.integers(16, 300)), int(rng.integers(16, 300))
        spec.append((h, w, 3, "cdf97", torch.float32, 0))
    jobs, _ = _jobs(spec, 7000)
    batch = D.Batch(jobs)
    launches, warps = batch.info()
    assert launches == 2  # phase 0: 2 fused levels, phase 1: the last level
    assert warps >= 256
    ws = batch.workspace()
    batch.upload(ws)
    batch.launch(ws)
    torch.cuda.synchronize()
    assert batch.status(ws) == 0
    _assert_same_as_single(jobs, "nonsep_reduced", "256 images")


@pytest.mark.parametrize("tuning", [{"fuse_first": 1, "fuse_max": 1}, {"warps_per_sm": 2},
                                    {"min_segment": 64}, {"fuse_first": 2, "warps_per_sm": 40}])
def test_tuning_knobs_keep_results(tuning):
    """Different fusion depths and decompositions: the same coefficients (the
    oracle's, within tolerance; bit-exact where only the decomposition moves)."""
    jobs, hosts = _jobs(MIXED[:6], 99)
    batch = D.Batch(jobs, tuning=tuning)
    ws = batch.workspace()
    batch.upload(ws)
    batch.launch(ws)
    torch.cuda.synchronize()
    assert batch.status(ws) == 0
    if "fuse_first" in tuning and tuning.get("fuse_max", 2) == 1:
        for (src, dst, lv, wav, inv), xh in zip(jobs, hosts):
            if not inv:
                assert_forward_matches(dst.cpu().numpy(), xh.numpy(), lv, wav, str(tuning))
    else:
        _assert_same_as_single(jobs, "nonsep_reduced", str(tuning))


def test_cuda_graph_replay_on_new_inputs():
    jobs, _ = _jobs(MIXED, 31)
    batch = D.Batch(jobs)
    ws = batch.workspace()
    side = torch.cuda.Stream()
    batch.upload(ws, stream=side)
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        batch.launch(ws, stream=side)
    for seed in (5, 6):
        for i, (src, dst, lv, wav, inv) in enumerate(jobs):
            h, w = src.shape
            src.copy_(_input(h, w, lv, wav, src.dtype, inv, seed * 100 + i))
            dst.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert batch.status(ws) == 0
        _assert_same_as_single(jobs, "nonsep_reduced", f"graph replay {seed}")


def test_single_item_batch_and_round_trip():
    x = synth.image("cdf97", 1030, 2050, 8)
    src = device_image(x)
    mid = D.empty_image(1030, 2050)
    out = D.empty_image(1030, 2050)
    b1 = D.Batch([(src, mid, 5, "cdf97", 0)])
    ws1 = b1.workspace()
    b1.upload(ws1)
    b1.launch(ws1)
    b2 = D.Batch([(mid, out, 5, "cdf97", 1)])
    ws2 = b2.workspace()
    b2.upload(ws2)
    b2.launch(ws2)
    torch.cuda.synchronize()
    ref = D.Plan(1030, 2050, 5).forward(src)
    torch.cuda.synchronize()
    assert torch.equal(mid.cpu(), ref.cpu())
    maxabs = float(np.max(np.abs(x)))
    assert float(np.max(np.abs(out.cpu().numpy() - x))) <= 2 * 5 * TOL_F32 * maxabs


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    from paper_1705_08266_gb300 import autotune

    jobs, _ = _jobs(MIXED[:6], 77)
    cands = [{"fuse_first": 2, "fuse_max": 2, "warps_per_sm": w, "min_segment": 2} for w in (12, 48)]
    cands.append({"fuse_first": 2, "fuse_max": 3, "warps_per_sm": 16, "min_segment": 2})  # refused
    path = str(tmp_path / "tune.json")
    best = autotune.tune(jobs, cache_path=path, iters=2, warmup=1, candidates=cands)
    assert best in cands[:2]
    import json
    entry = next(iter(json.load(open(path)).values()))
    assert len(entry["tried"]) == 2 and entry["tuning"] == best
    # the tuned batch computes the same coefficients as the single-image calls
    b = D.Batch(jobs, tuning=best)
    ws = b.workspace()
    b.upload(ws)
    b.launch(ws)
    torch.cuda.synchronize()
    assert b.status(ws) == 0
    _assert_same_as_single(jobs, "nonsep_reduced", "autotuned")


def test_programmatic_batch_launch_changes_nothing():
    """Batched launches with programmatic stream serialization (off by
    default), eager and replayed from a CUDA graph: the same bits as the
    serialized launches."""
    out = {}
    for pdl in ("0", "1"):
        jobs, _ = _jobs(MIXED, 555)
        batch = D.Batch(jobs, tuning=dict(programmatic_launch=int(pdl)))
        ws = batch.workspace()
        side = torch.cuda.Stream()
        batch.upload(ws, stream=side)
        for _ in range(3):
            batch.launch(ws, stream=side)
        side.synchronize()
        eager = [dst.cpu() for (_s, dst, _l, _w, _i) in jobs]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            batch.launch(ws, stream=side)
        for (_s, dst, _l, _w, _i) in jobs:
            dst.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert batch.status(ws) == 0
        out[pdl] = (eager, [dst.cpu() for (_s, dst, _l, _w, _i) in jobs])
    for a, b in zip(out["0"][0] + out["0"][1], out["1"][0] + out["1"][1]):
        assert torch.equal(a, b)


# ---- the persistent form: one launch per direction and storage type over a
# queue of work items

def _run_batch(jobs, scheme="nonsep_reduced", tuning=None):
    batch = D.Batch(jobs, scheme, tuning)
    ws = batch.workspace()
    batch.upload(ws)
    batch.launch(ws)
    torch.cuda.synchronize()
    assert batch.status(ws) == 0
    return batch, ws


@pytest.mark.parametrize("scheme", ["nonsep_reduced", "separable", "nonsep"])
def test_persistent_batch_equals_single_image_calls(scheme):
    jobs, _ = _jobs(MIXED, 2027, scheme)
    batch, ws = _run_batch(jobs, scheme, {"persistent": 1})
    launches, _ = batch.info()
    # one persistent launch per (direction, storage type) present in the mix
    kinds = {(inv, str(dt)) for (_h, _w, _l, _wv, dt, inv) in MIXED}
    assert launches == len(kinds)
    _assert_same_as_single(jobs, scheme, f"persistent {scheme}")


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("scheme", ["nonsep_reduced", "separable"])
def test_four_columns_per_lane_batch_equals_single_image_calls(scheme, persistent):
    """256-pixel strips (4 quadruple columns per lane) in both batched forms:
    the same bits as the single-image call."""
    jobs, _ = _jobs(MIXED, 2028, scheme)
    _run_batch(jobs, scheme, {"persistent": persistent, "cols_per_lane": 4})
    _assert_same_as_single(jobs, scheme, f"4 columns per lane, persistent={persistent} {scheme}")


def test_persistent_batch_graph_replay_on_new_inputs():
    """The queue counters are reset by the launch itself: a captured graph
    replays correctly, on new input contents, several times."""
    jobs, _ = _jobs(MIXED, 31, "nonsep_reduced")
    batch = D.Batch(jobs, "nonsep_reduced", {"persistent": 1})
    ws = batch.workspace()
    side = torch.cuda.Stream()
    batch.upload(ws, stream=side)
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        batch.launch(ws, stream=side)
    for rep, seed in enumerate((77, 78, 79)):
        fresh, _ = _jobs(MIXED, seed)
        for (src, dst, _l, _w, _i), (nsrc, _d, _l2, _w2, _i2) in zip(jobs, fresh):
            src.copy_(nsrc)
            dst.fill_(0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert batch.status(ws) == 0, rep
        _assert_same_as_single(jobs, "nonsep_reduced", f"graph replay {rep}")


def _c4_spec(seed=2017, n=256):
    """256 images, H, W ~ U{65..4096}, levels ~ U{1..6}, 75 % CDF 9/7 float32,
    25 % LeGall 5/3 int32, forward (the batching workload)."""
    rng = np.random.default_rng(seed)
    spec = []
    for _ in range(n):
        h, w = int(rng.integers(65, 4097)), int(rng.integers(65, 4097))
        lv = int(rng.integers(1, 7))
        wav = "cdf97" if rng.random() < 0.75 else "legall53"
        spec.append((h, w, lv, wav, torch.float32 if wav == "cdf97" else torch.int32, 0))
    return spec


@pytest.mark.parametrize("persistent,cols", [(0, 2), (1, 2), (1, 4)])
def test_c4_batch_full_workload(persistent, cols):
    """The whole 256-image batching workload: every image bit for bit as the
    single-image call, and sampled coefficients of every image against the
    oracle (each from its dependency window)."""
    spec = _c4_spec()
    base = {"cdf97": synth.gradient_noise(4096, 4096, 2017),
            "legall53": synth.uniform_int(4096, 4096, 2017)}
    jobs, hosts = [], []
    for (h, w, lv, wav, dt, inv) in spec:
        xh = np.ascontiguousarray(base[wav][:h, :w])
        src = D.empty_image(h, w, dt)
        src.copy_(torch.from_numpy(xh))
        jobs.append((src, D.empty_image(h, w, dt), lv, wav, 0))
        hosts.append(xh)
    _run_batch(jobs, "nonsep_reduced", {"persistent": persistent, "cols_per_lane": cols})
    _assert_same_as_single(jobs, "nonsep_reduced", f"C4 persistent={persistent} cols={cols}")
    if persistent == 0 or cols == 4:
        return  # the oracle samples once: every form gave the same bits
    rng = np.random.default_rng(99)
    for i, ((src, dst, lv, wav, _i), xh) in enumerate(zip(jobs, hosts)):
        h, w = xh.shape
        got = dst.cpu().numpy()
        he, we = (h + 1) // 2, (w + 1) // 2
        # two level-1 detail coefficients (small dependency windows), and every
        # 16th image one coefficient of its coarsest level as well
        pos = [(int(rng.integers(0, he)), int(rng.integers(we, w))),
               (int(rng.integers(he, h)), int(rng.integers(0, w)))]
        if i % 16 == 0:
            sizes = L.level_sizes(h, w, lv)
            hl, wl = sizes[-1]
            pos.append((int(rng.integers(0, (hl + 1) // 2)), int(rng.integers(0, wl))))
        maxabs = float(np.max(np.abs(xh)))
        for r, c in pos:
            ref = L.sample_coefficient(xh, lv, wav, r, c)
            if wav == "legall53":
                assert int(got[r, c]) == int(ref), (i, r, c)
            else:
                assert abs(float(got[r, c]) - float(ref)) <= TOL_F32 * maxabs, (i, r, c)
