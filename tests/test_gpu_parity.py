"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several warp strips (240 / 224 / 192 pixels) and several row
segments with ragged tails, odd sizes, axes of length 1 and 2.  CDF 9/7
float32 must stay within 1e-5 * max|x| per level; reversible 5/3 int32 must be
bit-exact for every scheme.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

from oracle import lifting as L
from paper_1705_08266_gb300 import dwt2d as D
from tests.parity_util import (TOL_F32, assert_forward_matches, assert_inverse_matches, device_image,
                               host, make_input)

pytestmark = pytest.mark.gpu

SCHEMES = list(D.SCHEMES)


def schemes_for(wavelet):
    """The separable convolution scheme exists for the linear CDF 9/7 filter bank only."""
    return [s for s in SCHEMES if not (wavelet == "legall53" and s == "separable_convolution")]
SHAPES_LEVELS = [
    ((8, 8), 1), ((8, 8), 3), ((7, 9), 2), ((9, 7), 3), ((1, 9), 2), ((9, 1), 2), ((1, 1), 2),
    ((2, 2), 1), ((3, 3), 2), ((33, 70), 3), ((64, 300), 4), ((130, 257), 5), ((40, 513), 3),
    ((512, 512), 1), ((512, 512), 5), ((65, 1000), 6), ((301, 497), 4),
    # wide and tall enough for the interior (border-free) code path at every fused level
    ((1030, 2050), 5), ((2048, 1536), 3), ((777, 3001), 2),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    D.lib()


def _fwd_inv(x, levels, wavelet, scheme, options=None):
    h, w = x.shape
    plan = D.Plan(h, w, levels, wavelet, scheme, options=options)
    ws = plan.workspace()
    xd = device_image(x)
    c = plan.forward(xd, workspace=ws)
    ref = L.forward(x, levels, wavelet)
    cref = device_image(ref.astype(x.dtype))
    y = plan.inverse(cref, workspace=ws)
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    return host(c), host(y), ref


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
@pytest.mark.parametrize("shape,levels", SHAPES_LEVELS)
def test_parity_all_schemes(wavelet, shape, levels):
    x = make_input(wavelet, *shape, seed=1705 + shape[0] * 7 + shape[1])
    for scheme in schemes_for(wavelet):
        c, y, ref = _fwd_inv(x, levels, wavelet, scheme)
        tag = f"{wavelet} {scheme} {shape} L{levels}"
        assert_forward_matches(c, x, levels, wavelet, tag)
        assert_inverse_matches(y, ref.astype(x.dtype), levels, wavelet, x, tag)


@pytest.mark.parametrize("fuse", ["1", "2", "3"])
@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
def test_parity_many_segments_and_fusion(fuse, wavelet):
    """Tiny row segments (many warps per strip) and every fusion depth."""
    opts = dict(fuse_max=int(fuse), min_segment=1, fwd_warps_per_sm=4000, inv_warps_per_sm=4000)
    for shape, levels in [((200, 777), 3), ((97, 515), 5), ((450, 250), 4)]:
        x = make_input(wavelet, *shape, seed=11 + shape[1])
        for scheme in ("separable", "nonsep", "nonsep_reduced"):
            c, y, ref = _fwd_inv(x, levels, wavelet, scheme, opts)
            tag = f"fuse={fuse} {wavelet} {scheme} {shape} L{levels}"
            assert_forward_matches(c, x, levels, wavelet, tag)
            assert_inverse_matches(y, ref.astype(x.dtype), levels, wavelet, x, tag)


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
@pytest.mark.parametrize("shape", [(16, 65536), (65536, 16)])
def test_extreme_aspect(wavelet, shape):
    """Largest allowed side (65536) with a short other side, 6 levels."""
    x = make_input(wavelet, *shape, seed=3)
    c, y, ref = _fwd_inv(x, 6, wavelet, "nonsep_reduced")
    assert_forward_matches(c, x, 6, wavelet, f"{shape}")
    assert_inverse_matches(y, ref.astype(x.dtype), 6, wavelet, x, f"{shape}")


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
def test_constant_and_ramp(wavelet):
    """Constant image: zero details and LL = value; ramp: zero interior details."""
    dt = np.int32 if wavelet == "legall53" else np.float32
    for x in (np.full((130, 257), 100, dtype=dt),
              (3 * np.arange(257)[None, :] + 5 * np.arange(130)[:, None]).astype(dt)):
        for scheme in schemes_for(wavelet):
            c, _, _ = _fwd_inv(x, 3, wavelet, scheme)
            assert_forward_matches(c, x, 3, wavelet, scheme)


def test_round_trip_gpu_only():
    """inverse(forward(x)) == x through the GPU alone (5/3 exactly)."""
    for wavelet in ("cdf97", "legall53"):
        x = make_input(wavelet, 777, 1029, seed=5)
        for scheme in schemes_for(wavelet):
            plan = D.Plan(777, 1029, 5, wavelet, scheme)
            ws = plan.workspace()
            y = host(plan.inverse(plan.forward(device_image(x), workspace=ws), workspace=ws))
            if wavelet == "legall53":
                assert np.array_equal(y, x), scheme
            else:
                # forward and inverse each stay within TOL per level: 2 * levels * TOL overall
                assert np.max(np.abs(y - x)) <= 2 * 5 * 1e-5 * np.max(np.abs(x)), scheme


def test_convolution_rejects_integer_wavelet():
    with pytest.raises(D.DwtError):
        D.Plan(64, 64, 2, "legall53", "separable_convolution")


def test_host_entry_points():
    """dwt2d_forward_host / inverse_host: host buffers in, host buffers out."""
    x = make_input("cdf97", 300, 500, seed=8)
    plan = D.Plan(300, 500, 4, "cdf97", "nonsep_reduced")
    ws = plan.workspace()
    hs = torch.from_numpy(x).pin_memory()
    hd = torch.empty_like(hs).pin_memory()
    din = D.empty_image(300, 500)
    dout = D.empty_image(300, 500)
    plan.forward_host(hs, hd, din, dout, ws)
    assert_forward_matches(hd.numpy(), x, 4, "cdf97", "host fwd")
    back = torch.empty_like(hs).pin_memory()
    plan.inverse_host(hd, back, din, dout, ws)
    assert np.max(np.abs(back.numpy() - x)) <= 1e-5 * np.max(np.abs(x))


@pytest.mark.parametrize("h,w,levels,wavelet,dtype", [
    (1030, 2050, 5, "cdf97", torch.float32), (2048, 1536, 3, "legall53", torch.int32),
    (4097, 333, 2, "cdf97", torch.float32), (1024, 1024, 1, "cdf97", torch.float32),
    (1500, 900, 6, "cdf97", torch.float16), (3001, 777, 4, "legall53", torch.int32)])
def test_host_pipelined_equals_device_entry_points(h, w, levels, wavelet, dtype):
    """The host-buffer forward and inverse overlap their copies with the
    transform by row bands; the results are the device entry points', bit for
    bit."""
    x = make_input(wavelet, h, w, seed=h + w)
    if dtype == torch.float16:
        x = x / float(np.max(np.abs(x)))
    xt = torch.from_numpy(x).to(dtype)
    plan = D.Plan(h, w, levels, wavelet, "nonsep_reduced", dtype)
    ws = plan.workspace()
    hs = xt.pin_memory()
    hd = torch.full_like(hs, 7).pin_memory()
    din = D.empty_image(h, w, dtype)
    dout = D.empty_image(h, w, dtype)
    plan.forward_host(hs, hd, din, dout, ws)
    ref = plan.forward(device_image(x).to(dtype) if dtype != torch.float16 else _dev16(xt))
    torch.cuda.synchronize()
    assert torch.equal(hd, ref.cpu())
    assert plan.status(ws) == 0
    # the inverse counterpart (coarse region first, detail bands by rows, image rows out)
    back = torch.full_like(hs, 5).pin_memory()
    plan.inverse_host(hd, back, din, dout, ws)
    ref_back = plan.inverse(_dev16(hd))
    torch.cuda.synchronize()
    assert torch.equal(back, ref_back.cpu())
    assert plan.status(ws) == 0


def _dev16(t):
    d = D.empty_image(t.shape[0], t.shape[1], t.dtype)
    d.copy_(t)
    return d


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
@pytest.mark.parametrize("shape,levels", [((130, 257), 5), ((1030, 2050), 5), ((777, 3001), 2)])
def test_cross_scheme_agreement(wavelet, shape, levels):
    """Separable, non-separable and reduced lifting compute one transform:
    bit-exact for the integer 5/3 (nested floors reproduce the separable
    order); for FP32 9/7 within twice the per-scheme oracle tolerance (each is
    within TOL_F32 * max|x| of the FP64 result)."""
    h, w = shape
    x = make_input(wavelet, h, w, seed=h * 7 + w)
    xd = device_image(x)
    outs = {}
    for scheme in ("separable", "nonsep", "nonsep_reduced", "nonsep_multipass"):
        outs[scheme] = D.Plan(h, w, levels, wavelet, scheme).forward(xd).cpu()
    torch.cuda.synchronize()
    ref = outs["separable"]
    for scheme, got in outs.items():
        if wavelet == "legall53":
            assert torch.equal(got, ref), scheme
        else:
            maxabs = float(np.max(np.abs(x)))
            d = float((got.double() - ref.double()).abs().max())
            assert d <= 2 * TOL_F32 * maxabs, (scheme, d / maxabs)


@pytest.mark.parametrize("wavelet,dtype,scheme", [
    ("cdf97", torch.float32, "nonsep_reduced"), ("cdf97", torch.float32, "separable"),
    ("cdf97", torch.float32, "nonsep"), ("legall53", torch.int32, "nonsep_reduced"),
    ("cdf97", torch.bfloat16, "nonsep_reduced")])
def test_programmatic_launch_changes_nothing(wavelet, dtype, scheme):
    """Launches with programmatic stream serialization start while the one
    before them drains and wait in griddepcontrol.wait before their first
    global access.  Chained transforms issued back to back on one stream (each
    forward overwrites what the previous inverse read, each inverse reads what
    the forward just wrote) give the same bits as serialized launches."""
    h, w, levels = 2050, 3001, 6
    x = make_input(wavelet, h, w, seed=99)
    if dtype == torch.bfloat16:
        x = x / float(np.max(np.abs(x)))
    xt = torch.from_numpy(x).to(dtype)
    res = {}
    for pdl in ("0", "1"):
        plan = D.Plan(h, w, levels, wavelet, scheme, dtype,
                      options=dict(programmatic_launch=1 if pdl == "1" else -1))
        assert plan.info()[0] >= 3
        ws = plan.workspace()
        src = _dev16(xt)
        c = D.empty_image(h, w, dtype)
        r = D.empty_image(h, w, dtype)
        for _ in range(4):
            plan.forward(src, c, ws)
            plan.inverse(c, r, ws)
            plan.forward(r, c, ws)
        torch.cuda.synchronize()
        assert plan.status(ws) == 0
        res[pdl] = (c.cpu(), r.cpu())
    assert torch.equal(res["0"][0], res["1"][0])
    assert torch.equal(res["0"][1], res["1"][1])


@pytest.mark.parametrize("bands", ["1", "5", "64"])
@pytest.mark.parametrize("h,w,levels,wavelet,dtype", [
    (1030, 2050, 5, "cdf97", torch.float32), (2051, 777, 3, "legall53", torch.int32)])
def test_host_pipelined_band_counts(bands, h, w, levels, wavelet, dtype):
    """Any number of row bands (one, a ragged count, more bands than row
    segments) gives the device entry points' results bit for bit."""
    x = make_input(wavelet, h, w, seed=h + 3 * w)
    xt = torch.from_numpy(x).to(dtype)
    plan = D.Plan(h, w, levels, wavelet, "nonsep_reduced", dtype, options=dict(host_bands=int(bands)))
    ws = plan.workspace()
    hs = xt.pin_memory()
    hd = torch.full_like(hs, 3).pin_memory()
    din = D.empty_image(h, w, dtype)
    dout = D.empty_image(h, w, dtype)
    plan.forward_host(hs, hd, din, dout, ws)
    ref = plan.forward(_dev16(xt))
    torch.cuda.synchronize()
    assert torch.equal(hd, ref.cpu())
    back = torch.full_like(hs, 9).pin_memory()
    plan.inverse_host(hd, back, din, dout, ws)
    ref_back = plan.inverse(_dev16(hd))
    torch.cuda.synchronize()
    assert torch.equal(back, ref_back.cpu())
    assert plan.status(ws) == 0


LAUNCH_OPTIONS = [
    {"fwd_cols_per_lane": 4},
    {"fwd_cols_per_lane": 4, "fwd_short_tail": 4, "fwd_warps_per_sm_large": 24},
    {"fwd_short_tail": 3, "inv_short_tail": 4},
    {"fwd_cols_per_lane": 4, "fwd_short_tail": 2, "min_segment": 1, "fwd_warps_per_sm": 4000,
     "inv_short_tail": 2, "inv_warps_per_sm": 4000},
    {"fwd_cols_per_lane": 4, "fuse_first": 1, "fwd_seg_interleave": 1, "inv_seg_interleave": -1},
    {"inv_cols_per_lane": 4, "inv_short_tail": -1},
    {"programmatic_launch": -1},
]


@pytest.mark.parametrize("opts", LAUNCH_OPTIONS, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
@pytest.mark.parametrize("wavelet,dtype", [("cdf97", torch.float32), ("legall53", torch.int32),
                                           ("cdf97", torch.float16)])
def test_launch_options_give_the_same_bits(opts, wavelet, dtype):
    """Launch options change how the rows are cut into launches, warps and
    segments (columns per lane, short last-wave segments, interleave, fusion),
    not the arithmetic: every setting gives the default plan's bits, forward
    and inverse, and the default plan matches the oracle.  (With 16-bit
    storage the LL between launches is rounded to 16 bits, so a different
    fusion depth is checked against the tolerance instead.)"""
    regroups = "fuse_first" in opts or "fuse_max" in opts
    for (h, w), levels in [((1030, 2050), 5), ((2048, 1536), 3), ((777, 3001), 2), ((301, 497), 4),
                           ((4099, 520), 6)]:
        x = make_input(wavelet, h, w, seed=h * 5 + w)
        scale = 1.0
        if dtype == torch.float16:
            scale = float(np.max(np.abs(x)))
            x = x / scale
        xt = torch.from_numpy(x).to(dtype)
        res = []
        for o in ({}, opts):
            plan = D.Plan(h, w, levels, wavelet, "nonsep_reduced", dtype, options=o or None)
            ws = plan.workspace()
            c = plan.forward(_dev16(xt), workspace=ws, scale=scale)
            y = plan.inverse(c, workspace=ws, scale=scale)
            torch.cuda.synchronize()
            assert plan.status(ws) == 0
            res.append((c.cpu(), y.cpu()))
        if dtype == torch.float16 and regroups:
            d = (res[0][0].float() - res[1][0].float()).abs().max().item()
            assert d <= 2e-3, (opts, h, w, levels, d)
            continue
        assert torch.equal(res[0][0], res[1][0]), (opts, h, w, levels, "forward")
        assert torch.equal(res[0][1], res[1][1]), (opts, h, w, levels, "inverse")
        if dtype != torch.float16:
            assert_forward_matches(res[0][0].numpy(), x, levels, wavelet, f"{h}x{w} L{levels}")


def test_plans_sharing_a_workspace():
    """Two different plans called alternately on one workspace, many times in
    a row on one stream, give the bits of calls on fresh workspaces."""
    shapes = [((2050, 3001), 6), ((1030, 2050), 5)]
    plans = [D.Plan(h, w, lv, "cdf97", "nonsep_reduced") for (h, w), lv in shapes]
    ws = torch.empty(max(p.workspace_bytes for p in plans), dtype=torch.uint8, device="cuda")
    D.lib().dwt2d_workspace_init(ctypes.c_void_p(ws.data_ptr()), None)
    xs = [device_image(make_input("cdf97", h, w, seed=h + w)) for (h, w), _lv in shapes]
    refs = [p.forward(x) for p, x in zip(plans, xs)]  # each on its own fresh workspace
    outs = [D.empty_image(x.shape[0], x.shape[1]) for x in xs]
    for _ in range(5):
        for p, x, o in zip(plans, xs, outs):
            p.forward(x, o, ws)
    torch.cuda.synchronize()
    assert plans[0].status(ws) == 0
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
