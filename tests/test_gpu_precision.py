"""16-bit coefficient storage (FP16 / BF16) with FP32 lifting arithmetic.

The caller stores value / scale in 16 bits (scale = max|x| of the image).  The
FP64 oracle transforms the same dequantized 16-bit image, so the error
measures the transform (and the 16-bit rounding of its outputs and of the LL
handed between launches), not the input quantisation.  Error per band and
level <= 2e-3 * max|x| (FP16) and <= 1.6e-2 * max|x| (BF16).
"""
import json

import numpy as np
import pytest
import torch

from oracle import lifting as L
from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {torch.float16: 2e-3, torch.bfloat16: 1.6e-2}


def _quantised(h, w, dtype, seed):
    x = synth.gradient_noise(h, w, seed)
    scale = float(np.max(np.abs(x)))
    xq = torch.from_numpy(x / scale).to(dtype)
    xdq = xq.to(torch.float64).numpy() * scale  # what the stored image means
    return x, scale, xq, xdq


def _to_dev(t):
    d = D.empty_image(t.shape[0], t.shape[1], t.dtype)
    d.copy_(t)
    return d


def _band_errors(got, ref, levels):
    g = L.band_views(got, levels)
    r = L.band_views(ref, levels)
    return {k: float(np.max(np.abs(g[k] - r[k]))) if r[k].size else 0.0 for k in r}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    D.lib()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("scheme", ["nonsep_reduced", "separable", "nonsep", "separable_convolution"])
@pytest.mark.parametrize("shape,levels", [((1030, 2050), 6), ((777, 513), 4), ((64, 300), 3)])
def test_16bit_forward_and_inverse(dtype, scheme, shape, levels):
    h, w = shape
    x, scale, xq, xdq = _quantised(h, w, dtype, seed=1606 + h)
    maxabs = float(np.max(np.abs(xdq)))
    plan = D.Plan(h, w, levels, "cdf97", scheme, dtype)
    ws = plan.workspace()
    c = plan.forward(_to_dev(xq), workspace=ws, scale=scale)
    torch.cuda.synchronize()
    got = c.cpu().to(torch.float64).numpy() * scale
    ref = L.forward(xdq, levels, "cdf97")
    errs = _band_errors(got, ref, levels)
    worst = max(errs.values())
    assert worst <= TOL[dtype] * maxabs, (dtype, scheme, {k: v / maxabs for k, v in errs.items()})
    # inverse of the stored oracle coefficients
    cq = torch.from_numpy(ref / scale).to(dtype)
    cdq = cq.to(torch.float64).numpy() * scale
    y = plan.inverse(_to_dev(cq), workspace=ws, scale=scale)
    torch.cuda.synchronize()
    yg = y.cpu().to(torch.float64).numpy() * scale
    yref = L.inverse(cdq, levels, "cdf97")
    assert float(np.max(np.abs(yg - yref))) <= TOL[dtype] * maxabs
    assert plan.status(ws) == 0


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_16bit_full_size_sampled(dtype):
    """16384 x 16384, 6 levels: coefficients sampled from the oracle's dependency windows."""
    h = w = 16384
    levels = 6
    x = synth.gradient_noise(h, w, synth.SEED_PRECISION)
    scale = float(np.max(np.abs(x)))
    xq = torch.from_numpy(x / scale).to(dtype)
    del x
    xdq32 = (xq.to(torch.float32).numpy() * np.float32(scale))  # exact: 16-bit values scaled in float32
    maxabs = float(np.max(np.abs(xdq32)))
    plan = D.Plan(h, w, levels, "cdf97", "nonsep_reduced", dtype)
    c = plan.forward(_to_dev(xq), scale=scale)
    torch.cuda.synchronize()
    ch = c.cpu()
    rng = np.random.default_rng(1606)
    sizes = L.level_sizes(h, w, levels)
    pos = []
    for lvl, (hl, wl) in enumerate(sizes, start=1):
        he, we = (hl + 1) // 2, (wl + 1) // 2
        for r0, c0, r1, c1 in [(0, we, he, wl), (he, 0, hl, we), (he, we, hl, wl)] + (
                [(0, 0, he, we)] if lvl == levels else []):
            pos += [(r0, c0), (r1 - 1, c1 - 1)]
            pos += [(int(rng.integers(r0, r1)), int(rng.integers(c0, c1))) for _ in range(6)]
    worst = {}
    for r, cc in pos:
        ref = L.sample_coefficient(xdq32, levels, "cdf97", r, cc)
        got = float(ch[r, cc].to(torch.float64)) * scale
        key = _band_of(r, cc, sizes, levels)
        worst[key] = max(worst.get(key, 0.0), abs(got - ref) / maxabs)
    # the achieved error per band and level, as a fraction of max|x| (printed
    # for the record; pytest -s shows it)
    print("precision_report", json.dumps({"dtype": str(dtype).replace("torch.", ""),
                                          "image": [h, w], "levels": levels, "samples": len(pos),
                                          "max_err_over_maxabs": {f"L{k[0]} {k[1]}": round(v, 7)
                                                                  for k, v in sorted(worst.items())}}))
    for k, v in worst.items():
        assert v <= TOL[dtype], (k, v)


def _band_of(r, c, sizes, levels):
    """(level, band) of Mallat position (r, c)."""
    for lvl, (hl, wl) in enumerate(sizes, start=1):
        he, we = (hl + 1) // 2, (wl + 1) // 2
        if r < hl and c < wl and (r >= he or c >= we or lvl == levels):
            band = ("H" if c >= we else "L") + ("H" if r >= he else "L")
            return lvl, band
    raise ValueError((r, c))


def test_16bit_rejects_bad_scale_and_multipass():
    plan = D.Plan(64, 64, 2, "cdf97", "nonsep_reduced", torch.float16)
    xq = _to_dev(torch.zeros(64, 64, dtype=torch.float16))
    with pytest.raises(D.DwtError):
        plan.forward(xq, scale=0.0)
    with pytest.raises(D.DwtError):
        D.Plan(64, 64, 2, "cdf97", "nonsep_multipass", torch.float16)
