"""Parity at the benchmark's full size (8192 x 8192, 5 levels), in the launch
configuration bench.py times.

Every scheme: forward coefficients sampled at band corners, band edges and
random positions, each recomputed by the oracle from its dependency window
(oracle.lifting.sample_coefficient); and the GPU round trip.  The headline
scheme (non-separable reduced, CDF 9/7) and the 5/3 scheme are also compared
element by element against the full FP64 oracle, forward and inverse (the
inverse of the oracle's own coefficients against the oracle's inverse).
"""
import numpy as np
import pytest
import torch

from oracle import lifting as L
from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import synth
from tests.parity_util import TOL_F32, device_image, per_level_errors

pytestmark = pytest.mark.gpu

H = W = 8192
LEVELS = 5


@pytest.fixture(scope="module")
def images():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return {w: synth.image(w, H, W, synth.SEED_LARGE) for w in ("cdf97", "legall53")}


def _positions(rng):
    pos = []
    sizes = L.level_sizes(H, W, LEVELS)
    for lvl, (h, w) in enumerate(sizes, start=1):
        he, we = (h + 1) // 2, (w + 1) // 2
        bands = [(0, we, he, w), (he, 0, h, we), (he, we, h, w)]
        if lvl == LEVELS:
            bands.append((0, 0, he, we))
        for r0, c0, r1, c1 in bands:
            pos += [(r0, c0), (r0, c1 - 1), (r1 - 1, c0), (r1 - 1, c1 - 1)]
            pos += [(r0, (c0 + c1) // 2), (r1 - 1, (c0 + c1) // 2), ((r0 + r1) // 2, c0),
                    ((r0 + r1) // 2, c1 - 1)]
            for _ in range(8):
                pos.append((int(rng.integers(r0, r1)), int(rng.integers(c0, c1))))
    return pos


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
@pytest.mark.parametrize("scheme", list(D.SCHEMES))
def test_fullsize_sampled_and_round_trip(images, wavelet, scheme):
    if wavelet == "legall53" and scheme == "separable_convolution":
        pytest.skip("the convolution scheme is the linear CDF 9/7 filter bank")
    x = images[wavelet]
    plan = D.Plan(H, W, LEVELS, wavelet, scheme)
    ws = plan.workspace()
    xd = device_image(x)
    c = plan.forward(xd, workspace=ws)
    y = plan.inverse(c, workspace=ws)
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    ch = c.cpu().numpy()
    maxabs = float(np.max(np.abs(x)))
    rng = np.random.default_rng(8266)
    for r, cc in _positions(rng):
        ref = L.sample_coefficient(x, LEVELS, wavelet, r, cc)
        if wavelet == "legall53":
            assert int(ch[r, cc]) == int(ref), (scheme, r, cc)
        else:
            assert abs(float(ch[r, cc]) - float(ref)) <= TOL_F32 * maxabs, (scheme, r, cc)
    yh = y.cpu().numpy()
    if wavelet == "legall53":
        assert np.array_equal(yh, x), scheme
    else:
        assert float(np.max(np.abs(yh - x))) <= 2 * LEVELS * TOL_F32 * maxabs, scheme


@pytest.mark.parametrize("wavelet,scheme", [("cdf97", "nonsep_reduced"), ("legall53", "nonsep")])
def test_fullsize_elementwise(images, wavelet, scheme):
    x = images[wavelet]
    plan = D.Plan(H, W, LEVELS, wavelet, scheme)
    c = plan.forward(device_image(x)).cpu().numpy()
    ref = L.forward(x, LEVELS, wavelet)
    if wavelet == "legall53":
        assert np.array_equal(c.astype(np.int64), ref)
    else:
        maxabs = float(np.max(np.abs(x)))
        for lvl, e in per_level_errors(c, ref, LEVELS).items():
            assert e <= TOL_F32 * maxabs, (lvl, e)


@pytest.mark.parametrize("wavelet,scheme", [("cdf97", "nonsep_reduced"), ("legall53", "nonsep")])
def test_fullsize_inverse_elementwise(images, wavelet, scheme):
    """GPU inverse of the oracle's coefficients == oracle inverse (Eq. 2 undone, coarse to fine)."""
    x = images[wavelet]
    coeffs = L.forward(x, LEVELS, wavelet).astype(x.dtype)  # what the GPU is given
    ref = L.inverse(coeffs, LEVELS, wavelet)
    plan = D.Plan(H, W, LEVELS, wavelet, scheme)
    ws = plan.workspace()
    cd = device_image(coeffs)
    y = plan.inverse(cd, workspace=ws)
    torch.cuda.synchronize()
    assert plan.status(ws) == 0
    yh = y.cpu().numpy()
    if wavelet == "legall53":
        assert np.array_equal(yh.astype(np.int64), ref)
    else:
        # the inverse's one output is held to the forward's per-level bound
        maxabs = float(np.max(np.abs(x)))
        assert float(np.max(np.abs(yh.astype(np.float64) - ref))) <= TOL_F32 * maxabs
