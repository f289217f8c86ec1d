"""Helpers shared by the GPU parity tests (compare against the FP64 oracle)."""
import numpy as np
import torch

from oracle import lifting as L
from paper_1705_08266_gb300 import dwt2d as D
from paper_1705_08266_gb300 import synth

# Tolerance for float32 CDF 9/7: per level, max |gpu - oracle| over that level's
# bands <= TOL_F32 * max|x| (the image's own magnitude).
TOL_F32 = 1e-5


def device_image(x: np.ndarray) -> torch.Tensor:
    t = D.empty_image(x.shape[0], x.shape[1], torch.from_numpy(x).dtype, "cuda")
    t.copy_(torch.from_numpy(x))
    return t


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def make_input(wavelet: str, h: int, w: int, seed: int) -> np.ndarray:
    return synth.image(wavelet, h, w, seed)


def per_level_errors(got: np.ndarray, ref: np.ndarray, levels: int):
    """{level: max abs error over the bands of that level} (LL counts for the last level)."""
    g = L.band_views(got.astype(np.float64), levels)
    r = L.band_views(ref.astype(np.float64), levels)
    out = {}
    for key in r:
        lvl = key[0]
        e = float(np.max(np.abs(g[key] - r[key]))) if r[key].size else 0.0
        out[lvl] = max(out.get(lvl, 0.0), e)
    return out


def assert_forward_matches(got: np.ndarray, x: np.ndarray, levels: int, wavelet: str, what=""):
    ref = L.forward(x, levels, wavelet)
    if wavelet == "legall53":
        assert got.dtype == np.int32
        bad = np.argwhere(got.astype(np.int64) != ref)
        assert bad.size == 0, f"{what}: {len(bad)} mismatches, first at {bad[:5].tolist()}"
        return
    maxabs = float(np.max(np.abs(x)))
    errs = per_level_errors(got, ref, levels)
    for lvl, e in errs.items():
        assert e <= TOL_F32 * maxabs, f"{what}: level {lvl} max err {e:.3g} > {TOL_F32 * maxabs:.3g}"


def assert_inverse_matches(got: np.ndarray, coeffs: np.ndarray, levels: int, wavelet: str, x,
                           what=""):
    ref = L.inverse(coeffs, levels, wavelet)
    if wavelet == "legall53":
        bad = np.argwhere(got.astype(np.int64) != ref)
        assert bad.size == 0, f"{what}: {len(bad)} mismatches, first at {bad[:5].tolist()}"
        return
    # the inverse's one output is the image: the same 1e-5 max|x| bound as each forward level
    maxabs = float(np.max(np.abs(x)))
    e = float(np.max(np.abs(got.astype(np.float64) - ref)))
    assert e <= TOL_F32 * maxabs, f"{what}: inverse max err {e:.3g} > {TOL_F32 * maxabs:.3g}"
