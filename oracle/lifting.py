"""O1 / O3: separable lifting, written out step by step (test infrastructure only).

Paper: Barina et al., arXiv 1705.08266.

* Sec. 2, Eq. 2: the polyphase matrix of a wavelet filter bank factors into
  pairs of lifting steps, a predict P followed by an update U.
* Sec. 2, separable lifting scheme ``S_U^V | S_U^H | T_P^V | T_P^H``: for every
  (P, U) pair the 2-D transform runs, in this order, the horizontal predict
  T_P^H, the vertical predict T_P^V, the horizontal update S_U^H and the
  vertical update S_U^V ("M2 | M1" means M1 runs first).  Predicts always
  precede updates.
* Sec. 2, the 2-D transform splits the image into a quadruple of polyphase
  components; here c0 = x[2r, 2c], c1 = x[2r, 2c+1], c2 = x[2r+1, 2c],
  c3 = x[2r+1, 2c+1], consistent with T_P^H updating components 1 and 3 from
  components 0 and 2.

Readings where the paper is silent:

* Lifting filters: predict P = p (1 + z) reads the even sample at i and i+1,
  update U = u (1 + z^-1) reads the odd sample at i-1 and i.  CDF 9/7 uses
  the Daubechies-Sweldens pairs (alpha, beta), (gamma, delta) and a final
  scaling low / K, high * K on every active axis (DC gain 1 for the low
  pass, Nyquist gain 2 for the high pass).  Linear 5/3 uses (-1/2, 1/4)
  with no scaling.
* Boundary: whole-sample symmetric extension of the full-rate signal:
  x[-j] = x[j], x[N-1+j] = x[N-1-j].  In the polyphase domain this makes
  odd[-1] = odd[0], even[ne] = even[ne-1] (N even) and odd[no] = odd[no-1]
  (N odd); the symmetric lifting filters keep every intermediate signal
  symmetric, so mirroring before each step is exact (pinned by lifting ==
  convolution in the tests).
* Odd lengths: even-indexed samples are low pass, so the low band has
  ceil(N/2) samples and the high band floor(N/2).  An axis of length 1 is
  left unchanged (no lifting, no scaling).
* Reversible integer 5/3 (O3): d = x_odd - floor((e_i + e_{i+1}) / 2),
  s = x_even + floor((d_{i-1} + d_i + 2) / 4), floors toward -inf, in the
  same T^H, T^V, S^H, S^V order (with floors the order changes the result;
  the paper's interleaved order is the definition).
* Multilevel: Mallat recursion on LL with the same rules at every level; the
  result is stored in the Mallat layout, LL top-left (ceil(H/2) x ceil(W/2)),
  HL top-right, LH bottom-left, HH bottom-right.
"""
from __future__ import annotations

import numpy as np

# Daubechies-Sweldens lifting constants of CDF 9/7 (the paper cites the
# factorisation of Daubechies & Sweldens for Eq. 2 but prints no values).
ALPHA = -1.586134342059924
BETA = -0.052980118572961
GAMMA = 0.882911075530934
DELTA = 0.443506852043971
K97 = 1.230174104914001

CDF97_PAIRS = ((ALPHA, BETA), (GAMMA, DELTA))
LINEAR53_PAIRS = ((-0.5, 0.25),)

WAVELETS = ("cdf97", "linear53", "legall53")


# ---------------------------------------------------------------------------
# 1-D lifting steps along one axis of an array (..., H, W); axis is -1
# (horizontal, the paper's z_m) or -2 (vertical, z_n).  Each call mirrors the
# neighbours it reads (whole-sample symmetric extension) and updates in place.
# ---------------------------------------------------------------------------

def _polyphase(a: np.ndarray, axis: int):
    v = np.moveaxis(a, axis, -1)
    return v[..., 0::2], v[..., 1::2]


def _even_next(even: np.ndarray, no: int) -> np.ndarray:
    """even[i + 1] for i = 0 .. no-1, mirrored (even[ne] = even[ne-1] if N is even)."""
    if even.shape[-1] > no:  # N odd: even[no] exists
        return even[..., 1:no + 1]
    return np.concatenate([even[..., 1:], even[..., -1:]], axis=-1)


def _odd_prev_cur(odd: np.ndarray, ne: int):
    """(odd[i - 1], odd[i]) for i = 0 .. ne-1, mirrored (odd[-1] = odd[0]; odd[no] = odd[no-1])."""
    no = odd.shape[-1]
    cur = odd if no == ne else np.concatenate([odd, odd[..., -1:]], axis=-1)
    prev = np.concatenate([odd[..., :1], odd[..., :ne - 1]], axis=-1)
    return prev, cur


def predict(a: np.ndarray, p: float, axis: int) -> None:
    """T_P along `axis`: odd[i] += p * (even[i] + even[i+1])  (P = p (1 + z))."""
    if a.shape[axis] < 2:
        return
    even, odd = _polyphase(a, axis)
    no = odd.shape[-1]
    odd += p * (even[..., :no] + _even_next(even, no))


def update(a: np.ndarray, u: float, axis: int) -> None:
    """S_U along `axis`: even[i] += u * (odd[i-1] + odd[i])  (U = u (1 + z^-1))."""
    if a.shape[axis] < 2:
        return
    even, odd = _polyphase(a, axis)
    prev, cur = _odd_prev_cur(odd, even.shape[-1])
    even += u * (prev + cur)


def predict_int53(a: np.ndarray, axis: int, sign: int = 1) -> None:
    """Reversible 5/3 predict: odd[i] -= floor((even[i] + even[i+1]) / 2).

    sign = -1 undoes it (odd[i] += the same floor).
    """
    if a.shape[axis] < 2:
        return
    even, odd = _polyphase(a, axis)
    no = odd.shape[-1]
    odd -= sign * np.floor_divide(even[..., :no] + _even_next(even, no), 2)


def update_int53(a: np.ndarray, axis: int, sign: int = 1) -> None:
    """Reversible 5/3 update: even[i] += floor((odd[i-1] + odd[i] + 2) / 4).

    sign = -1 undoes it.
    """
    if a.shape[axis] < 2:
        return
    even, odd = _polyphase(a, axis)
    prev, cur = _odd_prev_cur(odd, even.shape[-1])
    even += sign * np.floor_divide(prev + cur + 2, 4)


def _scale(a: np.ndarray, k: float, axis: int) -> None:
    """Low / k, high * k along `axis` (skipped for an axis of length 1)."""
    if a.shape[axis] < 2:
        return
    even, odd = _polyphase(a, axis)
    even *= 1.0 / k
    odd *= k


# ---------------------------------------------------------------------------
# One level of the 2-D transform, in place on the interleaved image.
# ---------------------------------------------------------------------------

H_AXIS, V_AXIS = -1, -2


def lift2d_forward_interleaved(a: np.ndarray, wavelet: str) -> None:
    """One level, separable lifting in the paper's order T^H, T^V, S^H, S^V per pair."""
    if wavelet == "legall53":
        predict_int53(a, H_AXIS)
        predict_int53(a, V_AXIS)
        update_int53(a, H_AXIS)
        update_int53(a, V_AXIS)
        return
    pairs = CDF97_PAIRS if wavelet == "cdf97" else LINEAR53_PAIRS
    for p, u in pairs:
        predict(a, p, H_AXIS)
        predict(a, p, V_AXIS)
        update(a, u, H_AXIS)
        update(a, u, V_AXIS)
    if wavelet == "cdf97":
        _scale(a, K97, H_AXIS)
        _scale(a, K97, V_AXIS)


def lift2d_inverse_interleaved(a: np.ndarray, wavelet: str) -> None:
    """Exact inverse of lift2d_forward_interleaved: every step undone in reverse order."""
    if wavelet == "legall53":
        update_int53(a, V_AXIS, sign=-1)
        update_int53(a, H_AXIS, sign=-1)
        predict_int53(a, V_AXIS, sign=-1)
        predict_int53(a, H_AXIS, sign=-1)
        return
    pairs = CDF97_PAIRS if wavelet == "cdf97" else LINEAR53_PAIRS
    if wavelet == "cdf97":
        _scale(a, 1.0 / K97, V_AXIS)
        _scale(a, 1.0 / K97, H_AXIS)
    for p, u in reversed(pairs):
        update(a, -u, V_AXIS)
        update(a, -u, H_AXIS)
        predict(a, -p, V_AXIS)
        predict(a, -p, H_AXIS)


def band_shapes(h: int, w: int):
    """(LL, HL, LH, HH) shapes of one level of an h x w image."""
    he, ho, we, wo = (h + 1) // 2, h // 2, (w + 1) // 2, w // 2
    return (he, we), (he, wo), (ho, we), (ho, wo)


def deinterleave(a: np.ndarray) -> np.ndarray:
    """Interleaved quadruples -> Mallat layout (LL | HL over LH | HH)."""
    h, w = a.shape[-2:]
    he, we = (h + 1) // 2, (w + 1) // 2
    out = np.empty_like(a)
    out[..., :he, :we] = a[..., 0::2, 0::2]
    out[..., :he, we:] = a[..., 0::2, 1::2]
    out[..., he:, :we] = a[..., 1::2, 0::2]
    out[..., he:, we:] = a[..., 1::2, 1::2]
    return out


def interleave(m: np.ndarray) -> np.ndarray:
    """Mallat layout -> interleaved quadruples (inverse of deinterleave)."""
    h, w = m.shape[-2:]
    he, we = (h + 1) // 2, (w + 1) // 2
    a = np.empty_like(m)
    a[..., 0::2, 0::2] = m[..., :he, :we]
    a[..., 0::2, 1::2] = m[..., :he, we:]
    a[..., 1::2, 0::2] = m[..., he:, :we]
    a[..., 1::2, 1::2] = m[..., he:, we:]
    return a


def _work_dtype(wavelet: str):
    if wavelet not in WAVELETS:
        raise ValueError(f"unknown wavelet {wavelet!r}")
    return np.int64 if wavelet == "legall53" else np.float64


def level_sizes(h: int, w: int, levels: int):
    """[(H_0, W_0), (H_1, W_1), ...]: the extent each level transforms."""
    sizes = []
    for _ in range(levels):
        sizes.append((h, w))
        h, w = (h + 1) // 2, (w + 1) // 2
    return sizes


def forward(x: np.ndarray, levels: int, wavelet: str) -> np.ndarray:
    """Multilevel 2-D forward DWT (Mallat layout), FP64 (int64 for legall53).

    x has shape (..., H, W).  Level l transforms the top-left LL of level l-1.
    """
    if levels < 1:
        raise ValueError("levels must be >= 1")
    out = np.array(x, dtype=_work_dtype(wavelet), copy=True)
    if wavelet == "legall53" and not np.issubdtype(np.asarray(x).dtype, np.integer):
        raise TypeError("legall53 takes integer input")
    for h, w in level_sizes(*out.shape[-2:], levels):
        sub = out[..., :h, :w].copy()
        lift2d_forward_interleaved(sub, wavelet)
        out[..., :h, :w] = deinterleave(sub)
    return out


def inverse(c: np.ndarray, levels: int, wavelet: str) -> np.ndarray:
    """Inverse of forward(): coarse to fine."""
    if levels < 1:
        raise ValueError("levels must be >= 1")
    out = np.array(c, dtype=_work_dtype(wavelet), copy=True)
    for h, w in reversed(level_sizes(*out.shape[-2:], levels)):
        sub = interleave(out[..., :h, :w])
        lift2d_inverse_interleaved(sub, wavelet)
        out[..., :h, :w] = sub
    return out


def forward_per_level(x: np.ndarray, levels: int, wavelet: str):
    """Like forward(), also returning the Mallat array after each level (for per-level errors)."""
    out = np.array(x, dtype=_work_dtype(wavelet), copy=True)
    snaps = []
    for h, w in level_sizes(*out.shape[-2:], levels):
        sub = out[..., :h, :w].copy()
        lift2d_forward_interleaved(sub, wavelet)
        out[..., :h, :w] = deinterleave(sub)
        snaps.append(out.copy())
    return snaps


def band_views(m: np.ndarray, levels: int):
    """{(level, band): view} of a Mallat-layout array; band in LL, HL, LH, HH (LL only at the last level)."""
    views = {}
    sizes = level_sizes(*m.shape[-2:], levels)
    for lvl, (h, w) in enumerate(sizes, start=1):
        he, we = (h + 1) // 2, (w + 1) // 2
        views[(lvl, "HL")] = m[..., :he, we:w]
        views[(lvl, "LH")] = m[..., he:h, :we]
        views[(lvl, "HH")] = m[..., he:h, we:w]
        if lvl == levels:
            views[(lvl, "LL")] = m[..., :he, :we]
    return views


def sample_coefficient(x: np.ndarray, levels: int, wavelet: str, r: int, c: int) -> float:
    """One output coefficient of forward(x) at Mallat position (r, c), from a bounded input window.

    The forward transform is a local stencil: the coefficient at a Mallat
    position depends only on input pixels inside a window around its spatial
    footprint.  This evaluates forward() on the smallest aligned crop of x
    that both contains that window and keeps every image border that the
    window touches (so symmetric extension is the same as in the full
    image); far from a border, the crop's own border is outside the
    coefficient's dependency cone and cannot influence it.
    """
    h, w = x.shape[-2:]
    sizes = level_sizes(h, w, levels)
    # locate (level, band, band row, band col) of the Mallat position
    lvl = None
    for l, (hl, wl) in enumerate(sizes, start=1):
        he, we = (hl + 1) // 2, (wl + 1) // 2
        if r < hl and c < wl and (r >= he or c >= we or l == levels):
            lvl, br, bc = l, r if r < he else r - he, c if c < we else c - we
            band_r_odd, band_c_odd = r >= he, c >= we
            break
    if lvl is None:
        raise ValueError("position is not a coefficient")
    scale = 1 << lvl
    # support radius of one level in that level's own samples, 9/7 is the widest
    rad = 4 if wavelet == "cdf97" else 2
    # cone at input resolution: sum of the radii of every level, plus one quad
    margin = sum(rad << l for l in range(lvl)) + 2 * scale
    y0 = br * scale - margin
    x0 = bc * scale - margin
    y1 = (br + 1) * scale + margin
    x1 = (bc + 1) * scale + margin
    # keep the real border if the window crosses it; else align the crop to the level grid
    cy0 = 0 if y0 <= 0 else (y0 // scale) * scale
    cx0 = 0 if x0 <= 0 else (x0 // scale) * scale
    cy1 = h if y1 >= h else min(h, -(-y1 // scale) * scale)
    cx1 = w if x1 >= w else min(w, -(-x1 // scale) * scale)
    crop = np.asarray(x[..., cy0:cy1, cx0:cx1])
    sub = forward(crop, lvl, wavelet)
    csz = level_sizes(cy1 - cy0, cx1 - cx0, lvl)
    ch, cw = csz[-1]
    che, cwe = (ch + 1) // 2, (cw + 1) // 2
    rr = br - cy0 // scale
    cc = bc - cx0 // scale
    if band_r_odd:
        rr += che
    if band_c_odd:
        cc += cwe
    return sub[..., rr, cc]
