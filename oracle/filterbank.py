"""O2: the convolution filter bank, derived in closed form (test infrastructure only).

Paper: Barina et al., arXiv 1705.08266, Sec. 2, Eq. 1: a single-scale DWT is a
pair of filters G0 (low pass) and G1 (high pass) followed by subsampling by two;
Eq. 2 (lifting) is a factorisation of the same polyphase matrix.  This module
computes the Eq. 1 side independently of the lifting constants, so that the
two can be checked against each other.

Taps come from the Daubechies half-band product filter, not from a table.
With y = sin^2(w/2) = (2 - z - z^-1)/4 and cos^2(w/2) = 1 - y, the
biorthogonal CDF family with 2N vanishing moments splits

    P(y) = (1 - y)^N * Q_N(y),   Q_N(y) = sum_{k<N} C(N-1+k, k) y^k,

between an analysis low pass h and a synthesis low pass ht.  For CDF 9/7
(N = 4, Q = 1 + 4y + 10y^2 + 20y^3) h takes (1-y)^2 and the complex pair of
roots of Q (9 taps), ht takes (1-y)^2 and the real root (7 taps).  For the
linear 5/3 (N = 2, Q = 1 + 2y) h takes (1-y) and the root of Q (5 taps), ht
takes (1-y) (3 taps).  Both low passes are normalised to unit DC gain; the
analysis high pass is g[k] = 2 (-1)^k ht[k] (k centred at 0), which has
Nyquist gain 2.  These are the normalisations the lifting oracle uses (low
/ K, high * K for 9/7).

low[n]  = sum_k h[k] x~[2n + k]
high[n] = sum_k g[k] x~[2n + 1 + k]

with x~ the whole-sample symmetric extension of x (x[-j] = x[j],
x[N-1+j] = x[N-1-j]).  A signal of length 1 passes unchanged.
"""
from __future__ import annotations

from math import comb

import numpy as np
from numpy.polynomial import polynomial as P


def _y_poly_to_taps(ycoef) -> np.ndarray:
    """Coefficients of a polynomial in y -> symmetric taps in z (centred, odd length)."""
    # y = (2 - z - z^-1)/4 as a Laurent polynomial; represent z-powers -d..d as an array
    deg = len(ycoef) - 1
    size = 2 * deg + 1
    acc = np.zeros(size, dtype=np.complex128)
    ypow = np.zeros(size, dtype=np.complex128)
    ypow[deg] = 1.0  # y^0
    y1 = np.array([-0.25, 0.5, -0.25])  # coefficients of z^-1, z^0, z^1
    for k, a in enumerate(ycoef):
        acc += a * ypow
        if k < deg:
            ypow = _shift_conv(ypow, y1)
    taps = acc.real
    if np.max(np.abs(acc.imag)) > 1e-12:
        raise ArithmeticError("taps are not real")
    return taps


def _shift_conv(a: np.ndarray, b3: np.ndarray) -> np.ndarray:
    """Multiply a centred Laurent polynomial by a 3-tap centred one, keeping the array size."""
    full = np.convolve(a, b3)  # length len(a) + 2
    return full[1:-1]


def _halfband_factor(n: int):
    """Q_N(y) coefficients (ascending) of the Daubechies half-band product filter."""
    return np.array([comb(n - 1 + k, k) for k in range(n)], dtype=np.float64)


def cdf_taps(wavelet: str):
    """(h, g): analysis low pass (centred, odd length) and analysis high pass (centred)."""
    if wavelet == "cdf97":
        n = 4
    elif wavelet in ("linear53", "legall53"):
        n = 2
    else:
        raise ValueError(wavelet)
    q = _halfband_factor(n)
    roots = P.polyroots(q)
    real = [r for r in roots if abs(r.imag) < 1e-12]
    cplx = [r for r in roots if abs(r.imag) >= 1e-12]
    one_minus_y = np.array([1.0, -1.0])
    half = P.polypow(one_minus_y, n // 2)
    if n == 4:
        # h: complex pair, ht: real root
        h_y = half.astype(np.complex128)
        for r in cplx:
            h_y = P.polymul(h_y, np.array([1.0, -1.0 / r]))
        ht_y = half.astype(np.complex128)
        for r in real:
            ht_y = P.polymul(ht_y, np.array([1.0, -1.0 / r]))
    else:
        h_y = half.astype(np.complex128)
        for r in real:
            h_y = P.polymul(h_y, np.array([1.0, -1.0 / r]))
        ht_y = half.astype(np.complex128)
    h = _y_poly_to_taps(h_y)
    ht = _y_poly_to_taps(ht_y)
    h = h / h.sum()
    ht = ht / ht.sum()
    c = len(ht) // 2
    g = np.array([2.0 * (-1.0) ** (k - c) * ht[k] for k in range(len(ht))])
    return h, g


def _mirror(j: np.ndarray, n: int) -> np.ndarray:
    """Whole-sample symmetric index map (repeated, so any j maps into [0, n))."""
    if n == 1:
        return np.zeros_like(j)
    period = 2 * (n - 1)
    j = np.mod(j, period)
    return np.where(j >= n, period - j, j)


def analysis_1d(x: np.ndarray, wavelet: str, axis: int = -1):
    """(low, high) along `axis` by convolution + subsampling (Eq. 1)."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    n = x.shape[-1]
    if n == 1:
        return np.moveaxis(x.copy(), -1, axis), np.moveaxis(x[..., :0].copy(), -1, axis)
    h, g = cdf_taps(wavelet)
    rh, rg = len(h) // 2, len(g) // 2
    ne, no = (n + 1) // 2, n // 2
    low = np.zeros(x.shape[:-1] + (ne,))
    high = np.zeros(x.shape[:-1] + (no,))
    ln = np.arange(ne)
    hn = np.arange(no)
    for k in range(-rh, rh + 1):
        low += h[k + rh] * x[..., _mirror(2 * ln + k, n)]
    for k in range(-rg, rg + 1):
        high += g[k + rg] * x[..., _mirror(2 * hn + 1 + k, n)]
    return np.moveaxis(low, -1, axis), np.moveaxis(high, -1, axis)


def forward_2d_single(x: np.ndarray, wavelet: str) -> np.ndarray:
    """One level of the separable convolution scheme N^V | N^H (Mallat layout)."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = analysis_1d(x, wavelet, axis=-1)
    ll, lh = analysis_1d(lo, wavelet, axis=-2)
    hl, hh = analysis_1d(hi, wavelet, axis=-2)
    he, we = ll.shape[-2], ll.shape[-1]
    out = np.empty(x.shape, dtype=np.float64)
    out[..., :he, :we] = ll
    out[..., :he, we:] = hl
    out[..., he:, :we] = lh
    out[..., he:, we:] = hh
    return out


def forward(x: np.ndarray, levels: int, wavelet: str) -> np.ndarray:
    """Multilevel separable convolution (Mallat recursion on LL)."""
    out = np.array(x, dtype=np.float64, copy=True)
    h, w = out.shape[-2:]
    for _ in range(levels):
        out[..., :h, :w] = forward_2d_single(out[..., :h, :w], wavelet)
        h, w = (h + 1) // 2, (w + 1) // 2
    return out
