"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here touches the CUDA path.  Each test names the passage it follows
(Barina et al., arXiv 1705.08266).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import filterbank as FB
from oracle import lifting as L
from oracle import operators as O
from paper_1705_08266_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Eq. 1 side: the closed-form filter bank ---------------------------------

@pytest.mark.parametrize("wavelet,nh,ng", [("cdf97", 9, 7), ("linear53", 5, 3)])
def test_taps_shape_and_gains(wavelet, nh, ng):
    h, g = FB.cdf_taps(wavelet)
    assert len(h) == nh and len(g) == ng
    assert np.allclose(h, h[::-1]) and np.allclose(g, g[::-1])
    assert abs(h.sum() - 1.0) < 1e-14                       # DC gain 1
    k = np.arange(len(g)) - len(g) // 2
    assert abs(np.sum(g * (-1.0) ** k) - 2.0) < 1e-13        # Nyquist gain 2
    assert abs(g.sum()) < 1e-14                              # high pass kills DC


@pytest.mark.parametrize("wavelet", ["cdf97", "linear53"])
def test_filter_bank_is_perfect_reconstruction(wavelet):
    """Biorthogonality: the product of analysis and synthesis low passes is half-band.

    With ht recovered from g (g[k] = 2 (-1)^k ht[k]), the product filter
    Pz = H(z) Ht(z) must satisfy Pz(z) + Pz(-z) = 2 c, i.e. its even taps
    vanish except the centre one (Eq. 1 has an inverse).
    """
    h, g = FB.cdf_taps(wavelet)
    k = np.arange(len(g)) - len(g) // 2
    ht = g * (-1.0) ** k / 2.0
    prod = np.convolve(h, ht)
    c = len(prod) // 2
    even = prod[c % 2::2]
    centre = prod[c]
    others = np.array([v for i, v in enumerate(prod) if (i - c) % 2 == 0 and i != c])
    assert np.max(np.abs(others)) < 1e-14
    assert centre > 0
    assert len(even) > 1


def test_vanishing_moments_of_high_pass():
    """CDF 9/7 high pass kills polynomials of degree <= 3, linear 5/3 of degree <= 1."""
    for wavelet, order in (("cdf97", 4), ("linear53", 2)):
        _, g = FB.cdf_taps(wavelet)
        k = np.arange(len(g)) - len(g) // 2
        for d in range(order):
            assert abs(np.sum(g * k.astype(float) ** d)) < 1e-12, (wavelet, d)
        assert abs(np.sum(g * k.astype(float) ** order)) > 1e-3, (wavelet, order)


# --- Eq. 2 side: lifting == convolution -------------------------------------

def _lift1d(x, wavelet):
    a = np.array(x, dtype=np.float64)
    pairs = L.CDF97_PAIRS if wavelet == "cdf97" else L.LINEAR53_PAIRS
    for p, u in pairs:
        L.predict(a, p, -1)
        L.update(a, u, -1)
    if wavelet == "cdf97":
        L._scale(a, L.K97, -1)
    return a[..., 0::2], a[..., 1::2]


@pytest.mark.parametrize("wavelet", ["cdf97", "linear53"])
def test_lifting_equals_convolution_1d(wavelet):
    """Eq. 1 and Eq. 2 are the same transform, at every length, borders included."""
    rng = np.random.default_rng(11)
    for n in range(1, 41):
        x = rng.standard_normal((4, n)) * 100
        lo, hi = _lift1d(x, wavelet)
        clo, chi = FB.analysis_1d(x, wavelet)
        assert np.max(np.abs(lo - clo)) <= 1e-12 * 100, n
        if n > 1:
            assert np.max(np.abs(hi - chi)) <= 1e-12 * 100, n


@pytest.mark.parametrize("wavelet", ["cdf97", "linear53"])
@pytest.mark.parametrize("shape,levels", [((8, 8), 1), ((7, 9), 2), ((33, 17), 3),
                                          ((64, 48), 4), ((2, 2), 1), ((1, 9), 2), ((9, 1), 2)])
def test_lifting_equals_convolution_2d(wavelet, shape, levels):
    """Separable lifting S^V|S^H|T^V|T^H == separable convolution N^V|N^H, Mallat recursion."""
    x = synth.gradient_noise(*shape, seed=3).astype(np.float64)
    a = L.forward(x, levels, wavelet)
    b = FB.forward(x, levels, wavelet)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(x))


# --- perfect reconstruction --------------------------------------------------

@pytest.mark.parametrize("wavelet", ["cdf97", "linear53"])
@pytest.mark.parametrize("shape,levels", [((8, 8), 3), ((7, 9), 3), ((65, 31), 5), ((1, 1), 2)])
def test_perfect_reconstruction_float(wavelet, shape, levels):
    x = synth.gradient_noise(*shape, seed=5).astype(np.float64)
    c = L.forward(x, levels, wavelet)
    y = L.inverse(c, levels, wavelet)
    assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("shape,levels", [((8, 8), 3), ((7, 9), 3), ((65, 31), 6), ((2, 1), 1)])
def test_perfect_reconstruction_int(shape, levels):
    x = synth.uniform_int(*shape, seed=6)
    c = L.forward(x, levels, "legall53")
    assert c.dtype == np.int64
    y = L.inverse(c, levels, "legall53")
    assert np.array_equal(x, y)


def test_int53_exhaustive_3x3():
    """Every 3x3 image over {0, 1, 4095}: the reversible 5/3 round-trips exactly."""
    vals = np.array([0, 1, 4095], dtype=np.int64)
    imgs = np.array(list(itertools.product(vals, repeat=9)), dtype=np.int64).reshape(-1, 3, 3)
    for levels in (1, 2):
        c = L.forward(imgs, levels, "legall53")
        assert np.array_equal(L.inverse(c, levels, "legall53"), imgs)


# --- vanishing moments, DC gain ----------------------------------------------

@pytest.mark.parametrize("wavelet", ["cdf97", "legall53", "linear53"])
def test_constant_image(wavelet):
    """Constant image: every detail band is zero at every level and LL keeps the value (DC gain 1)."""
    levels = 4
    val = 100 if wavelet == "legall53" else 100.0
    x = np.full((37, 50), val, dtype=np.int32 if wavelet == "legall53" else np.float64)
    c = L.forward(x, levels, wavelet)
    for (lvl, band), v in L.band_views(c, levels).items():
        if band == "LL":
            assert np.max(np.abs(v - val)) < 1e-10
        else:
            assert np.max(np.abs(v)) < 1e-10, (lvl, band)


def _interior(v, margin):
    return v[..., margin:v.shape[-2] - margin, margin:v.shape[-1] - margin]


@pytest.mark.parametrize("wavelet", ["cdf97", "legall53", "linear53"])
def test_linear_ramp_interior_details_vanish(wavelet):
    """Ramp x = 3c + 5r: zero detail away from the borders (both wavelets have >= 2 moments).

    Mirroring a ramp makes a kink at the border, so coefficients within the
    filter support of an edge are excluded.
    """
    levels = 3
    if wavelet == "legall53":
        x = synth.ramp(96, 80, a=4, b=8, dtype=np.int32)
    else:
        x = synth.ramp(96, 80, dtype=np.float64)
    c = L.forward(x, levels, wavelet)
    for (lvl, band), v in L.band_views(c, levels).items():
        if band != "LL":
            assert np.max(np.abs(_interior(v, 4))) < 1e-9, (lvl, band)


def test_cubic_separates_97_from_53():
    """A cubic in c is annihilated by the 9/7 high pass (4 moments) but not by 5/3 (2)."""
    cc = np.arange(64, dtype=np.float64)
    x = np.tile(((cc - 30.0) / 8.0) ** 3, (16, 1))
    for wavelet, zero in (("cdf97", True), ("linear53", False)):
        c = L.forward(x, 1, wavelet)
        hl = L.band_views(c, 1)[(1, "HL")]
        inner = np.max(np.abs(hl[:, 4:-4]))
        assert (inner < 1e-9) == zero, (wavelet, inner)


# --- the paper's matrices (Sec. 2, Sec. 3) -----------------------------------

SIZES = [(8, 8), (7, 9), (9, 7), (5, 5), (2, 2), (3, 3), (2, 5), (6, 4)]


@pytest.mark.parametrize("h,w", SIZES)
def test_nonseparable_equals_separable_operators(h, w):
    """T_P = T_P^V T_P^H and S_U = S_U^V S_U^H (Sec. 3), mirrored borders included."""
    P, U = O.predict_filter(L.ALPHA), O.update_filter(L.BETA)
    TH, TV = O.operator(O.T_H(P), h, w), O.operator(O.T_V(P), h, w)
    SH, SV = O.operator(O.S_H(U), h, w), O.operator(O.S_V(U), h, w)
    assert np.max(np.abs(O.operator(O.T_nonsep(P), h, w) - TV @ TH)) < 1e-14
    assert np.max(np.abs(O.operator(O.S_nonsep(U), h, w) - SV @ SH)) < 1e-14
    # horizontal and vertical steps commute (Sec. 2, linear filters)
    assert np.max(np.abs(TV @ TH - TH @ TV)) < 1e-14
    assert np.max(np.abs(SV @ SH - SH @ SV)) < 1e-14


@pytest.mark.parametrize("h,w", SIZES)
def test_reduced_split_equals_nonseparable(h, w):
    """P = P0 + P1: the P1 part non-separably, then the P0 part separably, is T_P (Sec. 3)."""
    P, U = O.predict_filter(L.GAMMA), O.update_filter(L.DELTA)
    op = lambda m: O.operator(m, h, w)
    T_red = op(O.T_V(O.split0(P))) @ op(O.T_H(O.split0(P))) @ op(O.T_nonsep(O.split1(P)))
    S_red = op(O.S_V(O.split0(U))) @ op(O.S_H(O.split0(U))) @ op(O.S_nonsep(O.split1(U)))
    assert np.max(np.abs(T_red - op(O.T_nonsep(P)))) < 1e-14
    assert np.max(np.abs(S_red - op(O.S_nonsep(U)))) < 1e-14


@pytest.mark.parametrize("h,w", SIZES)
def test_oracle_matches_paper_matrices_impulses(h, w):
    """The oracle's lifting on every impulse == the product of the paper's matrices.

    One CDF 9/7 level: per pair S^V S^H T^V T^H, then the scaling; the 2-D
    operator is built from the 4x4 polyphase matrices with an independent
    mirror rule (full-rate sample positions), the oracle mirrors polyphase
    indices.
    """
    n = h * w
    E = np.eye(n).reshape(n, h, w).copy()
    L.lift2d_forward_interleaved(E, "cdf97")
    A_oracle = E.reshape(n, n).T
    op = lambda m: O.operator(m, h, w)
    A = np.eye(n)
    for p, u in L.CDF97_PAIRS:
        A = op(O.S_nonsep(O.update_filter(u))) @ op(O.T_nonsep(O.predict_filter(p))) @ A
    scale = np.empty(n)
    for r in range(h):
        for c in range(w):
            scale[r * w + c] = (L.K97 if r % 2 else 1 / L.K97) * (L.K97 if c % 2 else 1 / L.K97)
    A = scale[:, None] * A
    assert np.max(np.abs(A_oracle - A)) < 1e-13


def test_table1_counts_match_paper():
    """Table 1: steps and MACs per quadruple; the paper's reduced non-separable scheme is 18/36."""
    with open(os.path.join(GOLDEN, "table1.json")) as f:
        t1 = json.load(f)
    counts = O.table1_counts()
    for wav in ("cdf53", "cdf97"):
        pairs = t1["lifting_pairs"][wav]
        for scheme in ("separable_lifting", "nonseparable_lifting"):
            steps, macs = counts[scheme]
            assert steps * pairs == t1[wav][scheme]["steps"], (wav, scheme)
            assert macs * pairs == t1[wav][scheme]["ops_opencl"], (wav, scheme)
            assert macs * pairs == t1[wav][scheme]["ops_shaders"], (wav, scheme)
    # plain (not reduced) non-separable lifting: 12 + 12 per pair, not printed by the paper
    assert counts["nonseparable_lifting_plain"] == (2, 24)


# --- integer 5/3 readings ----------------------------------------------------

def _int53_row_then_column(x):
    a = np.array(x, dtype=np.int64)
    L.predict_int53(a, -1)
    L.update_int53(a, -1)
    L.predict_int53(a, -2)
    L.update_int53(a, -2)
    return a


def test_int53_order_matters():
    """With floors the interleaved order T^H T^V S^H S^V differs from rows-then-columns."""
    x = synth.uniform_int(64, 64, seed=7)
    a = np.array(x, dtype=np.int64)
    L.lift2d_forward_interleaved(a, "legall53")
    b = _int53_row_then_column(x)
    diff = np.count_nonzero(a != b)
    assert diff > 100
    assert np.max(np.abs(a - b)) <= 4


def test_int53_close_to_linear():
    """Reversible 5/3 == linear 5/3 up to the rounding of its floors.

    One level: per-step rounding bounds (floor(v/2) in [v/2 - 1/2, v/2],
    floor((v + 2)/4) in [v/4 - 1/4, v/4 + 1/2]) propagated through T^H, T^V,
    S^H, S^V give |LL| <= 2.125, |HL|, |LH| <= 1.75, |HH| <= 1.5.
    """
    x = synth.uniform_int(65, 66, seed=8)
    a = L.forward(x, 1, "legall53").astype(np.float64)
    b = L.forward(x.astype(np.float64), 1, "linear53")
    d = np.abs(a - b)
    v = L.band_views(d, 1)
    assert v[(1, "LL")].max() <= 2.125
    assert v[(1, "HL")].max() <= 1.75
    assert v[(1, "LH")].max() <= 1.75
    assert v[(1, "HH")].max() <= 1.5
    assert d.max() > 0.2  # the floors do act


# --- the reversible 5/3 rounding rule (floor toward -inf, update offset +2) ---
# The paper prints no rounding rule for its CDF 5/3; the reading is the usual
# reversible 5/3 (floor of half the predict sum, floor of a quarter of the
# update sum plus 2).  These pins fix both halves of that rule: a hand-worked
# example (tests/golden/legall53_worked.json) and the exact rounding residuals
# of each integer step against the linear step it rounds.

def _worked():
    with open(os.path.join(GOLDEN, "legall53_worked.json")) as f:
        return json.load(f)


def _worked_example_holds():
    g = _worked()
    x = np.array([g["one_d"]["x"]], dtype=np.int64)
    ok = L.forward(x, 1, "legall53")[0].tolist() == g["one_d"]["mallat"]
    ok = ok and L.forward(x.T.copy(), 1, "legall53")[:, 0].tolist() == g["one_d"]["mallat"]
    y = np.array(g["two_d"]["x"], dtype=np.int64)
    return ok and L.forward(y, 1, "legall53").tolist() == g["two_d"]["mallat"]


def test_int53_worked_example():
    """The oracle reproduces the hand-worked 1-D (row and column) and 2-D examples, and inverts them."""
    assert _worked_example_holds()
    g = _worked()
    back = L.inverse(np.array(g["two_d"]["mallat"], dtype=np.int64), 1, "legall53")
    assert back.tolist() == g["two_d"]["x"]


def _step_residuals(axis):
    """Sets of (integer step - linear step) over a signed random image, predict and update apart.

    The predict residual is s/2 - floor(s/2) for the even-neighbour sum s, the
    update residual floor((v + 2)/4) - v/4 for the odd-neighbour sum v; both
    are taken on the same input, so each set isolates one rounding.
    """
    rng = np.random.default_rng(5)
    x = rng.integers(-4096, 4097, size=(37, 41)).astype(np.int64)
    a = x.copy()
    L.predict_int53(a, axis)
    b = x.astype(np.float64)
    L.predict(b, -0.5, axis)
    pred = set((a - b).ravel().tolist())
    c = a.copy()
    L.update_int53(c, axis)
    d = a.astype(np.float64)
    L.update(d, 0.25, axis)
    upd = set((c - d).ravel().tolist())
    return pred, upd


@pytest.mark.parametrize("axis", [-1, -2])
def test_int53_rounding_residuals(axis):
    """floor((e_i + e_i+1)/2) differs from the linear half-sum by 0 or -1/2 (so d by 0 or +1/2),
    floor((d_i-1 + d_i + 2)/4) from the linear quarter-sum by exactly {-1/4, 0, 1/4, 1/2};
    every value occurs (signed inputs, every residue)."""
    pred, upd = _step_residuals(axis)
    assert pred == {0.0, 0.5}
    assert upd == {-0.25, 0.0, 0.25, 0.5}


# --- planted mistakes: the pins catch a perturbed oracle ----------------------

@pytest.mark.parametrize("name", ["ALPHA", "BETA", "GAMMA", "DELTA", "K97"])
def test_perturbed_constant_is_caught(monkeypatch, name):
    """Plant a mistake in one lifting constant: lifting no longer equals convolution."""
    monkeypatch.setattr(L, name, getattr(L, name) * (1 + 1e-6))
    monkeypatch.setattr(L, "CDF97_PAIRS", ((L.ALPHA, L.BETA), (L.GAMMA, L.DELTA)))
    x = synth.gradient_noise(16, 16, seed=9).astype(np.float64)
    a = L.forward(x, 1, "cdf97")
    b = FB.forward(x, 1, "cdf97")
    assert np.max(np.abs(a - b)) > 1e-9 * np.max(np.abs(x))


def test_swapped_step_order_is_caught():
    """Plant a mistake: update before predict gives a different (wrong) transform."""
    x = synth.gradient_noise(16, 16, seed=10).astype(np.float64)
    a = np.array(x)
    for p, u in L.CDF97_PAIRS:
        L.update(a, u, -1)
        L.predict(a, p, -1)
        L.update(a, u, -2)
        L.predict(a, p, -2)
    L._scale(a, L.K97, -1)
    L._scale(a, L.K97, -2)
    b = FB.forward(x, 1, "cdf97")
    assert np.max(np.abs(L.deinterleave(a) - b)) > 1e-3


# --- the sampled-coefficient helper used for full-size parity ---------------

@pytest.mark.parametrize("wavelet", ["cdf97", "legall53"])
def test_sample_coefficient_matches_full_transform(wavelet):
    h, w, levels = 203, 150, 4
    x = synth.image(wavelet, h, w, seed=12)
    full = L.forward(x, levels, wavelet)
    rng = np.random.default_rng(1)
    pos = [(0, 0), (h - 1, w - 1), (0, w - 1), (h - 1, 0), (5, 77), (100, 3)]
    pos += [(int(rng.integers(h)), int(rng.integers(w))) for _ in range(40)]
    for r, c in pos:
        assert L.sample_coefficient(x, levels, wavelet, r, c) == pytest.approx(full[r, c], abs=1e-9), (r, c)


# the two plausible misreadings of the rounding rule, planted in the oracle
def _predict_int53_trunc(a, axis, sign=1):
    if a.shape[axis] < 2:
        return
    even, odd = L._polyphase(a, axis)
    no = odd.shape[-1]
    s = even[..., :no] + L._even_next(even, no)
    odd -= sign * np.trunc(s / 2).astype(a.dtype)  # rounds toward zero, not -inf


def _update_int53_plus1(a, axis, sign=1):
    if a.shape[axis] < 2:
        return
    even, odd = L._polyphase(a, axis)
    prev, cur = L._odd_prev_cur(odd, even.shape[-1])
    even += sign * np.floor_divide(prev + cur + 1, 4)  # offset +1 instead of +2


@pytest.mark.parametrize("mutant", ["predict_truncates", "update_offset_1"])
def test_int53_rounding_mistakes_are_caught(monkeypatch, mutant):
    """Plant each misreading of the 5/3 rounding rule: the worked example and the residual sets fail."""
    if mutant == "predict_truncates":
        monkeypatch.setattr(L, "predict_int53", _predict_int53_trunc)
    else:
        monkeypatch.setattr(L, "update_int53", _update_int53_plus1)
    assert not _worked_example_holds()
    for axis in (-1, -2):
        pred, upd = _step_residuals(axis)
        assert pred != {0.0, 0.5} or upd != {-0.25, 0.0, 0.25, 0.5}
    # a consistent misreading still inverts exactly: round trips alone cannot see it
    x = synth.uniform_int(9, 7, seed=3) - 2048
    assert np.array_equal(L.inverse(L.forward(x, 2, "legall53"), 2, "legall53"), x)
