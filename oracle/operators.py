"""The paper's polyphase lifting matrices as explicit operators (test infrastructure only).

Paper: Barina et al., arXiv 1705.08266.

* Sec. 2 (z-transform notation): a 2-D filter G(z_m, z_n) = sum g_{km,kn}
  z_m^-km z_n^-kn; m is the horizontal axis, n the vertical one, and
  G*(z_m, z_n) = G(z_n, z_m) is the transposed filter.  A 1-D filter lifted
  to 2-D acts along the horizontal axis only.
* Sec. 2, separable lifting: T_P^H, T_P^V, S_U^H, S_U^V are 4x4 matrices of
  filters acting on the quadruple (c0, c1, c2, c3).
* Sec. 3, non-separable lifting: the spatial predict T_P with rows
  [1,0,0,0], [P,1,0,0], [P*,0,1,0], [PP*,P*,P,1] and the spatial update S_U
  with rows [1,U,U*,UU*], [0,1,0,U*], [0,0,1,U], [0,0,0,1].
* Sec. 3, operation reduction: P = P0 + P1 and U = U0 + U1 with P0, U0 the
  constant (same-quadruple) terms; P0, U0 go into the separable scheme and
  P1, U1 stay in the non-separable one; the two run with no barrier between
  them.
* Table 1: steps and multiply-accumulate counts per quadruple.

Filters are dicts {(km, kn): coefficient}.  Applying filter F from component j
to component i adds sum F[km, kn] * c_j[r - kn, c - km] to c_i[r, c].  With
the reading P = p (1 + z) and U = u (1 + z^-1): P reads the right (or lower)
neighbour, U the left (or upper) one.

Operators are built on an h x w image with whole-sample symmetric extension:
a source sample outside the image is replaced by its mirror, which has the
same parity and hence is the same polyphase component.
"""
from __future__ import annotations

import numpy as np

Filter = dict  # {(km, kn): coefficient}


def fmul(a: Filter, b: Filter) -> Filter:
    out: Filter = {}
    for (am, an), av in a.items():
        for (bm, bn), bv in b.items():
            k = (am + bm, an + bn)
            out[k] = out.get(k, 0.0) + av * bv
    return {k: v for k, v in out.items() if v != 0.0}


def transpose(f: Filter) -> Filter:
    """G*(z_m, z_n) = G(z_n, z_m)."""
    return {(kn, km): v for (km, kn), v in f.items()}


def predict_filter(p: float) -> Filter:
    """P = p (1 + z_m): the current and the next even sample."""
    return {(0, 0): p, (-1, 0): p}


def update_filter(u: float) -> Filter:
    """U = u (1 + z_m^-1): the previous and the current odd sample."""
    return {(0, 0): u, (1, 0): u}


def split0(f: Filter) -> Filter:
    """F0: the constant term (same quadruple)."""
    return {k: v for k, v in f.items() if k == (0, 0)}


def split1(f: Filter) -> Filter:
    """F1 = F - F0: the terms that read a neighbouring quadruple."""
    return {k: v for k, v in f.items() if k != (0, 0)}


def identity4():
    return [[{(0, 0): 1.0} if i == j else {} for j in range(4)] for i in range(4)]


# --- the paper's matrices (Sec. 2 and Sec. 3) ------------------------------

def T_H(P: Filter):
    m = identity4()
    m[1][0] = P
    m[3][2] = P
    return m


def T_V(P: Filter):
    m = identity4()
    m[2][0] = transpose(P)
    m[3][1] = transpose(P)
    return m


def S_H(U: Filter):
    m = identity4()
    m[0][1] = U
    m[2][3] = U
    return m


def S_V(U: Filter):
    m = identity4()
    m[0][2] = transpose(U)
    m[1][3] = transpose(U)
    return m


def T_nonsep(P: Filter):
    Ps = transpose(P)
    m = identity4()
    m[1][0] = P
    m[2][0] = Ps
    m[3][0] = fmul(P, Ps)
    m[3][1] = Ps
    m[3][2] = P
    return m


def S_nonsep(U: Filter):
    Us = transpose(U)
    m = identity4()
    m[0][1] = U
    m[0][2] = Us
    m[0][3] = fmul(U, Us)
    m[1][3] = Us
    m[2][3] = U
    return m


def mac_count(m) -> int:
    """Multiply-accumulates per quadruple: the number of terms off the unit diagonal."""
    n = 0
    for i in range(4):
        for j in range(4):
            if i != j:
                n += len(m[i][j])
    return n


# --- explicit operators on an image ----------------------------------------

_PAR = ((0, 0), (0, 1), (1, 0), (1, 1))  # (row parity, column parity) of c0..c3


def _mirror(i: int, n: int) -> int:
    if n == 1:
        return 0
    period = 2 * (n - 1)
    i %= period
    return period - i if i >= n else i


def operator(m, h: int, w: int) -> np.ndarray:
    """Dense (h*w x h*w) matrix of the 4x4 polyphase filter matrix m on an h x w image."""
    n = h * w
    A = np.zeros((n, n))
    for i in range(4):
        pr, pc = _PAR[i]
        for r in range((h - pr + 1) // 2):
            for c in range((w - pc + 1) // 2):
                out = (2 * r + pr) * w + (2 * c + pc)
                for j in range(4):
                    qr, qc = _PAR[j]
                    for (km, kn), g in m[i][j].items():
                        sr = _mirror(2 * (r - kn) + qr, h)
                        sc = _mirror(2 * (c - km) + qc, w)
                        A[out, sr * w + sc] += g
    return A


def table1_counts():
    """(steps, MACs) per quadruple for one (P, U) pair, by scheme (Table 1, per pair)."""
    P = predict_filter(1.0)
    U = update_filter(1.0)
    sep = [T_H(P), T_V(P), S_H(U), S_V(U)]
    nonsep = [T_nonsep(P), S_nonsep(U)]
    reduced_P = [T_nonsep(split1(P)), T_H(split0(P)), T_V(split0(P))]
    reduced_U = [S_nonsep(split1(U)), S_H(split0(U)), S_V(split0(U))]
    return {
        "separable_lifting": (len(sep), sum(mac_count(m) for m in sep)),
        "nonseparable_lifting_plain": (len(nonsep), sum(mac_count(m) for m in nonsep)),
        # each reduced step = the P1 (or U1) non-separable part plus the P0 (or U0)
        # separable part, with no barrier between them: one step
        "nonseparable_lifting": (2, sum(mac_count(m) for m in reduced_P + reduced_U)),
    }
