"""CPU oracle: the slot-domain DFT of CKKS factored into sparse diagonal
stages -- the matrices of the CoeffToSlot / SlotToCoeff transforms of
bootstrapping, the multi-stage linear transformations the LT algorithms are
built for (Sec. I; their strided diagonals are the offsets o_t = offset0 +
stride t of a window).

TEST INFRASTRUCTURE ONLY (see oracle/ckks.py).  Only the matrices are
defined here (FP64 values); evaluating them on ciphertexts is the LT
algorithms' job (oracle/lt.py).

Slots.  With n = N/2 slots, slot j is the value at the point
xi_j = zeta^(5^j mod 4n), zeta = exp(2 pi i / 4n): the slot vector of the
plaintext m is U w with w_k = m_k + i m_{k+n} and U[j][k] = xi_j^k (the
point's n-th power is i, since 5^j = 1 mod 4).  U is the SlotToCoeff map
(coefficients held in slots -> slots); CoeffToSlot is U^-1 = U^H / n (the
points are the n distinct roots of X^n = i, so U^H U = n I).

Factorisation, from the radix-2 split of the evaluation.  For size L (a
power of two) let xi^(L)_j = exp(2 pi i (5^j mod 4L) / 4L), j < L, and
P(X) = E(X^2) + X O(X^2) with E, O of degree < L/2.  Then
(xi^(L)_j)^2 = xi^(L/2)_j, which depends on j mod L/2 only, and
xi^(L)_{j+L/2} = -xi^(L)_j because 5^(L/2) = 1 + 2L mod 4L.  Hence
    P(xi_j) = E_j + xi_j O_j,     P(xi_{j+L/2}) = E_j - xi_j O_j,   j < L/2,
a butterfly on the evaluations E, O of the even and odd halves.  Applied for
L = 2, 4, .., n to the bit-reversed coefficient vector this gives
    U R = S_m ... S_2 S_1       (m = log2 n, R the bit reversal),
where S_t (L = 2^t, h = L/2) maps x to
    y[b + j]     = x[b + j] + xi^(L)_j x[b + j + h]
    y[b + j + h] = x[b + j] - xi^(L)_j x[b + j + h]        (b a multiple of L)
and has three nonzero diagonals, at offsets 0, +h and -h.  Its inverse
    x[b + j] = (y[b + j] + y[b + j + h]) / 2,
    x[b + j + h] = (y[b + j] - y[b + j + h]) / (2 xi_j)
has the same three diagonals.  So SlotToCoeff on bit-reversed slots is
S_m ... S_1 and CoeffToSlot to bit-reversed slots is S_1^-1 ... S_m^-1; a
product of r consecutive stages S_{t+r-1} .. S_t has its diagonals at the
multiples of 2^(t-1) in the window -(2^r - 1) 2^(t-1) .. (2^r - 1) 2^(t-1)
(mod n), which is one LT per group of stages and one level per LT.

Diagonal convention (the LT's): y[j] = sum_o d_o[j] x[(j + o) mod n].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def points(L: int) -> np.ndarray:
    """xi^(L)_j = exp(2 pi i (5^j mod 4L) / 4L), j < L."""
    e = np.array([pow(5, j, 4 * L) for j in range(L)], dtype=np.float64)
    return np.exp(2j * np.pi * e / (4 * L))


def u_matrix(n: int) -> np.ndarray:
    """U[j][k] = xi_j^k (dense; small n only)."""
    xi = points(n)
    return xi[:, None] ** np.arange(n)[None, :]


def bitrev(n: int) -> np.ndarray:
    """Index permutation of the bit reversal on log2(n) bits."""
    b = int(math.log2(n))
    return np.array([int(format(i, f"0{b}b")[::-1], 2) if b else 0 for i in range(n)], dtype=np.int64)


def stage(n: int, t: int, inverse: bool = False) -> dict:
    """Diagonals {offset mod n: values[n]} of S_t (or S_t^-1), L = 2^t."""
    L, h = 1 << t, 1 << (t - 1)
    xi = points(L)[:h]
    r = np.arange(n)
    pos = r % L
    upper = pos < h
    w = np.where(upper, xi[np.minimum(pos, h - 1)], xi[np.maximum(pos - h, 0)])
    d0 = np.where(upper, 1.0 + 0j, -w)
    dp = np.where(upper, w, 0j)
    dm = np.where(upper, 0j, 1.0 + 0j)
    if inverse:
        d0 = np.where(upper, 0.5 + 0j, -0.5 / w)
        dp = np.where(upper, 0.5 + 0j, 0j)
        dm = np.where(upper, 0j, 0.5 / w)
    out = {}
    for o, v in ((0, d0), (h, dp), (-h, dm)):
        k = o % n
        out[k] = out.get(k, np.zeros(n, dtype=np.complex128)) + v
    return out


def compose(a: dict, b: dict, n: int) -> dict:
    """Diagonals of the product A B (B applied first):
    (A B)[j][j + o + p] += a_o[j] b_p[(j + o) mod n]."""
    out = {}
    idx = np.arange(n)
    for o, ao in a.items():
        for p, bp in b.items():
            k = (o + p) % n
            out[k] = out.get(k, np.zeros(n, dtype=np.complex128)) + ao * bp[(idx + o) % n]
    return out


def to_dense(d: dict, n: int) -> np.ndarray:
    M = np.zeros((n, n), dtype=np.complex128)
    j = np.arange(n)
    for o, v in d.items():
        M[j, (j + o) % n] += v
    return M


@dataclass
class Window:
    """One LT stage: diagonals f_t at offsets offset0 + stride t, t < D."""
    offset0: int
    stride: int
    fvals: np.ndarray      # [D][n] complex

    @property
    def D(self) -> int:
        return self.fvals.shape[0]


def as_window(d: dict, n: int, pad: bool = False) -> Window:
    """The smallest window offset0 + stride t (stride = gcd of the offsets and
    n) that covers every diagonal of d; diagonals inside the window that d
    does not have are zero.  offset0 is taken in [-n/2, n/2).  With `pad`,
    D is rounded up to a power of two (zero diagonals appended), which gives
    the BSGS splits more factors, as long as the offsets stay distinct."""
    offs = sorted(d)
    s = n
    for o in offs:
        s = math.gcd(s, o)
    m = n // s
    pos = sorted({o // s for o in offs})
    if len(pos) == 1:
        start, D = pos[0], 1
    else:
        gaps = [((pos[(i + 1) % len(pos)] - pos[i]) % m, i) for i in range(len(pos))]
        g, i = max(gaps)
        start = pos[(i + 1) % len(pos)]
        D = m - g + 1
    off0 = start * s
    if off0 >= n // 2:
        off0 -= n
    if pad:
        D = min(1 << (D - 1).bit_length(), m)
    f = np.zeros((D, n), dtype=np.complex128)
    for t in range(D):
        k = (off0 + s * t) % n
        if k in d:
            f[t] = d[k]
    return Window(off0, s, f)


def _groups(m: int, radices) -> list:
    radices = list(radices)
    if sum(radices) != m or min(radices) < 1:
        raise ValueError(f"radices {radices} must be positive and sum to log2 n = {m}")
    return radices


def slot_to_coeff(n: int, radices, pad: bool = False) -> list:
    """The stages of S_m ... S_1 grouped by `radices` (first group applied
    first: S_{r1} .. S_1), as windows."""
    m = int(math.log2(n))
    out, t = [], 1
    for r in _groups(m, radices):
        d = stage(n, t)
        for u in range(t + 1, t + r):
            d = compose(stage(n, u), d, n)
        out.append(as_window(d, n, pad))
        t += r
    return out


def coeff_to_slot(n: int, radices, pad: bool = False) -> list:
    """The stages of S_1^-1 ... S_m^-1 grouped by `radices` (first group
    applied first: S_{m-r1+1}^-1 .. S_m^-1), as windows."""
    m = int(math.log2(n))
    out, t = [], m
    for r in _groups(m, radices):
        d = stage(n, t, inverse=True)
        for u in range(t - 1, t - r, -1):
            d = compose(stage(n, u, inverse=True), d, n)
        out.append(as_window(d, n, pad))
        t -= r
    return out


def apply_windows(z: np.ndarray, windows) -> np.ndarray:
    """FP64 chain: each window's y[j] = sum_t f_t[j] z[(j + offset0 + stride t) mod n]."""
    n = z.shape[0]
    idx = np.arange(n)
    for w in windows:
        y = np.zeros(n, dtype=np.complex128)
        for t in range(w.D):
            y += w.fvals[t] * z[(idx + w.offset0 + w.stride * t) % n]
        z = y
    return z
