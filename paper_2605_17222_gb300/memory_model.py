"""Off-chip memory model of the paper's memory-optimized TH-BSGS data path
(Sec. IV): the per-phase off-chip access and peak on-chip requirement of
its memory-requirement table, as functions of the HE shape, the split
(n'1, n'2, n'3) and the parallelism knobs m1..m6, l1..l5 of its parallelism
table.  Host-side arithmetic for comparing the FPGA design's traffic with
this library's measured HBM traffic on the same shapes; the LT itself never
calls it.

Units.  Every term counts limbs of N words; the paper's words are w = 54
bits and its totals are in units of 2^30 bytes, which is how the printed
off-chip totals of its resource table (2.84, 107.91 and 903.47 for Set-A,
B and C at the knobs of its parameter table) are reproduced here, within
0.2 %, with the quotients n'/m taken as exact fractions.

Phases (Sec. IV): 1 = Alg. 2 lines 1-5, 2 = lines 6-7, 3 = lines 8-11,
4 = lines 12-14, 5 = lines 15-18, 6 = line 19.  Off-chip access has five
categories per phase: (I)NTT twiddles, the LT matrix, switching keys,
polynomial reads and polynomial writes.
"""
from __future__ import annotations

from dataclasses import dataclass

CATEGORIES = ("twiddle", "matrix", "swk", "read", "write")


@dataclass(frozen=True)
class Shape:
    """N, L + 1 (Q limbs), alpha (digit size, also the P limb count in the
    paper), beta (digits), n (nonzero diagonals), split (n'1, n'2, n'3)."""
    N: int
    Lp1: int
    alpha: int
    beta: int
    n: int
    split: tuple

    @property
    def ext(self) -> int:
        return self.Lp1 + self.alpha


@dataclass(frozen=True)
class Knobs:
    """m1..m6 (polynomials / keys processed together per phase) and l1..l5
    (limbs processed together per phase)."""
    m1: int
    l1: int
    m2: int
    l2: int
    m3: int
    m4: int
    l3: int
    m5: int
    l4: int
    m6: int
    l5: int


# The paper's evaluation shapes (table of HE parameters) with the split and the
# knobs of its parameter table, and the off-chip totals of its resource table.
PAPER_SETS = {
    "Set-A": (Shape(2 ** 13, 5, 5, 1, 2 ** 12, (16, 16, 16)), Knobs(5, 5, 15, 10, 15, 8, 1, 86, 1, 8, 4), 2.84),
    "Set-B": (Shape(2 ** 15, 16, 8, 2, 2 ** 14, (32, 16, 32)), Knobs(8, 1, 1, 12, 8, 1, 1, 25, 1, 4, 1), 107.91),
    "Set-C": (Shape(2 ** 16, 32, 12, 3, 2 ** 15, (32, 32, 32)), Knobs(1, 1, 1, 1, 4, 1, 1, 12, 1, 1, 1), 903.47),
}


def offchip_limbs(s: Shape, m: Knobs) -> list:
    """Per phase, {category: limbs read or written off chip}."""
    n1, n2, n3 = s.split
    E, L1, b = s.ext, s.Lp1, s.beta
    return [
        {"twiddle": 3 * L1 + 2 * s.alpha, "matrix": 0, "swk": 2 * (n1 - 1) * b * E,
         "read": 2 * L1, "write": 3 * (n1 - 1) * E + 2 * L1},
        {"twiddle": (n1 - 1) / m.m2 * E, "matrix": 0, "swk": 0,
         "read": (n1 - 1) * E, "write": (n1 - 1) * b * E},
        {"twiddle": 0, "matrix": 0, "swk": 2 * (n2 - 1) * b * E,
         "read": (n2 - 1) / m.m3 * n1 * (b + 1) * E, "write": 2 * n1 * n2 * E},
        {"twiddle": E, "matrix": s.n * E, "swk": 0,
         "read": 2 * (n1 * n2 + (n1 * n2 / m.m5 - 1) * n3) * E, "write": 2 * (n1 * n2 / m.m5) * n3 * E},
        {"twiddle": n3 / m.m6 * E, "matrix": 0, "swk": 2 * (n3 - 1) * b * E,
         "read": 2 * (n3 + n3 / m.m6 - 1) * E, "write": 2 * (n3 / m.m6) * E},
        {"twiddle": E, "matrix": 0, "swk": 0, "read": 2 * E, "write": 2 * L1},
    ]


def onchip_limbs(s: Shape, m: Knobs) -> list:
    """Peak on-chip requirement per phase, in limbs, as the table prints it.
    (Not reproduced against the paper's 43 MB device: at Set-C's knobs phase 2
    alone already exceeds it, so the paper's compiler must count differently.)"""
    E, L1, b = s.ext, s.Lp1, s.beta
    return [
        2 * L1 + (b + 4) * m.l1 + (4 * b + 6) * m.m1 * m.l1,
        2 * E + m.m2 * (L1 + 2 * b * m.l2) + 2 * m.l2,
        2 * m.l3 * ((b + 1) * m.m4 + 2 * b * m.m3 + 2 * m.m3 * m.m4),
        6 * m.m5 * m.l4 + 5 * m.l4,
        m.m6 * E + (5 * b * m.m6 + 2 * m.m6 + 6) * m.l5 + 2 * m.l5,
        2 * E,
    ]


def limb_bytes(N: int, word_bits: int = 54) -> float:
    return N * word_bits / 8


def offchip_bytes(s: Shape, m: Knobs, word_bits: int = 54) -> float:
    """Total off-chip bytes of one LT on the paper's data path."""
    return sum(sum(p.values()) for p in offchip_limbs(s, m)) * limb_bytes(s.N, word_bits)


def offchip_by_category(s: Shape, m: Knobs, word_bits: int = 54) -> dict:
    tot = {c: 0.0 for c in CATEGORIES}
    for p in offchip_limbs(s, m):
        for c, v in p.items():
            tot[c] += v
    return {c: v * limb_bytes(s.N, word_bits) for c, v in tot.items()}


def paper_units(nbytes: float) -> float:
    """Bytes in the unit of the paper's totals (2^30 bytes)."""
    return nbytes / 2 ** 30
