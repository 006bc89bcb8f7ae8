"""CPU oracle: the paper's complexity formulas, used as pins.

TEST INFRASTRUCTURE ONLY (see oracle/ckks.py).

* Table "complexity comparisons": Decompose / ModDown / coefficient-wise
  multiplication / switching-key counts per algorithm.  Algorithm 2 itself
  (and the text after the table) gives TH-BSGS n'1 + n'3 - 1 Decompose and
  n'1 + n'3 ModDown; the table prints n'1 + n'3 and n'1 + n'3 + 1.  The
  algorithm is followed.
* Table "number of modular multiplications and switching key size": modular
  multiplications counted with (I)NTT = (N/2) log2 N per limb, and
  SWK memory = keys x 2 beta (L+1+alpha) N w / 8 bytes, reported in GiB.
"""
from __future__ import annotations

import math


def counts(algo: str, split, beta: int, limbs_q: int, alpha: int, n: int) -> dict:
    """Operation counts of one LT (limbs_q = L + 1, the Q limbs in use)."""
    ext = limbs_q + alpha
    if algo == "diag":
        return dict(decompose=1, moddown=2, ks_products=n - 1,
                    cw_mult=2 * beta * (n - 1) * ext + 2 * n * ext, keys=n - 1)
    if algo == "bsgs":
        n1, n2 = split
        r = n1 + n2 - 2
        return dict(decompose=r, moddown=2 * r, ks_products=r,
                    cw_mult=2 * beta * r * ext + 2 * n * limbs_q, keys=r)
    if algo == "dh":
        n1, n2 = split
        r = n1 + n2 - 2
        return dict(decompose=n2, moddown=n2 + 1, ks_products=r,
                    cw_mult=2 * beta * r * ext + 2 * n * ext, keys=r)
    if algo == "th":
        n1, n2, n3 = split
        r = n1 * n2 + n3 - 2
        return dict(decompose=n1 + n3 - 1, moddown=n1 + n3, ks_products=r,
                    cw_mult=2 * beta * r * ext + 2 * n * ext, keys=n1 + n2 + n3 - 3)
    raise ValueError(algo)


def modmul_count(algo: str, split, N: int, limbs_q: int, alpha: int) -> int:
    """Modular multiplications of one LT at n = N/2 (dense matrix)."""
    beta = -(-limbs_q // alpha)
    n = N // 2
    ntt = (N // 2) * int(math.log2(N))          # per limb, NTT or INTT
    decompose = limbs_q * ntt + N * beta * (alpha + alpha * limbs_q) + beta * limbs_q * ntt
    moddown = alpha * ntt + N * (alpha + alpha * limbs_q) + limbs_q * ntt + N * limbs_q
    c = counts(algo, split, beta, limbs_q, alpha, n)
    return c["cw_mult"] * N + c["decompose"] * decompose + c["moddown"] * moddown


def swk_gib(algo: str, split, N: int, limbs_q: int, alpha: int, w: int) -> float:
    beta = -(-limbs_q // alpha)
    keys = counts(algo, split, beta, limbs_q, alpha, N // 2)["keys"]
    return keys * 2 * beta * (limbs_q + alpha) * N * w / 8 / 2 ** 30
