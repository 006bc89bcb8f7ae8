"""The integer bounds the kernels' lazy arithmetic rests on, checked with exact
Python integers on random and extreme inputs (CPU only).  Each test restates
one formula the CUDA code evaluates in 64-bit registers and checks the bound
its comment claims, so that a change to either side has something to fail.

  * the three-product Shoup quotient of the growing forward butterflies is at
    most 2 below floor(b ws / 2^64), so the remainder lies in [0, 4q);
  * the growing butterflies' word bounds (68q forward from [0, 4q), 2^9 q per
    inverse pass from [0, 2q)) stay below 2^64 for the moduli that take them;
  * K6's fold of a middle-layer sum x = sum_b d_b k_b + A (beta <= 8, q < 2^41)
    is below 2^64, congruent to x mod q, and 64 of its products with a word
    below q fit the 128-bit accumulators;
  * the lazy 128-bit Barrett reduction's estimate leaves a remainder in [0, 4q).
"""
import random

import pytest

from paper_2605_17222_gb300 import synth

M64 = (1 << 64) - 1
RNG = random.Random(2605)


def primes(bits_list, log_n=16):
    out = []
    for bits in bits_list:
        out.extend(synth.ntt_primes(bits, 2, 2 << log_n))
    return out


MODULI = primes([30, 40, 50, 54, 55]) + primes([60])


def shoup_const(w, q):
    return (w << 64) // q


def approx_quotient(b, ws):
    """The kernel's estimate: high product plus the high halves of the two middle ones."""
    b0, b1 = b & 0xFFFFFFFF, b >> 32
    s0, s1 = ws & 0xFFFFFFFF, ws >> 32
    return b1 * s1 + ((b0 * s1) >> 32) + ((b1 * s0) >> 32)


def samples(q, n=400):
    extremes = [0, 1, q - 1, q, 2 * q - 1, 4 * q - 1, M64, M64 - q, 1 << 63, (1 << 63) - 1]
    return extremes + [RNG.getrandbits(64) for _ in range(n)]


@pytest.mark.parametrize("q", MODULI)
def test_three_product_shoup_quotient(q):
    for w in [0, 1, q - 1, q // 2] + [RNG.randrange(q) for _ in range(8)]:
        ws = shoup_const(w, q)
        for b in samples(q):
            exact = (b * ws) >> 64
            qe = approx_quotient(b, ws)
            assert 0 <= exact - qe <= 2, (q, w, b)
            r = (b * w - qe * q) & M64
            assert r == (b * w - qe * q) and 0 <= r < 4 * q
            assert r % q == (b * w) % q


def test_growing_butterfly_word_bounds():
    """Forward: 16 stages from [0, 4q) add at most 4q each; inverse: a pass of
    8 stages from [0, 2q) at most doubles a word per stage."""
    for q in MODULI:
        if q < (1 << 57):
            assert 4 * q + 16 * 4 * q <= M64
        if q < (1 << 55):
            assert (2 * q) << 8 <= M64 and (q << 8) <= M64
    assert 68 * ((1 << 57) - 1) <= M64
    assert ((1 << 55) - 1) << 9 <= M64


def fold(x, q):
    lo, hi = x & M64, x >> 64
    c63, c64 = (1 << 63) % q, (1 << 64) % q
    return (lo & ~(1 << 63) & M64) + (c63 if lo >> 63 else 0) + hi * c64


@pytest.mark.parametrize("q", [m for m in MODULI if m < (1 << 41)])
def test_middle_layer_fold(q):
    for beta in (1, 2, 6, 8):
        worst = beta * (q - 1) ** 2 + (q - 1)
        assert worst < (1 << 85)
        for x in [0, worst, worst - 1, (1 << 64) - 1, 1 << 64, (1 << 63)] + \
                 [sum(RNG.randrange(q) * RNG.randrange(q) for _ in range(beta)) + RNG.randrange(q)
                  for _ in range(300)]:
            if x > worst:
                continue
            v = fold(x, q)
            assert v <= M64 and v % q == x % q
            assert 64 * v * (q - 1) < (1 << 128)


@pytest.mark.parametrize("q", MODULI)
def test_lazy_barrett_128(q):
    mu = (1 << 128) // q
    mu_hi, mu_lo = mu >> 64, mu & M64
    for _ in range(300):
        x = RNG.getrandbits(127)
        x_lo, x_hi = x & M64, x >> 64
        qe = (x_hi * mu_hi + ((x_hi * mu_lo) >> 64) + ((x_lo * mu_hi) >> 64)) & M64
        r = (x_lo - qe * q) & M64
        assert r % q == x % q and 0 <= r < 4 * q
