"""The integer bounds the kernels' lazy arithmetic rests on, checked with exact
Python integers on random and extreme inputs (CPU only).  Each test restates
one formula the CUDA code evaluates in 64-bit registers and checks the bound
its comment claims, so that a change to either side has something to fail.

  * the three-product Shoup quotient of the growing forward butterflies is at
    most 2 below floor(b ws / 2^64), so the remainder lies in [0, 4q);
  * the growing forward butterflies' word bound (68q from [0, 4q)) stays
    below 2^64 for the moduli that take them;
  * K6's fold of a middle-layer sum x = sum_b d_b k_b + A (beta <= 8, q < 2^41)
    is below 2^64, congruent to x mod q, and 64 of its products with a word
    below q fit the 128-bit accumulators;
  * the lazy 128-bit Barrett reduction's estimate leaves a remainder in [0, 4q);
  * for 2^32 < q < 2^41: the NTT epilogues' 32-bit quotient estimate leaves
    [0, 3q) for words below 2^50;
  * the inverse passes' one lazy butterfly keeps every modulus's words in
    [0, 2q).
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
    """Forward: 16 stages from [0, 4q) add at most 4q each (moduli below 2^57);
    the reducing butterflies' 4q stays below 2^64 for every modulus."""
    for q in MODULI:
        if q < (1 << 57):
            assert 4 * q + 16 * 4 * q <= M64
        assert 4 * q <= M64
    assert 68 * ((1 << 57) - 1) <= M64


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


# ------------------------------------------------------------------ 96-bit multiply-accumulate (K6, q < 2^41)
M32 = (1 << 32) - 1


def mac96(lo, hi, a, b):
    """The seven 32-bit multiply-adds of modarith.cuh's mac96 with their carry
    flag, word for word: (lo, hi) += a b."""
    w0, w1 = lo & M32, lo >> 32
    x0, x1, y0, y1 = a & M32, a >> 32, b & M32, b >> 32

    def add(dst, v, cin):  # 32-bit add with carry in; (result, carry out)
        s = dst + v + cin
        return s & M32, s >> 32

    w0, c = add(w0, (x0 * y0) & M32, 0)               # mad.lo.cc
    w1, c = add(w1, (x0 * y0) >> 32, c)               # madc.hi.cc
    hi = (hi + ((x1 * y1) & M32) + c) & M32           # madc.lo (no carry out)
    w1, c = add(w1, (x0 * y1) & M32, 0)               # mad.lo.cc
    hi = (hi + ((x0 * y1) >> 32) + c) & M32           # madc.hi
    w1, c = add(w1, (x1 * y0) & M32, 0)               # mad.lo.cc
    hi = (hi + ((x1 * y0) >> 32) + c) & M32           # madc.hi
    return w0 | (w1 << 32), hi


def small_moduli():
    """The moduli that take K6's 96-bit path: 2^32 < q < 2^41 (mu = floor(2^64 / q) fits 32 bits)."""
    out = [q for q in MODULI if (1 << 32) < q < (1 << 41)]
    assert out
    return out


def test_mac96_is_exact_below_2_96():
    """For operands below 2^41 the three-word sum is the exact integer sum as
    long as it stays below 2^96 -- the middle layer's 6 products plus A, and
    64 outer products of a word below 3q with one below q."""
    for q in small_moduli():
        ops = [0, 1, q - 1, (1 << 41) - 1] + [RNG.randrange(q) for _ in range(60)]
        for terms in (7, 64):
            lo = hi = 0
            exact = 0
            for t in range(terms):
                a = ops[(t * 7) % len(ops)] if t % 5 else (1 << 41) - 1
                b = ops[(t * 13 + 3) % len(ops)]
                lo, hi = mac96(lo, hi, a, b)
                exact += a * b
            assert exact < 1 << 96
            assert lo | (hi << 64) == exact


def test_middle_sum_reduction_for_the_96_bit_products():
    """K6's reduction of a middle-layer sum x < 2^85 for the 96-bit outer
    products: the fold to below 2^64, then the quotient estimate
    ((a1 mu + hi(a0 mu)) >> 32), mu = floor(2^64 / q), leaves a word in
    [0, 3q) congruent to x, and 64 of its products with a word below q stay
    below 2^96."""
    for q in small_moduli():
        mu = (1 << 64) // q
        assert mu < 1 << 32
        c63, c64 = (1 << 63) % q, (1 << 64) % q
        xs = [(1 << 85) - 1, 0, q, 6 * (q - 1) ** 2 + q - 1] + [RNG.getrandbits(85) for _ in range(300)]
        for x in xs:
            lo, hi = x & M64, x >> 64
            f = (lo & ~(1 << 63)) + (c63 if lo >> 63 else 0) + hi * c64
            assert f < 1 << 64 and f % q == x % q
            a0, a1 = f & M32, f >> 32
            qe = (a1 * mu + ((a0 * mu) >> 32)) >> 32
            r = (f - qe * q) & M64
            assert r < 3 * q and r % q == x % q
            assert 64 * r * (q - 1) < 1 << 96


def test_column_pass_basis_conversion_96_bit_path():
    """The NTT column pass's 96-bit basis conversion: 2^64 mod q and 2^63 mod q
    derived from mu_hi = floor(2^128 / q) >> 64 as the kernel derives them,
    four products of words below 2^41 summed by mac96, then the fold and the
    32-bit quotient estimate: a word in [0, 3q) congruent to the sum (below
    4q, the butterflies' input range)."""
    for q in small_moduli():
        mu_hi = ((1 << 128) // q) >> 64
        c64 = (0 - q * mu_hi) & M64
        c63 = (c64 + (q if c64 & 1 else 0)) >> 1
        assert c64 == (1 << 64) % q and c63 == (1 << 63) % q
        mu32 = mu_hi & M32
        assert mu32 == mu_hi
        for trial in range(200):
            ys = [RNG.randrange(1 << 41) if trial % 3 else (1 << 41) - 1 for _ in range(4)]
            cs = [RNG.randrange(q) if trial % 5 else q - 1 for _ in range(4)]
            lo = hi = 0
            for y, cst in zip(ys, cs):
                lo, hi = mac96(lo, hi, y, cst)
            x = sum(y * cst for y, cst in zip(ys, cs))
            assert lo | (hi << 64) == x
            f = (lo & ~(1 << 63)) + (c63 if lo >> 63 else 0) + hi * c64
            assert f < 1 << 64
            qe = ((f >> 32) * mu32 + (((f & M32) * mu32) >> 32)) >> 32
            r = (f - qe * q) & M64
            assert r < 3 * q and r % q == x % q


def red3_small(x, q):
    """The NTT epilogues' reduction for 2^32 < q < 2^41: quotient estimate
    floor(floor(x / 2^32) mu32 / 2^32), mu32 = floor(2^64 / q)."""
    mu32 = (((1 << 128) // q) >> 64) & M32
    assert mu32 == (1 << 64) // q
    qe = ((x >> 32) * mu32) >> 32
    return qe, (x - qe * q) & M64


def test_small_modulus_epilogue_reduction():
    """Words below 2^50 (the forward row pass ends below 68q < 2^48) reduce to
    [0, 3q): the estimate never exceeds floor(x / q) and falls short by at
    most 2."""
    for q in small_moduli():
        assert 68 * q < 1 << 48 and (q << 9) < 1 << 50
        xs = [0, 1, q - 1, q, 3 * q - 1, 68 * q - 1, (q << 9) - 1, (1 << 50) - 1]
        xs += [k * q + d for k in (1, 2, 67, 255, 511) for d in (-1, 0, 1)]
        xs += [RNG.getrandbits(50) for _ in range(2000)] + [RNG.randrange(68 * q) for _ in range(2000)]
        for x in xs:
            qe, r = red3_small(x, q)
            assert 0 <= x // q - qe <= 2, (q, x)
            assert r == x - qe * q and r < 3 * q and r % q == x % q


@pytest.mark.parametrize("q", MODULI)
def test_inverse_butterfly_keeps_words_below_2q(q):
    """The inverse passes' one butterfly for every modulus: words in [0, 2q);
    (a + b, (a - b + 2q) w) with the lazy Shoup product (exact quotient
    floor(x ws / 2^64)) and one conditional subtraction stay in [0, 2q),
    congruent to (a + b, (a - b) w)."""
    edge = [0, 1, q - 1, q, 2 * q - 1]
    for w in [1, q - 1, q // 2] + [RNG.randrange(q) for _ in range(6)]:
        ws = shoup_const(w, q)
        pairs = [(a, b) for a in edge for b in edge] + [(RNG.randrange(2 * q), RNG.randrange(2 * q)) for _ in range(300)]
        for a, b in pairs:
            s_ = a + b
            a2 = s_ - 2 * q if s_ >= 2 * q else s_
            x = a - b + 2 * q
            assert 0 < x < 4 * q <= M64
            b2 = (x * w - ((x * ws) >> 64) * q) & M64
            assert a2 < 2 * q and b2 < 2 * q
            assert a2 % q == (a + b) % q and b2 % q == ((a - b) * w) % q
