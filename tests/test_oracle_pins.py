"""Pins of the CPU oracle against facts it does not compute itself: big-integer
arithmetic, O(N^2) definitions, schoolbook products, exact CRT, the paper's
printed example and tables.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import _native as nat
from oracle import cost_model
from oracle.ckks import Ctx, find_psi
from paper_2605_17222_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    return Ctx(synth.param_set("tiny"))


def _rand_poly(ctx, basis, seed):
    return synth.uniform_mod(seed, "pin", basis, ctx.N)


# ----------------------------------------------------------------- modular arithmetic
def test_mulmod_matches_bigint():
    L = nat.lib()
    rng = np.random.default_rng(1)
    for q in [synth.param_set("n16").q[0], synth.param_set("n16").p[0], synth.param_set("n16").q[5]]:
        vals = [0, 1, q - 1, q - 2, q // 2] + [int(v) % q for v in rng.integers(0, 2**63, 50, dtype=np.uint64)]
        for a in vals:
            for b in vals[:8]:
                assert L.orc_mulmod(a, b, q) == (a * b) % q


def test_bitrev_paper_example():
    """Sec. V: bitrev(1, 3) = bitrev('001', 3) = '100' = 4."""
    with open(os.path.join(GOLDEN, "bitrev_example.json")) as f:
        g = json.load(f)
    assert nat.lib().orc_bitrev(g["x"], g["bits"]) == g["value"]


def test_psi_is_primitive_2n_root(tiny):
    for m, psi in tiny.psi.items():
        assert pow(psi, 2 * tiny.N, m) == 1
        assert pow(psi, tiny.N, m) == m - 1


# ----------------------------------------------------------------- NTT
def _brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


@pytest.mark.parametrize("log_n", [3, 5, 7])
def test_ntt_matches_definition(log_n):
    """A[s] = sum_t a_t psi^((2 brv(s) + 1) t) mod q, by O(N^2) big-int sums."""
    N = 1 << log_n
    q = synth.ntt_primes(50, 1, 2 * N)[0]
    p = synth.ntt_primes(60, 1, 2 * N)[0]
    ctx = Ctx(synth.ParamSet("x", log_n, (q,), (p,), 1))
    a = _rand_poly(ctx, [q, p], 3)
    A = ctx.ntt(a, [q, p])
    for row, m in enumerate([q, p]):
        psi = ctx.psi[m]
        for s in range(N):
            e = 2 * _brv(s, log_n) + 1
            want = sum(int(a[row, t]) * pow(psi, e * t, m) for t in range(N)) % m
            assert int(A[row, s]) == want
    assert np.array_equal(ctx.intt(A, [q, p]), a)


def test_ntt_product_is_negacyclic(tiny):
    B = tiny.basis(4, True)
    a = _rand_poly(tiny, B, 5)
    b = _rand_poly(tiny, B, 6)
    prod = tiny.intt(tiny.mul(tiny.ntt(a, B), tiny.ntt(b, B), B), B)
    N = tiny.N
    for row, m in enumerate(B):
        want = [0] * N
        for i in range(N):
            for j in range(N):
                v = int(a[row, i]) * int(b[row, j])
                if i + j < N:
                    want[i + j] += v
                else:
                    want[i + j - N] -= v
        assert [int(x) for x in prod[row]] == [w % m for w in want]


# ----------------------------------------------------------------- automorphism
def test_automorphism_ntt_matches_coefficient_form(tiny):
    """NTT(phi_r(a)) = gather(NTT(a)) (Eq. 7 derived from Eq. 2)."""
    B = tiny.basis(4, True)
    a = _rand_poly(tiny, B, 7)
    for r in [1, 3, -1, 5, tiny.N // 2 - 1]:
        lhs = tiny.ntt(tiny.auto_coeff(a, r, B), B)
        rhs = tiny.auto_ntt(tiny.ntt(a, B), r)
        assert np.array_equal(lhs, rhs), r


def test_automorphism_composes(tiny):
    B = tiny.basis(2, False)
    A = tiny.ntt(_rand_poly(tiny, B, 8), B)
    for r, s in [(1, 2), (3, -3), (5, 7)]:
        assert np.array_equal(tiny.auto_ntt(tiny.auto_ntt(A, r), s), tiny.auto_ntt(A, r + s))
    assert np.array_equal(tiny.auto_ntt(A, 0), A)


def test_automorphism_coeff_definition(tiny):
    """Eq. (2) by brute force: a(x^g) mod x^N + 1 with g = 5^r mod 2N."""
    B = tiny.basis(1, False)
    q = B[0]
    a = _rand_poly(tiny, B, 9)
    N = tiny.N
    for r in [1, 2, 7]:
        g = pow(5, r, 2 * N)
        want = [0] * N
        for t in range(N):
            e = (t * g) % (2 * N)
            if e < N:
                want[e] += int(a[0, t])
            else:
                want[e - N] -= int(a[0, t])
        got = tiny.auto_coeff(a, r, B)
        assert [int(x) for x in got[0]] == [w % q for w in want]


@pytest.mark.parametrize("dp", [8, 32, 128, 256, 512])
def test_automorphism_row_to_row_property(dp):
    """Eq. (8) and its proof: in bit-reversed storage with rows of d_p words,
    the gather of each row reads exactly one whole source row (a permutation
    within it).  Brute force over every g_r at N = 2^12."""
    log_n = 12
    N = 1 << log_n
    ctx_like = Ctx(synth.ParamSet("x", log_n, (synth.ntt_primes(40, 1, 2 * N)[0],), (), 1))
    src_of = np.empty(N, dtype=np.int64)
    for r in range(0, N // 2, 37):
        g = ctx_like.galois(r)
        for s in range(N):
            l = _brv(s, log_n)
            lp = ((g * (2 * l + 1)) % (2 * N) - 1) // 2
            src_of[s] = _brv(lp, log_n)
        rows = src_of.reshape(N // dp, dp) // dp
        assert np.all(rows == rows[:, :1]), (r, dp)
        # and the permutation within the row is a bijection
        pos = np.sort(src_of.reshape(N // dp, dp) % dp, axis=1)
        assert np.all(pos == np.arange(dp))


# ----------------------------------------------------------------- encoding
def test_encode_matches_direct_evaluation():
    ctx = Ctx(synth.ParamSet("x", 4, (synth.ntt_primes(50, 1, 32)[0],), (), 1))
    N = ctx.N
    z = synth.slots(11, "enc", N // 2)
    scale = 2.0 ** 30
    m = ctx.encode_coeffs(z, scale).astype(np.float64)
    zeta = np.exp(1j * np.pi / N)
    for j in range(N // 2):
        pt = zeta ** pow(5, j, 2 * N)
        val = sum(m[t] * pt ** t for t in range(N)) / scale
        assert abs(val - z[j]) < 1e-7
    zz = ctx.decode_coeffs(m, scale)
    assert np.max(np.abs(zz - z)) < 1e-7


def test_encode_decode_roundtrip_large():
    ctx = Ctx(synth.param_set("toy"))
    z = synth.slots(12, "enc", ctx.N // 2)
    m = ctx.encode_coeffs(z, 2.0 ** 40)
    assert np.max(np.abs(ctx.decode_coeffs(m.astype(np.float64), 2.0 ** 40) - z)) < 2 ** -30


# ----------------------------------------------------------------- basis conversion / ModDown / rescale
def _crt(res_cols, basis):
    """Integers in [0, prod) from residue columns (one per coefficient)."""
    M = math.prod(basis)
    out = []
    for col in res_cols:
        x = 0
        for r, m in zip(col, basis):
            Mi = M // m
            x += int(r) * Mi * pow(Mi, -1, m)
        out.append(x % M)
    return out


def test_decompose_digit_is_fast_bconv(tiny):
    """Digit b equals c mod Q_b plus u Q_b with 0 <= u < |b| on every modulus
    of the extended basis (exact CRT with big integers)."""
    level = 4
    Q = tiny.basis(level, False)
    ext = tiny.basis(level, True)
    c = tiny.ntt(_rand_poly(tiny, Q, 13), Q)
    digits = tiny.decompose(c, level)
    coeff = tiny.intt(c, Q)
    assert len(digits) == tiny.beta(level) == 2
    for b, d in enumerate(digits):
        rng = tiny.digit_range(b, level)
        Qb_list = [Q[j] for j in rng]
        Qb = math.prod(Qb_list)
        cval = _crt(coeff[rng.start:rng.stop].T, Qb_list)
        dval = _crt(tiny.intt(d, ext).T, ext)
        for i in range(tiny.N):
            u, rem = divmod(dval[i] - cval[i], Qb)
            assert rem == 0 and 0 <= u < len(Qb_list), (b, i, u)


def test_moddown_is_floor_division_within_k(tiny):
    """ModDown(x) = floor(x / P) - u mod Q with 0 <= u < k (Eq. 4)."""
    level = 3
    ext = tiny.basis(level, True)
    Q = tiny.basis(level, False)
    x = tiny.ntt(_rand_poly(tiny, ext, 14), ext)
    out = tiny.intt(tiny.moddown(x, level), Q)
    xv = _crt(tiny.intt(x, ext).T, ext)
    Qm = math.prod(Q)
    ov = _crt(out.T, Q)
    for a, o in zip(xv, ov):
        u = (a // tiny.P - o) % Qm
        assert 0 <= u < tiny.k


def test_rescale_is_exact_floor(tiny):
    """Eq. (1): out = (x - [x]_{q_last}) / q_last exactly."""
    level = 4
    Q = tiny.basis(level, False)
    x = tiny.ntt(_rand_poly(tiny, Q, 15), Q)
    out = tiny.intt(tiny.rescale(x, level), Q[:-1])
    xv = _crt(tiny.intt(x, Q).T, Q)
    ov = _crt(out.T, Q[:-1])
    for a, o in zip(xv, ov):
        assert o == a // Q[-1]


def test_moddown_rescale_bound(tiny):
    """Merged ModDown + rescale = floor(x / (P q_last)) - u, 0 <= u < k + 1."""
    level = 4
    ext = tiny.basis(level, True)
    Q = tiny.basis(level, False)
    x = tiny.ntt(_rand_poly(tiny, ext, 16), ext)
    out = tiny.intt(tiny.moddown_rescale(x, level), Q[:-1])
    xv = _crt(tiny.intt(x, ext).T, ext)
    Pp = tiny.P * Q[-1]
    Qm = math.prod(Q[:-1])
    ov = _crt(out.T, Q[:-1])
    for a, o in zip(xv, ov):
        u = (a // Pp - o) % Qm
        assert 0 <= u < tiny.k + 1


def test_moddown_rescale_without_p_is_rescale():
    """With k = 0 the merged step reduces exactly to Eq. (1)."""
    ps = synth.param_set("tiny")
    ctx = Ctx(synth.ParamSet("nop", ps.log_n, ps.q, (), 2))
    Q = ctx.basis(4, False)
    x = ctx.ntt(_rand_poly(ctx, Q, 17), Q)
    assert np.array_equal(ctx.moddown_rescale(x, 4), ctx.rescale(x, 4))


# ----------------------------------------------------------------- complexity tables
def test_tops_table_reproduced():
    """Table "number of modular multiplications and switching key size"
    (N = 2^16, n = 2^15, L + 1 = 32, alpha = 12, w = 54)."""
    with open(os.path.join(GOLDEN, "tops_table.json")) as f:
        g = json.load(f)
    for row in g["rows"]:
        split = tuple(row["split"])
        gib = cost_model.swk_gib(row["algo"], split, 2 ** 16, 32, 12, 54)
        assert abs(gib - row["swk_gib"]) < 0.01, (row, gib)
        if row.get("modmul_pinned", True):
            mm = cost_model.modmul_count(row["algo"], split, 2 ** 16, 32, 12)
            assert abs(mm - row["modmul"]) / row["modmul"] < 0.005, (row, mm)


def test_rotation_count_comment_formula():
    """Eq. (6) needs n'1 - 1 + (n'2 - 1) n'1 + n'3 - 1 = n'1 n'2 + n'3 - 2 rotations."""
    for n1, n2, n3 in [(2, 4, 8), (4, 8, 8), (32, 32, 32), (4, 128, 64)]:
        c = cost_model.counts("th", (n1, n2, n3), 3, 32, 12, n1 * n2 * n3)
        assert c["ks_products"] == (n1 - 1) + (n2 - 1) * n1 + (n3 - 1)
