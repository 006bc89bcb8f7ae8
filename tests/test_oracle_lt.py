"""The oracle's key switching and the four LT algorithms, pinned against the
FP64 matrix-vector product, the paper's operation counts, and the bitwise
identities the algorithms imply.  CPU only."""
import numpy as np
import pytest

from oracle import cost_model
from oracle import lt as olt
from oracle.ckks import Ops
from oracle.workload import add_keys, make_problem

TOY_SPLITS = {"diag": None, "bsgs": (8, 8), "dh": (8, 8), "th": (4, 4, 4)}


@pytest.fixture(scope="module")
def toy():
    """Functional toy: N = 2^12, Q = 50b + 3x40b, P = 60b, dnum 4, D = 64, seed 0."""
    pb = make_problem("toy", 0, 64)
    rots = set()
    for algo, split in TOY_SPLITS.items():
        rots |= set(olt.rotation_set(algo, 64, split, 1, pb.ctx.N // 2))
    rots |= set(olt.rotation_set("th", 64, (1, 8, 8), 1, pb.ctx.N // 2))
    add_keys(pb, rots)
    return pb


def test_rotation_decrypts_to_rotated_slots(toy):
    ctx = toy.ctx
    for r in [1, 3, 8]:
        out = ctx.rotate(toy.ct, r, ctx.key_at_level(toy.keys[r], toy.level), toy.level)
        z = ctx.decrypt(out, toy.s, toy.scale)
        assert np.max(np.abs(z - np.roll(toy.z, -r))) < 1e-6


def test_hoisting_identity(toy):
    """phi_r(<d, phi_{-r}(swk)>) = <phi_r(d), swk> bit for bit (the form the
    GPU evaluates: the automorphism is a pure permutation in the NTT domain)."""
    ctx = toy.ctx
    lvl = toy.level
    d = ctx.decompose(toy.ct[1], lvl)
    key = ctx.key_at_level(toy.keys[3], lvl)
    x0, x1 = ctx.inner(d, ctx.hoisted_key(key, 3), lvl)
    y0, y1 = ctx.inner([ctx.auto_ntt(db, 3) for db in d], key, lvl)
    assert np.array_equal(ctx.auto_ntt(x0, 3), y0)
    assert np.array_equal(ctx.auto_ntt(x1, 3), y1)


@pytest.fixture(scope="module")
def toy_results(toy):
    res = {}
    for algo, split in TOY_SPLITS.items():
        res[algo] = olt.run(toy.ctx, algo, toy.ct, toy.diags, toy.keys, split)
    return res


@pytest.mark.parametrize("algo", list(TOY_SPLITS))
def test_lt_matches_fp64(toy, toy_results, algo):
    """Every algorithm decrypts to the FP64 product within 1e-5 at 64 diagonals."""
    ct, _ = toy_results[algo]
    y = toy.decrypt(ct)
    err = np.max(np.maximum(np.abs((y - toy.expected()).real), np.abs((y - toy.expected()).imag)))
    assert err <= 1e-5, err


def test_algorithms_agree(toy, toy_results):
    ys = {a: toy.decrypt(r[0]) for a, r in toy_results.items()}
    for a in ys:
        assert np.max(np.abs(ys[a] - ys["th"])) <= 1e-6


@pytest.mark.parametrize("algo", list(TOY_SPLITS))
def test_op_counts_match_paper(toy, toy_results, algo):
    """Table "complexity comparisons" (TH-BSGS Decompose/ModDown per Alg. 2)."""
    _, ops = toy_results[algo]
    ctx = toy.ctx
    beta = ctx.beta(toy.level)
    split = TOY_SPLITS[algo] or ()
    want = cost_model.counts(algo, split, beta, toy.level, ctx.k, toy.D)
    assert ops.decompose == want["decompose"]
    assert ops.moddown == want["moddown"]
    assert ops.ks_products == want["ks_products"]
    assert ops.cw_mult == want["cw_mult"]
    assert len(ops.keys) == want["keys"]


def test_th_reduces_to_dh_and_diag(toy, toy_results):
    """TH(1, n2, n3) == DH(n2, n3) and TH(1, D, 1) == DH(D, 1) == diagonal, bit for bit."""
    ctx = toy.ctx
    th = olt.lt_th_bsgs(ctx, toy.ct, toy.diags, toy.keys, 1, 8, 8)[0]
    dh = olt.lt_dh_bsgs(ctx, toy.ct, toy.diags, toy.keys, 8, 8)[0]
    assert all(np.array_equal(a, b) for a, b in zip(th, dh))
    th1 = olt.lt_th_bsgs(ctx, toy.ct, toy.diags, toy.keys, 1, 64, 1)[0]
    dh1 = olt.lt_dh_bsgs(ctx, toy.ct, toy.diags, toy.keys, 64, 1)[0]
    dg = toy_results["diag"][0]
    assert all(np.array_equal(a, b) for a, b in zip(th1, dh1))
    assert all(np.array_equal(a, b) for a, b in zip(th1, dg))


def test_strided_offsets_and_lower_level():
    """Offsets o_t = 4t (a CoeffToSlot-like stride) at a level below the top."""
    pb = make_problem("toy", 3, 16, level=3, stride=4)
    add_keys(pb, olt.rotation_set("th", 16, (2, 2, 4), 4, pb.ctx.N // 2))
    ct, ops = olt.lt_th_bsgs(pb.ctx, pb.ct, pb.diags, pb.keys, 2, 2, 4, stride=4)
    y = pb.decrypt(ct)
    assert np.max(np.abs(y - pb.expected())) < 1e-5
    assert ct[0].shape[0] == 2


# ---------------------------------------------------------------- base offset (offsets offset0 + stride t)
BASED_SPLITS = {"diag": None, "bsgs": (4, 4), "dh": (4, 4), "th": (2, 2, 4)}


@pytest.fixture(scope="module")
def based():
    """Offsets o_t = -7 + 2t, t < 16 (a window -7..23 at stride 2, the shape of
    one CoeffToSlot stage), toy parameters at level 3, seed 5."""
    pb = make_problem("toy", 5, 16, level=3, stride=2, offset0=-7)
    rots = set()
    for algo, split in BASED_SPLITS.items():
        rots |= set(olt.rotation_set(algo, 16, split, 2, pb.ctx.N // 2, offset0=-7))
    for split in [(1, 16, 1), (4, 1, 4), (1, 4, 4), (2, 2, 4)]:
        rots |= set(olt.rotation_set("th", 16, split, 2, pb.ctx.N // 2, offset0=-7))
    add_keys(pb, rots)
    return pb


def test_fp64_reference_with_base_is_the_dense_product():
    """The reference y = sum_t f_t . Rot(z, offset0 + stride t) equals the dense
    matrix with F[j][(j + o_t) mod n] = f_t[j] applied to z."""
    rng = np.random.default_rng(3)
    n, D, stride, off = 32, 5, 3, -4
    f = rng.standard_normal((D, n)) + 1j * rng.standard_normal((D, n))
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    M = np.zeros((n, n), dtype=np.complex128)
    for t in range(D):
        for j in range(n):
            M[j, (j + off + stride * t) % n] += f[t, j]
    assert np.allclose(olt.fp64_reference(z, f, stride, off), M @ z, atol=1e-12)


@pytest.mark.parametrize("algo", list(BASED_SPLITS))
def test_lt_with_base_matches_fp64(based, algo):
    ct, _ = olt.run(based.ctx, algo, based.ct, based.diags, based.keys, BASED_SPLITS[algo], 2, offset0=-7)
    e = based.decrypt(ct) - based.expected()
    assert np.max(np.maximum(np.abs(e.real), np.abs(e.imag))) <= 1e-5


def test_base_identities(based):
    """With a base offset: TH(1, D, 1) == diagonal method, DH(4, 4) == TH(4, 1, 4)
    == TH(1, 4, 4), bit for bit (the base joins the outermost layer in each)."""
    ctx, ct, F, K = based.ctx, based.ct, based.diags, based.keys
    th1 = olt.lt_th_bsgs(ctx, ct, F, K, 1, 16, 1, stride=2, offset0=-7)[0]
    dg = olt.lt_diag(ctx, ct, F, K, 2, offset0=-7)[0]
    assert all(np.array_equal(a, b) for a, b in zip(th1, dg))
    dh = olt.lt_dh_bsgs(ctx, ct, F, K, 4, 4, 2, offset0=-7)[0]
    for sp in [(4, 1, 4), (1, 4, 4)]:
        th = olt.lt_th_bsgs(ctx, ct, F, K, *sp, stride=2, offset0=-7)[0]
        assert all(np.array_equal(a, b) for a, b in zip(th, dh))


def test_outer_amount_wrapping_to_zero_needs_no_key():
    """offset0 = -16 at stride 2 and split (2, 2, 4): outer amounts -16 + 8k, so
    k = 2 is the identity (its partial sum is added without a key switch)."""
    pb = make_problem("toy", 6, 16, level=3, stride=2, offset0=-16)
    rots = olt.rotation_set("th", 16, (2, 2, 4), 2, pb.ctx.N // 2, offset0=-16)
    assert 0 not in rots and len(rots) == 1 + 1 + 3
    add_keys(pb, rots)
    ct, ops = olt.lt_th_bsgs(pb.ctx, pb.ct, pb.diags, pb.keys, 2, 2, 4, stride=2, offset0=-16)
    assert ops.keys == set(rots)
    assert ops.decompose == 2 + 3 and ops.moddown == 2 + 3 + 1
    e = pb.decrypt(ct) - pb.expected()
    assert np.max(np.abs(e)) <= 1e-5


def test_base_of_a_full_turn_is_no_base(toy):
    """offset0 = N/2 is the same matrix as offset0 = 0: same residues."""
    n = toy.ctx.N // 2
    a = olt.lt_th_bsgs(toy.ctx, toy.ct, toy.diags, toy.keys, 4, 4, 4)[0]
    b = olt.lt_th_bsgs(toy.ctx, toy.ct, toy.diags, toy.keys, 4, 4, 4, offset0=n)[0]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
