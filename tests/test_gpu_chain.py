"""Diagonal windows with a base offset (offsets offset0 + stride t) and chains
of LTs on the GPU, bit-exact with the oracle: every algorithm over the window
-7 + 2t, an outer amount that wraps to 0, a batch over based windows, and the
factored slot DFT (SlotToCoeff and CoeffToSlot, Sec. I's multi-stage sparse
LTs) through lt_eval_chain at N = 2^12 and N = 2^16."""
import numpy as np
import pytest

from oracle import lt as olt
from oracle.workload import make_chain_problem, make_problem

from gpu_common import assert_same, ensure_keys, gpu_context, oracle_lt, upload_chain, upload_problem

pytestmark = pytest.mark.gpu

BASED_SPLITS = {"diag": None, "bsgs": (4, 4), "dh": (4, 4), "th": (2, 2, 4)}


def max_err(pb, ct):
    e = pb.decrypt((ct[0], ct[1])) - pb.expected()
    return float(np.max(np.maximum(np.abs(e.real), np.abs(e.imag))))


@pytest.fixture(scope="module")
def based():
    """toy parameters at level 3, 16 diagonals at offsets -7, -5, .., 23, seed 5."""
    pb = make_problem("toy", 5, 16, level=3, stride=2, offset0=-7)
    for algo, sp in BASED_SPLITS.items():
        ensure_keys(pb, algo, sp)
    for sp in [(1, 16, 1), (4, 1, 4), (8, 2, 1)]:
        ensure_keys(pb, "th", sp)
    g = gpu_context("toy")
    f = upload_problem(g, pb, stride=2)
    return pb, g, f


@pytest.mark.parametrize("algo", list(BASED_SPLITS))
def test_based_window_every_algorithm(based, algo):
    pb, g, f = based
    split = BASED_SPLITS[algo]
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    got = out.numpy()
    assert_same(got, oracle_lt(pb, algo, split), f"based {algo}")
    assert max_err(pb, got) <= 1e-5


def test_based_window_special_splits(based):
    """TH(1, D, 1) == diagonal method and TH(4, 1, 4) == DH(4, 4) with a base offset."""
    pb, g, f = based
    ct = g.ct_from_host(np.stack(pb.ct))
    a, _ = g.lt_eval(ct, f, "th", (1, 16, 1))
    b, _ = g.lt_eval(ct, f, "diag")
    assert_same(a.numpy(), b.numpy(), "TH(1,16,1) vs diagonal")
    c, _ = g.lt_eval(ct, f, "th", (4, 1, 4))
    d, _ = g.lt_eval(ct, f, "dh", (4, 4))
    assert_same(c.numpy(), d.numpy(), "TH(4,1,4) vs DH(4,4)")
    e, _ = g.lt_eval(ct, f, "th", (8, 2, 1))
    assert_same(e.numpy(), oracle_lt(pb, "th", (8, 2, 1)), "TH(8,2,1)")


def test_required_rotations_match_the_oracle(based):
    pb, g, _ = based
    n = pb.ctx.N // 2
    for algo, sp in BASED_SPLITS.items():
        assert g.required_rotations(algo, sp, 16, 2, offset0=-7) == olt.rotation_set(algo, 16, sp, 2, n, -7)


def test_outer_amount_wrapping_to_zero():
    """offset0 = -16, stride 2, split (2, 2, 4): the k = 2 outer amount is 0 and
    its partial sum seeds the accumulator (no key); DH(4, 4) likewise at j = 2."""
    pb = make_problem("toy", 6, 16, level=3, stride=2, offset0=-16)
    ensure_keys(pb, "th", (2, 2, 4))
    ensure_keys(pb, "dh", (4, 4))
    ensure_keys(pb, "bsgs", (4, 4))
    g = gpu_context("toy")
    f = upload_problem(g, pb, stride=2)
    ct = g.ct_from_host(np.stack(pb.ct))
    for algo, sp in [("th", (2, 2, 4)), ("dh", (4, 4)), ("bsgs", (4, 4))]:
        out, _ = g.lt_eval(ct, f, algo, sp)
        assert_same(out.numpy(), oracle_lt(pb, algo, sp), f"wrap {algo}")
        assert max_err(pb, out.numpy()) <= 1e-5


def test_batch_over_based_windows(based):
    """lt_eval_batch over the based window at levels 3 and 2 plus a plain
    window: each item equals its separate lt_eval."""
    pb, g, f = based
    plain = make_problem("toy", 5, 8, level=3)
    ensure_keys(plain, "th", (2, 2, 2))
    fp = upload_problem(g, plain)
    lv2 = pb.ctx.encrypt(pb.z, pb.s, 2, pb.scale, 77, stream="lv2")
    ins = [g.ct_from_host(np.stack(pb.ct)), g.ct_from_host(np.stack(lv2)), g.ct_from_host(np.stack(plain.ct)),
           g.ct_from_host(np.stack(pb.ct))]
    fs = [f, f, fp, f]
    splits = [(2, 2, 4), (2, 2, 4), (2, 2, 2), (2, 2, 4)]
    outs = g.lt_eval_batch(ins, fs, algos=["th"] * 4, splits=splits)
    for n in range(4):
        single, _ = g.lt_eval(ins[n], fs[n], "th", splits[n])
        assert_same(outs[n].numpy(), single.numpy(), f"item {n}")
    assert_same(outs[0].numpy(), oracle_lt(pb, "th", (2, 2, 4)), "item 0 vs oracle")


# ---------------------------------------------------------------- chains: the factored slot DFT
@pytest.mark.parametrize("kind,radices,splits,tol", [
    ("stc", [4, 4, 3], [(2, 2, 8), (4, 4, 2), (2, 2, 2)], 1e-5),
    ("cts", [3, 4, 4], [(2, 2, 2), (4, 4, 2), (2, 2, 8)], 1e-6),
])
def test_toy_dft_chain(kind, radices, splits, tol):
    """N = 2^12: three LTs from level 4 to level 1 in one lt_eval_chain call,
    bit-exact with the oracle's chain; decrypts to U z[R] (StC) or
    (U^H z / n)[R] (CtS)."""
    cp = make_chain_problem("toy", 2, kind, radices, splits)
    g = gpu_context("toy")
    fs = upload_chain(g, cp)
    out, chosen = g.lt_eval_chain(g.ct_from_host(np.stack(cp.ct)), fs, splits=splits)
    assert chosen == [tuple(s) for s in splits]
    got = out.numpy()
    assert_same(got, np.stack(olt.lt_chain(cp.ctx, cp.ct, cp.stages(), cp.keys)), f"{kind} chain")
    y = cp.decrypt((got[0], got[1]))
    assert np.max(np.abs(y - cp.expected())) < tol


def test_chain_rejects_a_missing_level():
    """Four stages on a level-4 input (one level per stage) are refused before any launch."""
    cp = make_chain_problem("toy", 2, "stc", [4, 4, 3], [(2, 2, 8), (4, 4, 2), (2, 2, 2)])
    g = gpu_context("toy")
    fs = upload_chain(g, cp)
    from paper_2605_17222_gb300 import binding
    with pytest.raises(binding.CkksError):
        g.lt_eval_chain(g.ct_from_host(np.stack(cp.ct)), fs + [fs[0]], out=g.ct_empty(1))


def test_full_size_coeff_to_slot_chain():
    """N = 2^16 (32768 slots), CoeffToSlot in three levels (radices 5, 5, 5:
    32, 64 and 64 diagonals at strides 1024, 32 and 1) from level 24 to 21.

    The error has two parts.  Most slots see white rounding noise (median
    about 2e-8 here).  A few low-frequency slots also see the bias of the
    rounding in c1: the fast basis conversion of the merged ModDown + rescale
    leaves u in [0, k + 1) and the floor rescale of Eq. 1 leaves -1/2, both
    with nonzero mean mu.  Decryption turns mu (1 + X + .. + X^(N-1)) s into
    mu (2 / (1 - xi)) s(xi) at slot xi, which peaks near xi = zeta:
    about mu (2N / pi) sqrt(N) / 2^40, roughly 2e-5 per stage."""
    cp = make_chain_problem("n16", 8, "cts", [5, 5, 5], [(2, 4, 4), (4, 4, 4), (4, 4, 4)])
    assert [(w.offset0, w.stride, w.D) for w in cp.windows] == [(0, 1024, 32), (-992, 32, 64), (-31, 1, 64)]
    g = gpu_context("n16")
    fs = upload_chain(g, cp)
    out, _ = g.lt_eval_chain(g.ct_from_host(np.stack(cp.ct)), fs, splits=cp.splits)
    got = out.numpy()
    assert_same(got, np.stack(olt.lt_chain(cp.ctx, cp.ct, cp.stages(), cp.keys)), "n16 CtS chain")
    err = np.abs(cp.decrypt((got[0], got[1])) - cp.expected())
    assert np.median(err) < 1e-7
    assert np.max(err) < 5e-5


def test_recorded_chain_replays_on_new_inputs():
    """lt_graph_begin/end records an lt_eval_chain queued on a created stream;
    replays recompute from the input's current contents, bit-exact with the
    oracle; the legacy default stream is refused."""
    import torch
    from paper_2605_17222_gb300 import binding
    cp = make_chain_problem("toy", 2, "stc", [4, 4, 3], [(2, 2, 8), (4, 4, 2), (2, 2, 2)])
    g = gpu_context("toy")
    fs = upload_chain(g, cp)
    ct = g.ct_from_host(np.stack(cp.ct))
    out = g.ct_empty(1)
    st = torch.cuda.Stream()
    g.lt_eval_chain(ct, fs, splits=cp.splits, out=out, stream=st)  # first use sets up the tables
    st.synchronize()
    g.graph_begin(st)
    g.lt_eval_chain(ct, fs, splits=cp.splits, out=out, stream=st)
    rec = g.graph_end(st, keep=(ct, out, fs))
    out.tensor.zero_()
    rec.launch(st)
    st.synchronize()
    assert_same(out.numpy(), np.stack(olt.lt_chain(cp.ctx, cp.ct, cp.stages(), cp.keys)), "replay 1")
    ct2 = cp.ctx.encrypt(cp.z[::-1].copy(), cp.s, cp.level, cp.scale, 41, stream="replay")
    ct.tensor.copy_(torch.from_numpy(np.stack(ct2).view(np.int64)).cuda())
    torch.cuda.synchronize()
    rec.launch(st)
    st.synchronize()
    assert_same(out.numpy(), np.stack(olt.lt_chain(cp.ctx, ct2, cp.stages(), cp.keys)), "replay 2")
    rec.close()
    with pytest.raises(binding.CkksError) as e:
        g.graph_begin(0)
    assert e.value.status == 1


@pytest.mark.parametrize("algo,split", [("th", (4, 4, 4)), ("dh", (8, 8)), ("bsgs", (8, 8))])
def test_full_size_based_window_every_hoisting(algo, split):
    """N = 2^16 at level 24: 64 diagonals at offsets -31*32 .. +32*32 (stride 32,
    the middle stage of a radix-32 CoeffToSlot), bit-exact with the oracle for
    TH-BSGS, DH-BSGS and BSGS."""
    pb = make_problem("n16", 12, 64, stride=32, offset0=-992)
    ensure_keys(pb, algo, split)
    g = gpu_context("n16")
    f = upload_problem(g, pb, stride=32)
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    got = out.numpy()
    assert_same(got, oracle_lt(pb, algo, split), f"n16 based {algo} {split}")
    assert max_err(pb, got) <= 1e-4
