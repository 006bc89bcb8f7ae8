"""End-to-end parity of lt_eval with the CPU oracle: every algorithm, several
splits, strided offsets, lower levels, the library's own split choice, and
the full-size workload (N = 2^16, 24 Q limbs, 4 special primes, dnum 6,
256 consecutive diagonals).  Output residues must be identical bit for bit;
the decrypted result must match the FP64 product within 1e-5 (64 diagonals)
or 1e-4 (256 diagonals)."""
import numpy as np
import pytest

from oracle.workload import make_problem
from paper_2605_17222_gb300 import binding

from gpu_common import TOY_SPLITS, assert_same, ensure_keys, gpu_context, oracle_lt, upload_problem

pytestmark = pytest.mark.gpu


def max_err(pb, ct):
    y = pb.decrypt((ct[0], ct[1]))
    e = y - pb.expected()
    return float(np.max(np.maximum(np.abs(e.real), np.abs(e.imag))))


@pytest.fixture(scope="module")
def toy():
    pb = make_problem("toy", 0, 64)
    for algo, split in TOY_SPLITS.items():
        ensure_keys(pb, algo, split)
    for split in [(2, 4, 8), (1, 8, 8), (8, 1, 8), (8, 8, 1), (1, 64, 1), (16, 2, 2)]:
        ensure_keys(pb, "th", split)
    ensure_keys(pb, "dh", (4, 16))
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    return pb, g, f


@pytest.mark.parametrize("algo", list(TOY_SPLITS))
def test_toy_all_algorithms(toy, algo):
    pb, g, f = toy
    split = TOY_SPLITS[algo]
    want = oracle_lt(pb, algo, split)
    out, chosen = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    got = out.numpy()
    assert_same(got, want, f"toy {algo}")
    assert max_err(pb, got) <= 1e-5


@pytest.mark.parametrize("algo,split", [("th", (2, 4, 8)), ("th", (1, 8, 8)), ("th", (8, 8, 1)),
                                        ("th", (16, 2, 2)), ("dh", (4, 16))])
def test_toy_other_splits(toy, algo, split):
    pb, g, f = toy
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    assert_same(out.numpy(), oracle_lt(pb, algo, split), f"toy {algo} {split}")


def test_toy_special_splits_match_other_algorithms(toy):
    """TH(1, 8, 8) == TH(8, 1, 8) == DH(8, 8) -- DH's two schedules, baby steps
    fused into the diagonal kernel or materialised -- and TH(1, 64, 1) ==
    diagonal method, on the GPU too."""
    pb, g, f = toy
    ct = g.ct_from_host(np.stack(pb.ct))
    a, _ = g.lt_eval(ct, f, "th", (1, 8, 8))
    a2, _ = g.lt_eval(ct, f, "th", (8, 1, 8))
    b, _ = g.lt_eval(ct, f, "dh", (8, 8))
    assert g.dh_schedule(f, pb.level, (8, 8)) in ("fused", "baby")
    assert_same(a.numpy(), b.numpy(), "TH(1,8,8) vs DH(8,8)")
    assert_same(a2.numpy(), b.numpy(), "TH(8,1,8) vs DH(8,8)")
    c, _ = g.lt_eval(ct, f, "th", (1, 64, 1))
    d, _ = g.lt_eval(ct, f, "diag")
    assert_same(c.numpy(), d.numpy(), "TH(1,64,1) vs diagonal")


def test_toy_strided_lower_level():
    """Offsets strided by 4 (a CoeffToSlot-like stage) at level 3, and the
    minimum level 2."""
    for level, stride, D, split in [(3, 4, 16, (2, 2, 4)), (2, 1, 8, (2, 2, 2))]:
        pb = make_problem("toy", 3, D, level=level, stride=stride)
        ensure_keys(pb, "th", split)
        g = gpu_context("toy")
        f = upload_problem(g, pb, stride=stride)
        out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th", split)
        got = out.numpy()
        assert_same(got, oracle_lt(pb, "th", split), f"strided level {level}")
        assert max_err(pb, got) <= 1e-5


def test_toy_autotuned_split(toy):
    pb, g, f = toy
    split = g.choose_split("th", pb.level, pb.D)
    ensure_keys(pb, "th", split)
    upload_problem(g, pb)
    out, chosen = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th")
    assert chosen == split
    assert_same(out.numpy(), oracle_lt(pb, "th", split), f"auto {split}")


def test_missing_key_is_reported(toy):
    """A context holding only some keys refuses the LT with CKKS_ENOKEY before any launch."""
    pb, _, _ = toy
    g = gpu_context("toy")
    g.upload_rotation_key(1, pb.keys[1])
    f = g.upload_diagonals(pb.diags)
    with pytest.raises(binding.CkksError) as e:
        g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th", (2, 2, 16))
    assert e.value.status == 3


def test_bad_split_is_rejected(toy):
    pb, g, f = toy
    with pytest.raises(binding.CkksError) as e:
        g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th", (3, 3, 3))
    assert e.value.status == 1


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def full():
    """N = 2^16, Q = 55b + 23x40b, P = 4x60b, dnum 6, D = 256 consecutive, seed 1."""
    pb = make_problem("n16", 1, 256)
    g = gpu_context("n16")
    f = upload_problem(g, pb)
    return pb, g, f


@pytest.mark.parametrize("algo,split", [("th", (4, 8, 8)), ("dh", (16, 16)), ("bsgs", (16, 16))])
def test_full_size_bit_exact(full, algo, split):
    pb, g, f = full
    ensure_keys(pb, algo, split)
    upload_problem(g, pb)
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    got = out.numpy()
    assert_same(got, oracle_lt(pb, algo, split), f"full {algo} {split}")
    assert max_err(pb, got) <= 1e-4


def test_full_size_autotuned_th(full):
    pb, g, f = full
    split = g.choose_split("th", pb.level, pb.D)
    ensure_keys(pb, "th", split)
    upload_problem(g, pb)
    out, chosen = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th")
    assert chosen == split
    assert_same(out.numpy(), oracle_lt(pb, "th", split), f"full auto {split}")


def test_toy_dh_autotuner_times_both_schedules(toy):
    """lt_autotune for DH-BSGS times each candidate in both schedules and keeps
    the faster; the LT then runs with it, bit-exact with the oracle."""
    pb, g, f = toy
    ct = g.ct_from_host(np.stack(pb.ct))
    cands = g.candidate_splits("dh", pb.level, pb.D, 3)
    for sp in cands:
        ensure_keys(pb, "dh", sp[:2])
    upload_problem(g, pb)
    split, ms = g.autotune("dh", ct, f, 3)
    assert split in cands and ms > 0
    assert g.dh_schedule(f, pb.level, split) in ("fused", "baby")
    out, chosen = g.lt_eval(ct, f, "dh")
    assert chosen == split
    assert_same(out.numpy(), oracle_lt(pb, "dh", split[:2]), f"DH autotuned {split}")


@pytest.mark.parametrize("split", [(4, 4, 4), (2, 4, 8), (1, 8, 8)])
def test_toy_every_diagonal_kernel_tile(toy, split):
    """Every tile of the diagonal kernel (outer indices per CTA below the
    default; 128, 256 or 512 positions per CTA) gives the oracle's residues."""
    pb, g, f = toy
    ct = g.ct_from_host(np.stack(pb.ct))
    want = oracle_lt(pb, "th", split)
    k3 = 1
    while k3 < split[2] and k3 < 8:
        k3 *= 2
    try:
        for outer in sorted({0, k3 // 2 or 0, 1}):
            for pos in (0, 128, 256, 512):
                g.debug_diag_mac_tile(outer, pos)
                out, _ = g.lt_eval(ct, f, "th", split)
                assert_same(out.numpy(), want, f"toy {split} tile ({outer}, {pos})")
    finally:
        g.debug_diag_mac_tile(0, 0)


def test_toy_measuring_autotuner(toy):
    """lt_autotune times the model's candidates that have keys, records the
    fastest, and lt_eval without a split then uses it (bit-exact with the oracle)."""
    pb, g, f = toy
    ct = g.ct_from_host(np.stack(pb.ct))
    cands = g.candidate_splits("th", pb.level, pb.D, 4)
    assert all(a * b * c == pb.D for a, b, c in cands)
    for sp in cands:
        ensure_keys(pb, "th", sp)
    upload_problem(g, pb)
    split, ms = g.autotune("th", ct, f, 4)
    assert split in cands and ms > 0
    assert g.tuned_tile("th", f, pb.level) is not None
    out, chosen = g.lt_eval(ct, f, "th")
    assert chosen == split
    assert_same(out.numpy(), oracle_lt(pb, "th", split), f"autotuned {split}")


def test_cost_model_is_the_one_restated_on_cpu():
    """lt_model_estimate computes exactly the model tests/test_cost_model.py
    restates and checks against measured DRAM bytes and LT times."""
    from test_cost_model import model

    g = gpu_context("n16")
    for sp in [(1, 64, 4), (2, 32, 4), (4, 16, 4), (4, 8, 8), (2, 16, 8), (1, 32, 8)]:
        b, s = g.model_estimate("th", 24, 256, sp)
        wb, ws = model(24, 256, *sp)
        assert abs(b - wb) <= 1e-9 * wb and abs(s - ws) <= 1e-9 * ws, (sp, b, wb, s, ws)
    g.close()
