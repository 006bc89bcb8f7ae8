"""Degenerate and extreme LT shapes on the GPU, bit-exact with the oracle: a
single diagonal under every algorithm, a prime diagonal count under every
split that factors it, the widest outer layer (n'3 = 64, one multi-key launch
of 63 keys) and the widest baby layer (n'1 = 64), an empty batch, and a
one-stage chain, which must equal lt_eval."""
import numpy as np
import pytest

from oracle import lt as olt
from oracle.workload import make_problem

from gpu_common import assert_same, ensure_keys, gpu_context, oracle_lt, upload_problem

pytestmark = pytest.mark.gpu


def max_err(pb, ct):
    e = pb.decrypt((ct[0], ct[1])) - pb.expected()
    return float(np.max(np.abs(e)))


@pytest.mark.parametrize("D,algo,split", [
    (1, "diag", None), (1, "th", (1, 1, 1)), (1, "dh", (1, 1)), (1, "bsgs", (1, 1)),
    (3, "th", (3, 1, 1)), (3, "th", (1, 3, 1)), (3, "th", (1, 1, 3)), (3, "dh", (3, 1)), (3, "dh", (1, 3)),
    (3, "bsgs", (3, 1)), (3, "bsgs", (1, 3)), (3, "diag", None),
])
def test_tiny_and_prime_diagonal_counts(D, algo, split):
    pb = make_problem("toy", 9, D)
    ensure_keys(pb, algo, split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, algo, split)
    got = out.numpy()
    assert_same(got, oracle_lt(pb, algo, split), f"D={D} {algo} {split}")
    assert max_err(pb, got) <= 1e-5


@pytest.mark.parametrize("split", [(1, 1, 64), (64, 1, 1)])
def test_widest_layers(split):
    pb = make_problem("toy", 10, 64)
    ensure_keys(pb, "th", split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    out, _ = g.lt_eval(g.ct_from_host(np.stack(pb.ct)), f, "th", split)
    got = out.numpy()
    assert_same(got, oracle_lt(pb, "th", split), f"th {split}")
    assert max_err(pb, got) <= 1e-5


def test_empty_batch_and_one_stage_chain():
    pb = make_problem("toy", 11, 16)
    ensure_keys(pb, "th", (2, 2, 4))
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    assert g.lt_eval_batch([], [], algos=[], splits=[]) == []
    ct = g.ct_from_host(np.stack(pb.ct))
    single, _ = g.lt_eval(ct, f, "th", (2, 2, 4))
    chained, chosen = g.lt_eval_chain(ct, [f], splits=[(2, 2, 4)])
    assert chosen == [(2, 2, 4)]
    assert_same(chained.numpy(), single.numpy(), "one-stage chain vs lt_eval")
    assert_same(single.numpy(), np.stack(olt.lt_th_bsgs(pb.ctx, pb.ct, pb.diags, pb.keys, 2, 2, 4)[0]), "oracle")
