"""The serving loop on the GPU: requests at mixed levels and on two matrices,
submitted while earlier batches run, each give the residues a separate
lt_eval gives, bit for bit; latencies are recorded."""
import time

import numpy as np
import pytest

from oracle import lt as olt
from oracle.workload import add_keys, make_problem
from paper_2605_17222_gb300 import synth
from paper_2605_17222_gb300.serving import LtServer, Request, percentile

from gpu_common import assert_same, gpu_context, upload_problem

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    pb = make_problem("toy", 5, 64)
    pb16 = make_problem("toy", 6, 16)
    g = gpu_context("toy")
    for split in {g.choose_split("th", lv, d) for lv in (2, 3, 4) for d in (64, 16)}:
        add_keys(pb, olt.rotation_set("th", split[0] * split[1] * split[2], split, 1, pb.ctx.N // 2))
    f64 = upload_problem(g, pb)
    f16 = g.upload_diagonals(pb16.diags, stride=1, level=pb16.ctx.L)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(14):
        lvl = int(rng.choice([2, 3, 4]))
        z = synth.slots(200 + i, f"srv/{i}", pb.ctx.N // 2)
        ct = pb.ctx.encrypt(z, pb.s, lvl, pb.scale, 200 + i, stream=f"srv/{i}")
        reqs.append((g.ct_from_host(np.stack(ct)), f64 if i % 3 else f16))
    srv = LtServer({"toy": g}, hbm_budget=8e9, streams=3, max_batch=4)
    t0 = time.perf_counter()
    sent = []
    for i, (ct, f) in enumerate(reqs):  # arrivals interleaved with scheduling
        r = Request(i, "toy", f, ct, time.perf_counter())
        srv.submit(r)
        sent.append(r)
        srv.step()
    srv.drain(timeout_s=60)
    assert srv.stats.completed == len(reqs)
    assert srv.stats.batches >= 2
    for r in sent:
        alone, _ = g.lt_eval(r.ct, r.matrix, "th", r.split)
        assert_same(r.out.numpy(), alone.numpy(), f"request {r.rid}")
    lat = srv.stats.latencies
    assert len(lat) == len(reqs) and percentile(lat, 99) < 60 and time.perf_counter() - t0 < 120


def test_two_ring_degrees_alone_equal_in_the_mix():
    """The serving workload's two contexts, N = 2^15 (Q = 50b + 15x40b, P =
    3x60b, dnum 4) and N = 2^16 (the benchmark parameters), served together
    from one queue: requests at several levels and diagonal counts arrive
    while earlier batches run, and each output equals a separate lt_eval of
    the same request bit for bit.  Values are uniform residues (the identity
    alone = in the mix needs no decryption)."""
    import torch

    from paper_2605_17222_gb300 import binding

    rng = np.random.default_rng(11)
    ctxs, mats, cts = {}, {}, {}
    for ln, name, levels in [(15, "n15", (6, 11, 16)), (16, "n16", (6, 15, 24))]:
        ps = synth.param_set(name)
        g = binding.Context.from_params(ps)
        ctxs[ln] = g
        rots = set()
        for d in (32, 64):
            for lv in levels:
                rots |= set(g.required_rotations("th", g.choose_split("th", lv, d), d, 1))
        for r in sorted(rots):
            g.upload_rotation_key_device(r, synth.uniform_mod_device(7, f"srv2/key/{ln}/{r}", ps.moduli, ps.n,
                                                                     count=2 * g.beta_max))
        top = list(ps.q) + list(ps.p)
        for d in (32, 64):
            mats[(ln, d)] = g.upload_diagonals_device(synth.uniform_mod_device(7, f"srv2/diag/{ln}/{d}", top, ps.n,
                                                                               count=d), stride=1, level=ps.L)
        for lv in levels:
            cts[(ln, lv)] = g.ct_wrap(synth.uniform_mod_device(7, f"srv2/ct/{ln}/{lv}", list(ps.q[:lv]), ps.n,
                                                               count=2), lv)
    torch.cuda.synchronize()
    srv = LtServer(ctxs, hbm_budget=60e9, streams=4, max_batch=4)
    sent = []
    for i in range(24):
        ln = int(rng.choice([15, 16]))
        lv = int(rng.choice((6, 11, 16) if ln == 15 else (6, 15, 24)))
        d = int(rng.choice([32, 64]))
        r = Request(i, ln, mats[(ln, d)], cts[(ln, lv)], time.perf_counter())
        srv.submit(r)
        sent.append(r)
        if i % 2:
            srv.step()
    srv.drain(timeout_s=120)
    assert srv.stats.completed == len(sent) and srv.stats.batches >= 4
    assert {r.ctx_key for r in sent} == {15, 16}
    for r in sent:
        alone, _ = ctxs[r.ctx_key].lt_eval(r.ct, r.matrix, "th", r.split)
        assert_same(r.out.numpy(), alone.numpy(), f"request {r.rid} (N = 2^{r.ctx_key})")
