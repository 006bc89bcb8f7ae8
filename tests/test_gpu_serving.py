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
