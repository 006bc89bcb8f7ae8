"""lt_eval_batch: ciphertexts at mixed levels and with mixed algorithms in one
call give, each, the residues a separate lt_eval gives (and the oracle's),
bit for bit."""
import numpy as np
import pytest

from oracle import lt as olt
from oracle.workload import add_keys, make_problem
from paper_2605_17222_gb300 import synth

from gpu_common import TOY_SPLITS, assert_same, ensure_keys, gpu_context, upload_problem

pytestmark = pytest.mark.gpu


def _encrypt_many(pb, levels, seed):
    cts, zs = [], []
    for n, lvl in enumerate(levels):
        z = synth.slots(seed + n, f"batch/{n}", pb.ctx.N // 2)
        cts.append(pb.ctx.encrypt(z, pb.s, lvl, pb.scale, seed + n, stream=f"batch/{n}"))
        zs.append(z)
    return cts, zs


def test_toy_batch_mixed_levels_and_algorithms():
    pb = make_problem("toy", 0, 64)
    for algo, split in TOY_SPLITS.items():
        ensure_keys(pb, algo, split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    levels = [4, 3, 2, 4, 3, 4, 4, 2]
    algos = ["th", "th", "th", "dh", "th", "diag", "bsgs", "th"]
    cts, zs = _encrypt_many(pb, levels, 50)
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    splits = [TOY_SPLITS[a] or (1, 64, 1) for a in algos]
    outs = g.lt_eval_batch(ins, [f] * len(ins), algos=algos, splits=splits)
    for n, (ct, lvl, algo) in enumerate(zip(cts, levels, algos)):
        single, _ = g.lt_eval(ins[n], f, algo, splits[n])
        got = outs[n].numpy()
        assert_same(got, single.numpy(), f"batch item {n} ({algo}, level {lvl}) vs single")
        if n < 3:
            want = np.stack(olt.run(pb.ctx, algo, ct, pb.diags, pb.keys, TOY_SPLITS[algo], 1)[0])
            assert_same(got, want, f"batch item {n} vs oracle")
            scale = pb.scale * pb.diag_scale / pb.ctx.q[lvl - 1]
            y = pb.ctx.decrypt((got[0], got[1]), pb.s, scale)
            assert np.max(np.abs(y - olt.fp64_reference(zs[n], pb.fvals))) < 1e-5


def test_full_size_batch_matches_single():
    """N = 2^16: five ciphertexts at levels 24 and 16 sharing 256 diagonals, TH (4,8,8)."""
    pb = make_problem("n16", 7, 256)
    split = (4, 8, 8)
    add_keys(pb, olt.rotation_set("th", 256, split, 1, pb.ctx.N // 2))
    g = gpu_context("n16")
    f = upload_problem(g, pb)
    levels = [24, 16, 24, 16, 24]
    cts, zs = _encrypt_many(pb, levels, 70)
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    outs = g.lt_eval_batch(ins, [f] * len(ins), algos=["th"] * len(ins), splits=[split] * len(ins))
    for n in range(len(ins)):
        single, _ = g.lt_eval(ins[n], f, "th", split)
        assert_same(outs[n].numpy(), single.numpy(), f"item {n} level {levels[n]}")
    # one item against the oracle at the lower level
    want = np.stack(olt.lt_th_bsgs(pb.ctx, cts[1], pb.diags, pb.keys, *split)[0])
    assert_same(outs[1].numpy(), want, "level-16 item vs oracle")


def test_recorded_batch_replays_on_new_inputs():
    """lt_graph: a recorded batch replays with no host work and recomputes from
    the inputs' current contents (results equal lt_eval_batch's, bit for bit)."""
    import torch
    pb = make_problem("toy", 0, 64)
    ensure_keys(pb, "th", (4, 4, 4))
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    levels = [4, 3, 4]
    cts, _ = _encrypt_many(pb, levels, 90)
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    rec = g.lt_graph(ins, [f] * 3, algos=["th"] * 3, splits=[(4, 4, 4)] * 3)
    first = [o.numpy().copy() for o in rec.launch()]
    want = [o.numpy() for o in g.lt_eval_batch(ins, [f] * 3, algos=["th"] * 3, splits=[(4, 4, 4)] * 3)]
    for a, b in zip(first, want):
        assert_same(a, b, "replay 1")
    # new input contents in the same buffers
    cts2, _ = _encrypt_many(pb, levels, 95)
    for t, ct in zip(ins, cts2):
        t.tensor.copy_(torch.from_numpy(np.stack(ct).view(np.int64)).cuda())
    second = [o.numpy() for o in rec.launch()]
    want2 = [o.numpy() for o in g.lt_eval_batch(ins, [f] * 3, algos=["th"] * 3, splits=[(4, 4, 4)] * 3)]
    for a, b in zip(second, want2):
        assert_same(a, b, "replay 2")
    assert not np.array_equal(first[0], second[0])
    rec.close()


def test_toy_batch_two_matrices_with_strides():
    """A batch mixing two matrices (16 diagonals at stride 4, 8 diagonals
    consecutive) at two levels: every item equals its separate lt_eval."""
    pa = make_problem("toy", 11, 16, stride=4)
    pb_ = make_problem("toy", 11, 8)
    g = gpu_context("toy")
    for split, pr in [((2, 2, 4), pa), ((2, 2, 2), pb_)]:
        add_keys(pa, olt.rotation_set("th", pr.D, split, pr.stride, pa.ctx.N // 2))
    fa = upload_problem(g, pa, stride=4)
    fb = g.upload_diagonals(pb_.diags, stride=1, level=pb_.ctx.L)
    levels = [4, 3, 4, 2, 3, 4]
    cts, _ = _encrypt_many(pa, levels, 300)
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    fs = [fa, fb, fa, fb, fa, fb]
    splits = [(2, 2, 4) if f is fa else (2, 2, 2) for f in fs]
    outs = g.lt_eval_batch(ins, fs, algos=["th"] * 6, splits=splits)
    for n in range(6):
        single, _ = g.lt_eval(ins[n], fs[n], "th", splits[n])
        assert_same(outs[n].numpy(), single.numpy(), f"item {n}")
    want = np.stack(olt.lt_th_bsgs(pa.ctx, cts[0], pa.diags, pa.keys, 2, 2, 4, stride=4)[0])
    assert_same(outs[0].numpy(), want, "strided item vs oracle")


def test_batch_autotuner_picks_a_candidate_and_stays_exact():
    """lt_autotune_batch times the candidates as one batch and returns one of
    them; the batch evaluated with it equals the oracle; mixed levels are refused."""
    from paper_2605_17222_gb300 import binding
    pb = make_problem("toy", 0, 64)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    cands = g.candidate_splits("th", pb.level, 64, 3)
    for sp in cands:
        ensure_keys(pb, "th", sp)
    upload_problem(g, pb)
    cts, _ = _encrypt_many(pb, [4, 4, 4, 4], 500)
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    split, ms = g.autotune_batch("th", ins, f, len(cands))
    assert split in cands and ms > 0
    outs = g.lt_eval_batch(ins, [f] * 4, algos=["th"] * 4, splits=[split] * 4)
    want = np.stack(olt.lt_th_bsgs(pb.ctx, cts[2], pb.diags, pb.keys, *split)[0])
    assert_same(outs[2].numpy(), want, "autotuned batch item vs oracle")
    mixed, _ = _encrypt_many(pb, [4, 3], 510)
    with pytest.raises(binding.CkksError) as e:
        g.autotune_batch("th", [g.ct_from_host(np.stack(c)) for c in mixed], f, 2)
    assert e.value.status == 1


def test_recording_one_stream_leaves_another_streams_batch_alone():
    """While one thread records stream S, another thread's batch on stream T,
    forked over T's own lanes, runs at once and is not captured; the graph
    recorded on S replays S's batch only.  (The recording thread itself may not
    queue work on other streams: thread-local capture forbids the allocations.)"""
    import threading

    import torch
    pb = make_problem("toy", 0, 64)
    ensure_keys(pb, "th", (4, 4, 4))
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    cts, _ = _encrypt_many(pb, [4, 3, 4, 3], 700)  # two levels: two groups, so the batch forks
    ins = [g.ct_from_host(np.stack(ct)) for ct in cts]
    args = dict(algos=["th"] * 4, splits=[(4, 4, 4)] * 4)
    want = [o.numpy() for o in g.lt_eval_batch(ins, [f] * 4, **args)]
    S, T = torch.cuda.Stream(), torch.cuda.Stream()
    out_s = [g.ct_empty(c.level - 1) for c in ins]
    out_t = [g.ct_empty(c.level - 1) for c in ins]
    g.lt_eval_batch(ins, [f] * 4, outs=out_s, stream=S, **args)  # first use of each stream's lanes
    g.lt_eval_batch(ins, [f] * 4, outs=out_t, stream=T, **args)
    torch.cuda.synchronize()
    for o in out_s + out_t:
        o.tensor.zero_()
    torch.cuda.synchronize()
    errors = []

    def other_thread():
        try:
            g.lt_eval_batch(ins, [f] * 4, outs=out_t, stream=T, **args)  # runs now
            T.synchronize()
        except Exception as e:  # reported below
            errors.append(e)

    g.graph_begin(S)
    g.lt_eval_batch(ins, [f] * 4, outs=out_s, stream=S, **args)  # recorded
    th = threading.Thread(target=other_thread)
    th.start()
    th.join()
    rec = g.graph_end(S, keep=(ins, out_s, f))
    assert not errors, errors
    for n, (o, w) in enumerate(zip(out_t, want)):
        assert_same(o.numpy(), w, f"stream T item {n}")
    assert not any(np.any(o.numpy()) for o in out_s)  # S's work was recorded, not run
    rec.launch(S)
    S.synchronize()
    for n, (o, w) in enumerate(zip(out_s, want)):
        assert_same(o.numpy(), w, f"replay item {n}")
    rec.close()
