"""Shared fixtures of the GPU parity tests: oracle-generated problems and the
library context they are uploaded to."""
import numpy as np

from oracle import lt as olt
from oracle.workload import add_keys, make_problem
from paper_2605_17222_gb300 import binding, synth

TOY_SPLITS = {"diag": None, "bsgs": (8, 8), "dh": (8, 8), "th": (4, 4, 4)}


def gpu_context(param_name: str):
    return binding.Context.from_params(synth.param_set(param_name))


def upload_keys(gctx, keys):
    for r, key in keys.items():
        if not gctx.has_key(r):
            gctx.upload_rotation_key(r, key)


def upload_problem(gctx, pb, stride=1):
    upload_keys(gctx, pb.keys)
    return gctx.upload_diagonals(pb.diags, stride=stride, level=pb.ctx.L, offset0=pb.offset0)


def upload_chain(gctx, cp):
    """A ChainProblem's keys and one Diagonals per stage window."""
    upload_keys(gctx, cp.keys)
    return [gctx.upload_diagonals(d, stride=w.stride, level=cp.ctx.L, offset0=w.offset0)
            for d, w in zip(cp.diags, cp.windows)]


def oracle_lt(pb, algo, split):
    ct, _ = olt.run(pb.ctx, algo, pb.ct, pb.diags, pb.keys, split, pb.stride, pb.offset0)
    return np.stack(ct)


def ensure_keys(pb, algo, split):
    add_keys(pb, olt.rotation_set(algo, pb.D, split, pb.stride, pb.ctx.N // 2, pb.offset0))


def assert_same(got: np.ndarray, want: np.ndarray, what: str = ""):
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError(f"{what}: {len(bad)} of {got.size} residues differ, first at {tuple(bad[0])}: "
                             f"{int(got[tuple(bad[0])])} != {int(want[tuple(bad[0])])}")
