"""ckks_moddown_noalloc: ModDown for callers that cannot allocate device
memory while they run (graph capture, external allocators or budgets).
Checked through the C ABI against ckks_moddown, bit for bit, on two calls in
a row (the fixed scratch keeps the previous call's contents)."""
import ctypes

import numpy as np
import pytest

from paper_2605_17222_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _noalloc():
    L = binding.lib()
    fn = L.ckks_moddown_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_moddown_noalloc_matches_moddown_on_two_calls():
    import torch
    ps = synth.param_set("n16")
    g = binding.Context.from_params(ps)
    fn = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    for call, level in enumerate([ps.L, ps.L - 5]):
        basis = list(ps.q[:level]) + list(ps.p)
        x = binding.to_device(synth.uniform_mod(100 + call, "noalloc", basis, ps.n))
        want = g.moddown(x, level)  # the existing entry point (also sets up this level's constants)
        got = torch.empty((level, ps.n), dtype=torch.int64, device="cuda")
        st = fn(g.h, level, x.data_ptr(), got.data_ptr(), stream)
        assert st == 0, binding.lib().ckks_last_error().decode()
        torch.cuda.synchronize()
        assert np.array_equal(binding.to_host(got), binding.to_host(want)), f"call {call}"


def test_moddown_noalloc_rejects_unprepared_level_and_bad_arguments():
    import torch
    ps = synth.param_set("toy")
    g = binding.Context.from_params(ps)
    fn = _noalloc()
    x = torch.zeros((ps.L + ps.k, ps.n), dtype=torch.int64, device="cuda")
    out = torch.empty((ps.L, ps.n), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(g.h, ps.L, x.data_ptr(), out.data_ptr(), stream) == 1          # constants not set up yet
    assert b"not set up" in binding.lib().ckks_last_error()
    assert fn(g.h, ps.L + 7, x.data_ptr(), out.data_ptr(), stream) == 1      # bad level
    assert fn(g.h, ps.L, x.data_ptr(), x.data_ptr(), stream) == 1            # in place
