"""ckks_moddown_noalloc: ModDown for host programs that cannot let the
library allocate GPU memory while it runs -- an application that owns every
byte of the device through its own allocator or budget, or a latency-bound
path where a cudaMalloc (and the device synchronisation it may imply) is not
acceptable.  Checked through the C ABI against ckks_moddown, bit for bit, on
two calls in a row (the fixed scratch keeps the previous call's contents), and
checked to allocate nothing: the context's device-memory count, torch's
caching allocator and the device's stream-ordered pool (which every other
library call draws its scratch from) all stay where they were.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_17222_gb300 import binding, synth

pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


class _DefaultPool:
    """The device's default stream-ordered memory pool through the driver API
    (the pool the library's cudaMallocAsync scratch comes from); None when the
    driver library cannot be opened."""

    def __init__(self, device: int):
        self.cu = None
        try:
            cu = ctypes.CDLL("libcuda.so.1")
        except OSError:
            return
        dev, pool = ctypes.c_int(), ctypes.c_void_p()
        if cu.cuDeviceGet(ctypes.byref(dev), device) != 0:
            return
        if cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) != 0:
            return
        self.cu, self.pool = cu, pool

    def get(self, attr: int) -> int:
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self) -> None:
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_moddown_noalloc_matches_moddown_on_two_calls_and_allocates_nothing():
    import torch
    ps = synth.param_set("n16")
    g = binding.Context.from_params(ps)
    pool = _DefaultPool(torch.cuda.current_device())
    for call, level in enumerate([ps.L, ps.L - 5]):
        basis = list(ps.q[:level]) + list(ps.p)
        x = binding.to_device(synth.uniform_mod(100 + call, "noalloc", basis, ps.n))
        want = g.moddown(x, level)  # the existing entry point (also sets up this level's constants)
        got = torch.empty((level, ps.n), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        ctx_bytes, reserved = g.bytes_in_use(), torch.cuda.memory_reserved()
        if pool.cu:
            pool.reset_high()
            used = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
        g.moddown_noalloc(x, level, got)
        torch.cuda.synchronize()
        assert np.array_equal(binding.to_host(got), binding.to_host(want)), f"call {call}"
        assert g.bytes_in_use() == ctx_bytes, f"call {call}: the context's device memory changed"
        assert torch.cuda.memory_reserved() == reserved, f"call {call}: torch's allocator grew"
        if pool.cu:
            assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) == used, f"call {call}: the stream-ordered pool was used"


def test_moddown_noalloc_rejects_unprepared_level_and_bad_arguments():
    import torch
    ps = synth.param_set("toy")
    g = binding.Context.from_params(ps)
    x = torch.zeros((ps.L + ps.k, ps.n), dtype=torch.int64, device="cuda")
    out = torch.empty((ps.L, ps.n), dtype=torch.int64, device="cuda")
    with pytest.raises(binding.CkksError, match="not set up") as e:   # constants not set up yet
        g.moddown_noalloc(x, ps.L, out)
    assert e.value.status == 1
    with pytest.raises(binding.CkksError) as e:                      # bad level
        g.moddown_noalloc(x, ps.L + 7, out)
    assert e.value.status == 1
    with pytest.raises(binding.CkksError) as e:                      # in place
        g.moddown_noalloc(x, ps.L, x)
    assert e.value.status == 1
