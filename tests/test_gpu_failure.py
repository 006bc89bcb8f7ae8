"""Failure detection without a GPU fault: a device wait that nothing
completes gives up after its limit, the host reads CKKS_ETIMEOUT, and the
context keeps working."""
import numpy as np
import pytest

from paper_2605_17222_gb300 import binding, synth

pytestmark = pytest.mark.gpu

CKKS_ETIMEOUT = 5


def test_bounded_wait_reports_timeout_and_context_survives():
    ps = synth.param_set("toy")
    g = binding.Context.from_params(ps)
    g.device_status()  # clean
    g.selftest_bounded_wait(100)
    with pytest.raises(binding.CkksError) as e:
        g.device_status()
    assert e.value.status == CKKS_ETIMEOUT
    g.device_status()  # the flag was cleared
    # the context still computes
    import torch
    a = synth.uniform_mod(1, "fail", list(ps.q) + list(ps.p), ps.n)
    t = binding.to_device(a)
    g.ntt(t, ps.L, ext=True, inverse=False)
    g.ntt(t, ps.L, ext=True, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(binding.to_host(t), a)
