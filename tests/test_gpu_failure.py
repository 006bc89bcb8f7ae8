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


def test_diag_mac_waits_run_out_in_the_production_kernel():
    """The staged diagonal kernel itself: with its test hook, step 1 is never
    issued and the step loop's waits give up after 20 us.  Every CTA stops,
    drains its copies in flight, the host reads CKKS_ETIMEOUT, the call comes
    back within milliseconds, and with the hook reset the same context
    computes the LT bit-exactly."""
    import time

    import torch

    from oracle.workload import make_problem

    from gpu_common import assert_same, ensure_keys, gpu_context, oracle_lt, upload_problem

    pb = make_problem("toy", 0, 64)
    split = (4, 4, 4)
    ensure_keys(pb, "th", split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    ct = g.ct_from_host(np.stack(pb.ct))
    g.lt_eval(ct, f, "th", split)  # warm: per-level tables, kernel attributes
    g.device_status()
    g.debug_diag_mac_waits(20_000, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.lt_eval(ct, f, "th", split)
    with pytest.raises(binding.CkksError) as e:
        g.device_status()
    elapsed = time.perf_counter() - t0
    assert e.value.status == CKKS_ETIMEOUT
    assert elapsed < 0.25, f"the failing LT took {elapsed:.3f} s (a wait or the drain used the 1 s default)"
    g.debug_diag_mac_waits(0, 0xFFFFFFFF)
    g.device_status()  # the flag was cleared
    out, _ = g.lt_eval(ct, f, "th", split)
    assert_same(out.numpy(), oracle_lt(pb, "th", split), "after the timeout")
    g.device_status()
