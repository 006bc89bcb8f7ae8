"""The integer-ALU roofline's two halves, through the C ABI.

  * The per-class work counters (ckks_profile_work): 128-bit
    multiply-accumulates and NTT butterflies of the profiled launches, against
    their closed forms for a forward and an inverse NTT, a Decompose (full and
    partial last digit) and a whole TH-BSGS LT.
  * The register-only rate probe (ckks_probe_int_rates): positive and below
    what the SM count and clock allow; no kernel's counted work runs faster
    than the probe by more than timing noise."""
import numpy as np
import pytest

from paper_2605_17222_gb300 import binding, synth

from gpu_common import TOY_SPLITS, ensure_keys, gpu_context, upload_problem

pytestmark = pytest.mark.gpu

CLASSES = binding.KERNEL_CLASSES


def profiled(fn):
    """Runs fn with every class profiled; returns {class: (macs, butterflies)}
    and {class: (ms, launches)}."""
    import torch
    for c in CLASSES:
        binding.profile_enable(c, True)
    binding.profile_reset()
    try:
        fn()
        torch.cuda.synchronize()
        work = {c: binding.profile_work(c) for c in CLASSES}
        runs = {c: binding.profile_read(c) for c in CLASSES}
    finally:
        for c in CLASSES:
            binding.profile_enable(c, False)
    return work, runs


def test_ntt_butterflies():
    """A forward and an inverse NTT of an extended polynomial: N/2 butterflies
    per stage and limb, log N stages split over the two passes, no MACs."""
    ps = synth.param_set("n16")
    g = binding.Context.from_params(ps)
    level, N = len(ps.q), ps.n
    ext = level + len(ps.p)
    t = binding.to_device(synth.uniform_mod(3, "prof", list(ps.q) + list(ps.p), N))
    logn = N.bit_length() - 1
    work, runs = profiled(lambda: g.ntt(t, level, ext=True, inverse=False))
    assert work["ntt_fwd_cols"][1] + work["ntt_fwd_rows"][1] == ext * (N // 2) * logn
    assert work["ntt_fwd_cols"][1] == ext * (N // 2) * 8 and work["ntt_fwd_cols"][0] == 0
    assert runs["ntt_fwd_cols"][1] == 1 and runs["ntt_fwd_rows"][1] == 1
    work, _ = profiled(lambda: g.ntt(t, level, ext=True, inverse=True))
    assert work["ntt_inv_rows"][1] + work["ntt_inv_cols"][1] == ext * (N // 2) * logn
    assert all(work[c] == (0.0, 0.0) for c in ("diag_mac", "ks_inner", "ntt_fwd_cols", "ntt_fwd_rows"))


@pytest.mark.parametrize("level", [24, 22])
def test_decompose_work(level):
    """Decompose at level l (alpha 4; level 22 has a partial last digit): the
    inverse NTT of l limbs; per digit b of n_b limbs, a forward NTT of the
    ext - n_b other limbs with n_b basis-conversion MACs per word (Eq. 3)."""
    ps = synth.param_set("n16")
    g = binding.Context.from_params(ps)
    N, k, alpha = ps.n, len(ps.p), 4
    ext = level + k
    logn = N.bit_length() - 1
    digits = [min(alpha, level - first) for first in range(0, level, alpha)]
    c = binding.to_device(synth.uniform_mod(4, "prof", list(ps.q[:level]), N))
    work, _ = profiled(lambda: g.decompose(c, level))
    fwd_limbs = sum(ext - n for n in digits)
    assert work["ntt_inv_rows"][1] + work["ntt_inv_cols"][1] == level * (N // 2) * logn
    assert work["ntt_fwd_cols"][1] + work["ntt_fwd_rows"][1] == fwd_limbs * (N // 2) * logn
    assert work["ntt_fwd_cols"][0] == sum(n * (ext - n) for n in digits) * N


def test_lt_diag_mac_work():
    """One TH-BSGS (4,4,4) LT on the toy set (N = 2^12, level 4, k 1, alpha 1,
    beta 4, 64 diagonals): the diagonal kernel counts 2 n'3 products per step
    and position and 2 beta middle-layer products per step with j > 0, over
    every limb of the extended basis; the key inner products count 2 beta per
    output word."""
    from oracle.workload import make_problem
    pb = make_problem("toy", 0, 64)
    split = TOY_SPLITS["th"]
    ensure_keys(pb, "th", split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    ct = g.ct_upload(np.stack(pb.ct))
    n1, n2, n3 = split
    level, N, k, beta = pb.ctx.L, pb.ctx.N, pb.ctx.k, 4
    ext = level + k
    work, runs = profiled(lambda: g.lt_eval(ct, f, "th", split))
    want = N * ext * (2 * n1 * n2 * n3 + 2 * beta * (n1 * n2 - n1))
    assert work["diag_mac"] == (float(want), 0.0)
    assert runs["diag_mac"][1] == 1
    macs_ks = work["ks_inner"][0]
    assert macs_ks > 0 and macs_ks % (2 * beta * ext * N) == 0


def test_probe_rates_are_physical():
    """The probe's rates are positive and below a ceiling no SM can pass: 128
    integer multiply lanes per SM per cycle at 2.2 GHz, with 8 multiplies per
    128-bit MAC (four 32 x 32 partial products, low and high halves) and at
    least 9 per butterfly (the Shoup quotient and two 64-bit low products).
    A real LT's kernels then stay within 1.1 of the probe."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    macs, bfly = binding.probe_int_rates(0)
    ceiling = sms * 128 * 2.2e9
    assert 1e10 < macs < ceiling / 8
    assert 1e10 < bfly < ceiling / 9
    from oracle.workload import make_problem
    pb = make_problem("toy", 0, 64)
    split = TOY_SPLITS["th"]
    ensure_keys(pb, "th", split)
    g = gpu_context("toy")
    f = upload_problem(g, pb)
    ct = g.ct_upload(np.stack(pb.ct))
    work, runs = profiled(lambda: [g.lt_eval(ct, f, "th", split) for _ in range(3)])
    for c in CLASSES:
        m, b = work[c]
        ms, n = runs[c]
        if n and (m or b):
            assert (m / macs + b / bfly) / (ms / 1e3) < 1.1, c
