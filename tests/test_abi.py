"""The C-ABI library builds, loads and exports every function include/ckks_lt.h
declares (no compute calls: CPU only)."""
import ctypes
import subprocess

from paper_2605_17222_gb300 import binding


def test_header_declares_the_boundary():
    names = binding.declared_functions()
    for n in ["ckks_ctx_create", "ckks_upload_rotation_key", "ckks_upload_diagonals", "ckks_ct_upload",
              "ckks_ct_wrap_device", "ckks_ct_download", "lt_eval", "lt_eval_batch", "ckks_free_ct",
              "ckks_free_diags", "ckks_last_error", "ckks_device_bytes_in_use"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    missing = [n for n in binding.declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_exported_symbols_are_c_linkage():
    path = binding.lib()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in binding.declared_functions():
        assert n in syms, n


def test_errors_without_device_are_reported():
    """A null context is rejected with CKKS_EINVAL and a message (no GPU needed)."""
    L = binding.lib()
    st = L.ckks_ctx_create(None, 12, None, 0, None, 0, 1, 0)
    assert st == 1
    assert b"null" in L.ckks_last_error()


def test_profile_calls_without_device():
    """The live-timing and work counters are host bookkeeping: every class reads
    zero after a reset, enabling launches nothing, and an unknown class or a
    null output is rejected with CKKS_EINVAL."""
    binding.profile_reset()
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, True)
        assert binding.profile_read(c) == (0.0, 0)
        assert binding.profile_work(c) == (0.0, 0.0)
        binding.profile_enable(c, False)
    for call in (lambda: binding.profile_read("no_such_kernel"), lambda: binding.profile_work("no_such_kernel"),
                 lambda: binding.profile_enable("no_such_kernel")):
        try:
            call()
        except binding.CkksError as e:
            assert e.status == 1
        else:
            raise AssertionError("unknown kernel class accepted")
    L = binding.lib()
    assert L.ckks_profile_work(b"diag_mac", None, None) == 1
    assert L.ckks_probe_int_rates(0, None, None) == 1
