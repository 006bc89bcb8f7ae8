"""Host-side arithmetic of bench.py's rooflines, on CPU: the integer-ALU
fraction with a stand-in for the library, the diagonal kernel's algorithmic
bytes at the headline split summed category by category, the whole-LT
compulsory bytes, and the rule that drops stale ncu traffic."""
import json

import pytest

import bench

LIMB = 8 * 2 ** 16  # one limb at N = 2^16


class FakeBinding:
    """Stands in for the library: fixed probe rates."""

    @staticmethod
    def probe_int_rates(device):
        return 2.0e12, 1.0e12


def test_alu_fraction_is_ideal_time_over_measured_time():
    shares = {"diag_mac": (10.0, 2), "ntt_fwd_rows": (4.0, 4), "automorphism": (1.0, 1), "ks_inner": (0.0, 0)}
    work = {"diag_mac": (2.0e10, 0.0), "ntt_fwd_rows": (0.0, 2.0e9), "automorphism": (0.0, 0.0),
            "ks_inner": (5.0e8, 0.0)}
    out = bench.alu_roofline(FakeBinding, 0, shares, work, "diag_mac", (6.0, 1), (1.2e10, 0.0))
    k = out["kernels"]
    # the dominant class uses its timed-region figures: 1.2e10 MACs at 2e12/s = 6 ms in 6 ms
    assert k["diag_mac"]["frac"] == pytest.approx(1.0)
    assert k["diag_mac"]["macs_per_launch"] == 12_000_000_000 and k["diag_mac"]["ms_per_launch"] == 6.0
    # 2e9 butterflies at 1e12/s = 2 ms of 4 ms over 4 launches
    assert k["ntt_fwd_rows"]["frac"] == pytest.approx(0.5)
    assert k["ntt_fwd_rows"]["butterflies_per_launch"] == 500_000_000
    # no counted work or no launches: not reported
    assert "automorphism" not in k and "ks_inner" not in k
    assert out["peak"] == {"macs_per_s": 2.0e12, "butterflies_per_s": 1.0e12}


def test_alu_fraction_adds_the_two_kinds_of_work():
    """A class doing both (the column pass with basis conversion) adds their times."""
    out = bench.alu_roofline(FakeBinding, 0, {"ntt_fwd_cols": (3.0, 1)}, {"ntt_fwd_cols": (2.0e9, 2.0e9)},
                             "diag_mac", (0.0, 0), (0.0, 0.0))
    assert out["kernels"]["ntt_fwd_cols"]["frac"] == pytest.approx((1e-3 + 2e-3) / 3e-3)


def test_diag_mac_bytes_at_the_headline_split():
    """(1,64,4), level 24, k 4, beta 6, 256 diagonals: the compulsory words K6
    streams -- 256 x 28 diagonal limbs and 63 middle-layer keys of 2 x 6 x 28
    limbs -- 14.86 GB; digits, inputs and partial sums are intermediates."""
    want = (256 * 28 + 63 * 336) * LIMB
    assert round(want / 1e9, 2) == 14.86
    assert bench.algorithmic_bytes("diag_mac", (1, 64, 4), 24, 4, 6, 256, 2 ** 16) == (want, 1)
    # no middle layer (DH as TH(n1, 1, n3)): diagonals only
    assert bench.algorithmic_bytes("diag_mac", (16, 1, 16), 24, 4, 6, 256, 2 ** 16) == (256 * 28 * LIMB, 1)


def test_ks_inner_bytes_are_the_inner_and_outer_keys():
    """(4,8,8): 3 inner-layer and 7 outer-layer keys of 2 x 6 x 28 limbs, over 10 products."""
    assert bench.algorithmic_bytes("ks_inner", (4, 8, 8), 24, 4, 6, 256, 2 ** 16) == (10 * 336 * LIMB, 10)


def test_lt_compulsory_bytes():
    """(4,16,4): 21 distinct keys; diagonals, keys, the input ciphertext and
    the output one level down, 7.51 GB."""
    limbs = 256 * 28 + 21 * 2 * 6 * 28 + 2 * 24 + 2 * 23
    assert bench.lt_compulsory_bytes((4, 16, 4), 24, 4, 6, 256, 2 ** 16) == limbs * LIMB
    assert round(limbs * LIMB / 1e9, 2) == 7.51


def test_stale_traffic_is_dropped(tmp_path, monkeypatch):
    """The committed DRAM traffic counts only while the kernel's sources still
    hash to the digest stored with them."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel v1")
    rec = {"diag_mac": {"dram_bytes_per_launch": 123, "sources": ["k.cu"]}}
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec["diag_mac"]["source_digest"] = bench.source_digest(["k.cu"])
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic("diag_mac") == 123
    (tmp_path / "k.cu").write_text("kernel v2")
    assert bench.ncu_traffic("diag_mac") is None
    assert bench.ncu_traffic("ks_inner") is None
