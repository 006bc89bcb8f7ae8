"""The split-selection cost model (lt_model_estimate) against measurement, on
CPU: the model is restated here term by term -- K6 at the slower of its DRAM
bytes and its multiply-accumulates, the key-switch inner products at their
bytes, the Decompose / ModDown limb transforms at their butterflies -- and
checked against the DRAM bytes ncu measured per LT and the LT times in
profiles/lt_cost_model_n16.json (N = 2^16, level 24, k = 4, beta 6, 256
diagonals).  tests/test_gpu_lt.py checks that the library computes the same
numbers."""
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BW, MAC4, MAC8, NTT, FIXED, NTT_LIMBS = 6.2e12, 9.5e11, 7.0e11, 5.8e11, 1e-4, 2.75


def model(level, D, n1, n2, n3, log_n=16, K=4, alpha=4):
    """(DRAM bytes, seconds) of one TH-shaped LT (n'1, n'2, n'3)."""
    N = 1 << log_n
    limb, ext, beta, L = 8.0 * N, level + K, -(-level // alpha), level
    mid = n2 > 1
    k3 = 1
    while k3 < n3 and k3 < 8:
        k3 *= 2
    blocks = -(-n3 // k3)
    k6_bytes = limb * (D * ext + ((n2 - 1) * 2 * beta * ext + n1 * beta * ext if mid else 0)
                       + 2 * (n1 - 1) * ext + 2 * L + 2 * n3 * ext)
    k6_macs = N * ext * (2 * D + (2 * beta * (n1 * n2 - n1) * blocks if mid else 0))
    t_k6 = max(k6_bytes / BW, k6_macs / (MAC8 if k3 >= 8 else MAC4))
    k4_bytes = limb * ((n1 - 1) * (3 * beta * ext + L + 2 * ext) + (n3 - 1) * (3 * beta * ext + ext) + 4 * ext)
    dec = 1 + (n1 - 1 if mid else 0) + (n3 - 1)
    mdp = (n1 - 1 if mid else 0) + (n3 - 1)
    ntt_limbs = dec * (L + beta * (ext - alpha)) + mdp * (K + L) + 2 * (K + L)
    seconds = t_k6 + k4_bytes / BW + ntt_limbs * (N / 2) * log_n / NTT + FIXED
    return k6_bytes + k4_bytes + limb * NTT_LIMBS * ntt_limbs, seconds


@pytest.fixture(scope="module")
def measured():
    with open(os.path.join(ROOT, "profiles", "lt_cost_model_n16.json")) as f:
        return json.load(f)


def split_of(key):
    return tuple(int(x) for x in key.split(","))


def test_dram_bytes_within_two_percent(measured):
    for key, m in measured["dram_per_lt_bytes"].items():
        b, _ = model(24, 256, *split_of(key))
        assert abs(b - m["total"]) / m["total"] < 0.02, (key, b, m["total"])


def test_lt_time_within_three_percent_and_ranking(measured):
    for key, ms in measured["lt_ms"].items():
        _, s = model(24, 256, *split_of(key))
        assert abs(s * 1e3 - ms) / ms < 0.03, (key, s * 1e3, ms)
    # the model orders the measured splits as the measurements do, fastest first
    by_meas = sorted(measured["lt_ms"], key=measured["lt_ms"].get)
    by_model = sorted(measured["lt_ms"], key=lambda k: model(24, 256, *split_of(k))[1])
    assert by_model[:3] == by_meas[:3]


def test_model_terms_follow_the_schedule():
    """Structural checks that a transposed or dropped term would break: no
    middle layer (n'2 = 1) means no middle keys and no baby-index digits, and
    halving n'3 at a fixed D doubles the middle layer's steps."""
    b_dh, _ = model(24, 256, 16, 1, 16)
    limb, ext = 8.0 * 2 ** 16, 28
    k6_no_mid = limb * (256 * ext + 2 * 15 * ext + 2 * 24 + 2 * 16 * ext)
    assert b_dh > k6_no_mid
    _, s4 = model(24, 256, 1, 64, 4)
    _, s8 = model(24, 256, 1, 32, 8)
    assert math.isfinite(s4) and math.isfinite(s8)
