"""The paper's off-chip memory model (Sec. IV, memory-requirement table) pinned
against the totals its resource table prints for Set-A, B and C at the knobs
of its parameter table (tests/golden/tmem_offchip.json), plus properties the
formulas must have.  CPU only."""
import json
import os

import pytest

from paper_2605_17222_gb300 import memory_model as mm

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tmem_offchip.json")))


def shape_knobs(g):
    s = mm.Shape(g["N"], g["Lp1"], g["alpha"], g["beta"], g["n"], tuple(g["split"]))
    m1, l1 = g["m1_l1"]
    m2, l2 = g["m2_l2"]
    m4, m3, l3 = g["m4_m3_l3"]
    m5, l4 = g["m5_l4"]
    m6, l5 = g["m6_l5"]
    return s, mm.Knobs(m1, l1, m2, l2, m3, m4, l3, m5, l4, m6, l5)


@pytest.mark.parametrize("name", list(GOLDEN["sets"]))
def test_reproduces_printed_offchip_totals(name):
    """Within 0.5 % (the model gives 2.846 / 107.81 / 901.9 for 2.84 / 107.91 / 903.47)."""
    g = GOLDEN["sets"][name]
    s, m = shape_knobs(g)
    got = mm.paper_units(mm.offchip_bytes(s, m, GOLDEN["word_bits"]))
    assert abs(got - g["offchip_gb"]) <= 0.005 * g["offchip_gb"], (name, got)
    # the module's own table holds the same figures
    ps, pm, pgb = mm.PAPER_SETS[name]
    assert (ps, pm, pgb) == (s, m, g["offchip_gb"])


@pytest.mark.parametrize("name", list(GOLDEN["sets"]))
def test_structure_of_the_terms(name):
    """The LT matrix is read exactly once (n (L+1+alpha) limbs, phase 4 only);
    switching keys are read once per key (n'1 + n'2 + n'3 - 3 keys of
    2 beta (L+1+alpha) limbs); the limb knobs l1..l5 change no off-chip term."""
    s, m = shape_knobs(GOLDEN["sets"][name])
    ph = mm.offchip_limbs(s, m)
    n1, n2, n3 = s.split
    assert sum(p["matrix"] for p in ph) == s.n * s.ext == ph[3]["matrix"]
    assert sum(p["swk"] for p in ph) == (n1 + n2 + n3 - 3) * 2 * s.beta * s.ext
    wide = mm.Knobs(m.m1, m.l1 + 3, m.m2, m.l2 + 3, m.m3, m.m4, m.l3 + 3, m.m5, m.l4 + 3, m.m6, m.l5 + 3)
    assert mm.offchip_bytes(s, wide) == mm.offchip_bytes(s, m)


def test_more_reuse_never_adds_traffic():
    """Raising m2, m3, m5 or m6 (more polynomials per pass) never increases off-chip access."""
    s, m = shape_knobs(GOLDEN["sets"]["Set-B"])
    base = mm.offchip_bytes(s, m)
    for field in ("m2", "m3", "m5", "m6"):
        bigger = mm.Knobs(**{**m.__dict__, field: getattr(m, field) * 2})
        assert mm.offchip_bytes(s, bigger) <= base
