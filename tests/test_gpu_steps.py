"""Step-by-step parity of the CUDA kernels with the CPU oracle, bit for bit,
through the C ABI: NTT/INTT, automorphism, Decompose, switching-key inner
product, ModDown, merged ModDown+rescale, rescale.  Sizes span several tiles
and every limb of the extended basis; edge inputs (0, q-1), the minimum level
and partial last digits are included."""
import numpy as np
import pytest

from oracle.ckks import Ctx
from paper_2605_17222_gb300 import binding, synth

from gpu_common import assert_same

pytestmark = pytest.mark.gpu

SETS = ["toy", "setA", "n14", "n15", "n16"]  # every NTT shape, N = 2^12 .. 2^16
_CACHE = {}


def env(name):
    if name not in _CACHE:
        ps = synth.param_set(name)
        _CACHE[name] = (Ctx(ps), binding.Context.from_params(ps))
    return _CACHE[name]


def rand(ctx, basis, seed, kind="uniform"):
    a = synth.uniform_mod(seed, "steps", basis, ctx.N)
    if kind == "zero":
        a[:] = 0
    elif kind == "max":
        a[:] = np.array(basis, dtype=np.uint64)[:, None] - np.uint64(1)
    return a


def dev(a):
    return binding.to_device(a)


def host(t):
    import torch
    torch.cuda.synchronize()
    return binding.to_host(t)


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("kind", ["uniform", "zero", "max"])
def test_ntt_forward_inverse(name, kind):
    octx, g = env(name)
    for level in sorted({octx.L, 2, max(2, octx.L - 3)}):
        B = octx.basis(level, True)
        a = rand(octx, B, 1 + level, kind)
        t = dev(a)
        g.ntt(t, level, ext=True, inverse=False)
        assert_same(host(t), octx.ntt(a, B), f"ntt {name} level {level}")
        g.ntt(t, level, ext=True, inverse=True)
        assert_same(host(t), a, f"intt {name} level {level}")


@pytest.mark.parametrize("name", SETS)
def test_automorphism(name):
    octx, g = env(name)
    B = octx.basis(3, True)
    a = rand(octx, B, 7)
    for r in [1, 5, -1, octx.N // 4 + 3]:
        assert_same(host(g.automorphism(dev(a), r)), octx.auto_ntt(a, r), f"auto {r}")


@pytest.mark.parametrize("name", SETS)
def test_decompose(name):
    octx, g = env(name)
    levels = {octx.L, 2}
    if octx.alpha > 1:
        levels.add(octx.L - octx.alpha // 2)  # partial last digit
    for level in sorted(levels):
        Q = octx.basis(level, False)
        c = rand(octx, Q, 11 + level)
        for rot in [0, 3]:
            want = np.stack(octx.decompose(octx.auto_ntt(c, rot) if rot else c, level))
            got = host(g.decompose(dev(c), level, rot=rot))
            assert_same(got, want, f"decompose {name} level {level} rot {rot}")


@pytest.fixture(scope="module")
def keyed():
    """toy and n15 contexts with two rotation keys (oracle keygen)."""
    out = {}
    for name in ["toy", "n15"]:
        octx, g = env(name)
        s = octx.secret(5)
        keys = {r: octx.keygen_rotation(s, r, 5) for r in (3, 8)}
        for r, k in keys.items():
            g.upload_rotation_key(r, k)
        out[name] = keys
    return out


@pytest.mark.parametrize("name", ["toy", "n15"])
def test_ks_inner_hoisted(name, keyed):
    """out = phi_r(P x0 + <d, phi_{-r}(swk_r)>), out1 = phi_r(<d, phi_{-r}(swk_r)>) (Alg. 2 lines 4-5)."""
    octx, g = env(name)
    for level in sorted({octx.L, 3}):
        Q = octx.basis(level, False)
        ext = octx.basis(level, True)
        c0 = rand(octx, Q, 21)
        d = octx.decompose(rand(octx, Q, 22), level)
        for r in (3, 8):
            kt = octx.hoisted_key(octx.key_at_level(keyed[name][r], level), r)
            x0, x1 = octx.inner(d, kt, level)
            want0 = octx.auto_ntt(octx.add(octx.lift(c0, level), x0, ext), r)
            want1 = octx.auto_ntt(x1, r)
            o0, o1 = g.ks_inner(level, dev(np.stack(d)), r, r, x0=dev(c0), lift_x0=True)
            assert_same(host(o0), want0, f"ks0 {name} {level} {r}")
            assert_same(host(o1), want1, f"ks1 {name} {level} {r}")
            # accumulate form with an extended x0 (Alg. 2 lines 17-18)
            u0 = rand(octx, ext, 23)
            base0, base1 = rand(octx, ext, 24), rand(octx, ext, 25)
            t0, t1 = dev(base0), dev(base1)
            g.ks_inner(level, dev(np.stack(d)), r, r, x0=dev(u0), out0=t0, out1=t1, accumulate=True)
            assert_same(host(t0), octx.add(base0, octx.auto_ntt(octx.add(u0, x0, ext), r), ext), "acc0")
            assert_same(host(t1), octx.add(base1, want1, ext), "acc1")


@pytest.mark.parametrize("name", SETS)
def test_moddown_family(name):
    octx, g = env(name)
    for level in sorted({octx.L, 2}):
        ext = octx.basis(level, True)
        Q = octx.basis(level, False)
        x = rand(octx, ext, 31 + level)
        assert_same(host(g.moddown(dev(x), level)), octx.moddown(x, level), f"moddown {name} {level}")
        assert_same(host(g.moddown_rescale(dev(x), level)), octx.moddown_rescale(x, level), f"mdr {name} {level}")
        xq = rand(octx, Q, 41 + level)
        assert_same(host(g.rescale(dev(xq), level)), octx.rescale(xq, level), f"rescale {name} {level}")


def test_errors_are_status_codes():
    octx, g = env("toy")
    import torch
    t = torch.zeros((5, octx.N), dtype=torch.int64, device="cuda")
    with pytest.raises(binding.CkksError) as e:
        g.moddown(t, 99)
    assert e.value.status == 1
    with pytest.raises(binding.CkksError) as e:
        g.ks_inner(4, torch.zeros((4, 5, octx.N), dtype=torch.int64, device="cuda"), 77, 77)
    assert e.value.status == 3  # CKKS_ENOKEY
