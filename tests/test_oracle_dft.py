"""The oracle's factored slot DFT (the CoeffToSlot / SlotToCoeff stages) pinned
against closed forms: the matrix U[j][k] = xi_j^k itself, the oracle's own
FFT-based decoder, U^H U = n I, and the stage windows' offsets; and the
homomorphic chain of LTs against the dense FP64 product.  CPU only."""
import numpy as np
import pytest

from oracle import dft
from oracle import lt as olt
from oracle.ckks import Ctx
from oracle.workload import make_chain_problem
from paper_2605_17222_gb300 import synth


def test_decoder_is_u_applied_to_coefficient_pairs():
    """The oracle decodes slot j as m(zeta^(5^j)) through an FFT; the same
    slots are U (m_k + i m_{k+n})_k, with U from its closed form."""
    ctx = Ctx(synth.param_set("tiny"))
    n = ctx.N // 2
    m = np.random.default_rng(1).standard_normal(ctx.N)
    assert np.allclose(ctx.decode_coeffs(m, 1.0), dft.u_matrix(n) @ (m[:n] + 1j * m[n:]), atol=1e-10)


@pytest.mark.parametrize("n", [2, 8, 16, 64, 256])
def test_stages_factor_u(n):
    """S_m ... S_1 = U R (R the bit reversal), and each S_t^-1 inverts S_t."""
    m = int(np.log2(n))
    P = np.eye(n, dtype=np.complex128)
    for t in range(1, m + 1):
        S = dft.to_dense(dft.stage(n, t), n)
        assert len(dft.stage(n, t)) == (3 if 2 ** (t - 1) != n // 2 else 2)
        assert np.allclose(dft.to_dense(dft.stage(n, t, inverse=True), n) @ S, np.eye(n))
        P = S @ P
    R = np.eye(n)[dft.bitrev(n)]
    assert np.allclose(P, dft.u_matrix(n) @ R)


def test_u_is_unitary_up_to_n():
    n = 64
    U = dft.u_matrix(n)
    assert np.allclose(U.conj().T @ U, n * np.eye(n))


@pytest.mark.parametrize("n,radices", [(64, [3, 3]), (256, [3, 3, 2]), (256, [2, 2, 2, 2]), (2048, [4, 4, 3])])
def test_windows_shapes_and_products(n, radices):
    """Group of r stages starting at S_t: stride 2^(t-1), window
    -(2^r - 1) 2^(t-1) .. +(2^r - 1) 2^(t-1) (2^(r+1) - 1 diagonals), except the
    group ending at S_m, whose offsets cover every multiple (2^r diagonals
    from 0).  The chain equals U z[R] (StC) and (U^H z / n)[R] (CtS)."""
    m = int(np.log2(n))
    z = synth.slots(4, "dft", n)
    stc = dft.slot_to_coeff(n, radices)
    t = 1
    for r, w in zip(radices, stc):
        h = 2 ** (t - 1)
        if t + r - 1 == m:
            assert (w.offset0, w.stride, w.D) == (0, h, 2 ** r)
        else:
            assert (w.offset0, w.stride, w.D) == (-(2 ** r - 1) * h, h, 2 ** (r + 1) - 1)
        t += r
    R = dft.bitrev(n)
    if n <= 256:
        U = dft.u_matrix(n)
        assert np.allclose(dft.apply_windows(z, stc), U @ z[R])
        cts = dft.coeff_to_slot(n, radices[::-1])
        assert np.allclose(dft.apply_windows(z, cts), (U.conj().T @ z / n)[R])
    # CtS then StC is the identity (any n)
    back = dft.apply_windows(dft.apply_windows(z, dft.coeff_to_slot(n, radices[::-1])), stc)
    assert np.allclose(back, z)


def test_padding_keeps_the_matrix():
    n = 256
    a = dft.slot_to_coeff(n, [3, 3, 2])
    b = dft.slot_to_coeff(n, [3, 3, 2], pad=True)
    assert [w.D for w in b] == [16, 16, 4]
    z = synth.slots(5, "pad", n)
    assert np.allclose(dft.apply_windows(z, a), dft.apply_windows(z, b))


def test_homomorphic_slot_to_coeff_chain():
    """N = 2^12 (2048 slots), three LTs of 31, 31 and 8 diagonals (radices
    4, 4, 3; the first two padded to 32) from level 4 to level 1, TH-BSGS:
    decrypts to U z[R]."""
    pb = make_chain_problem("toy", 2, "stc", [4, 4, 3], [(2, 2, 8), (4, 4, 2), (2, 2, 2)])
    assert [w.D for w in pb.windows] == [32, 32, 8]
    out = olt.lt_chain(pb.ctx, pb.ct, pb.stages(), pb.keys)
    assert out[0].shape[0] == 1
    y = pb.decrypt(out)
    assert np.max(np.abs(y - pb.expected())) < 1e-5


def test_homomorphic_coeff_to_slot_chain():
    """The inverse direction (outputs shrink by about 1/sqrt(n)): decrypts to (U^H z / n)[R]."""
    pb = make_chain_problem("toy", 3, "cts", [3, 4, 4], [(2, 2, 2), (4, 4, 2), (2, 2, 8)])
    out = olt.lt_chain(pb.ctx, pb.ct, pb.stages(), pb.keys)
    y = pb.decrypt(out)
    assert np.max(np.abs(y - pb.expected())) < 1e-6
