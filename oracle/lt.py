"""CPU oracle, linear-transformation layer: the four HE-LT algorithms.

TEST INFRASTRUCTURE ONLY (see oracle/ckks.py).

  * diagonal method ............. Sec. II-B, Table "complexity comparisons" row 1
  * BSGS ......................... Eq. (5)
  * DH-BSGS ...................... Algorithm 1
  * TH-BSGS ...................... Algorithm 2, Eq. (6)

Inputs: a ciphertext (c0, c1) at level `level` (NTT domain, Q limbs), the
encoded diagonals f_t as a top-level array [D][L + k][N] (all Q limbs then
all P limbs, NTT domain), and standard rotation keys {r: [beta_max][2][L+k][N]}.
Offsets are o_t = offset0 + stride * t (mod N/2).  The common base offset0
joins the outermost rotation layer of each algorithm: with g_t = Rot(f_t,
-offset0),  sum_t f_t . Rot(z, offset0 + stride t) = Rot(sum_t g_t . Rot(z,
stride t), offset0), so the giant (BSGS, DH-BSGS) or outer (TH-BSGS) rotation
amounts become offset0 + stride * n1 (n2) * index -- the first one included --
and the diagonal method ends with one rotation by offset0.  An outer amount
that is 0 mod N/2 needs no key: its partial sum is added as it is.  With
offset0 = 0 every algorithm is exactly the paper's.

Readings (where the paper is silent or inconsistent):
  * Sums printed with upper limit n'1n'2 (Alg. 2 lines 12, 14) and n
    (diagonal method) run to n'1n'2 - 1 and n - 1.
  * Alg. 1 loops i and j from 0; the i = 0 and j = 0 iterations are the
    identity (no rotation, no key, no ModDown/Decompose), as the counts in the
    complexity table (n2 Decompose, n2+1 ModDown, n1+n2-2 keys) require.
  * f^_{x} = phi_{-x}(f) is the automorphism applied to the encoded
    polynomial (exact), not a re-encoding of the rotated slots.
  * BSGS multiplies over Q only (the complexity table's 2n(L+1) term) and ends
    with the plain rescale of Eq. (1); the hoisted algorithms end with the
    merged ModDown + rescale.
"""
from __future__ import annotations

import numpy as np

from .ckks import Ctx, Ops


class _Diags:
    def __init__(self, ctx: Ctx, diags: np.ndarray, level: int, ext: bool):
        self.ctx = ctx
        rows = ctx.ext_rows(level) if ext else list(range(level))
        self.f = diags[:, rows]
        self.basis = ctx.basis(level, ext)

    def hat(self, idx: int, x: int) -> np.ndarray:
        """f^_idx = phi_{-x}(f_idx)."""
        if x == 0:
            return self.f[idx]
        return self.ctx.auto_ntt(self.f[idx], -x)


def _key(ctx: Ctx, keys: dict, r: int, level: int, ops: Ops) -> np.ndarray:
    r %= ctx.N // 2
    if r not in keys:
        raise KeyError(f"missing rotation key {r}")
    ops.keys.add(r)
    return ctx.key_at_level(keys[r], level)


def _outer(ctx: Ctx, x: int) -> int:
    """An outer/giant rotation amount reduced mod N/2 (0 = no rotation)."""
    return x % (ctx.N // 2)


def _rotate_ext(ctx: Ctx, u0, u1, r: int, keys: dict, level: int, ops: Ops):
    """Rotation of an extended-basis pair by r, the hoisted way (Alg. 2 lines
    15-18): ModDown(u1), Decompose, inner product with the hoisted key, then
    phi_r(u0 + x0), phi_r(x1)."""
    ext = ctx.basis(level, True)
    dd = ctx.decompose(ctx.moddown(u1, level, ops), level, ops)
    kt = ctx.hoisted_key(_key(ctx, keys, r, level, ops), r)
    x0, x1 = ctx.inner(dd, kt, level, ops)
    return ctx.auto_ntt(ctx.add(u0, x0, ext), r), ctx.auto_ntt(x1, r)


def lt_diag(ctx: Ctx, ct, diags: np.ndarray, keys: dict, stride: int = 1, ops: Ops | None = None,
            offset0: int = 0):
    """Diagonal method in hoisted form (complexity table row 1: one Decompose,
    two ModDowns, n-1 keys):  C = sum_t phi_t(ct) f_t with every rotation
    sharing Decompose(c1) and ModDown delayed to the accumulated sum.  A
    nonzero offset0 adds one final rotation of the sum (one more key, one more
    Decompose and ModDown)."""
    ops = ops if ops is not None else Ops()
    c0, c1 = ct
    level = c0.shape[0]
    ext = ctx.basis(level, True)
    D = diags.shape[0]
    F = _Diags(ctx, diags, level, True)
    b0 = _outer(ctx, offset0)
    d = ctx.decompose(c1, level, ops)
    A = ctx.lift(c0, level)
    B = ctx.lift(c1, level)
    ops.cw_mult += 2 * len(ext)
    f0 = F.hat(0, b0)
    C0 = ctx.mul(A, f0, ext)
    C1 = ctx.mul(B, f0, ext)
    for t in range(1, D):
        r = stride * t
        kt = ctx.hoisted_key(_key(ctx, keys, r, level, ops), r)
        x0, x1 = ctx.inner(d, kt, level, ops)
        a = ctx.auto_ntt(ctx.add(A, x0, ext), r)
        b = ctx.auto_ntt(x1, r)
        ops.cw_mult += 2 * len(ext)
        ft = F.hat(t, b0)
        C0 = ctx.add(C0, ctx.mul(a, ft, ext), ext)
        C1 = ctx.add(C1, ctx.mul(b, ft, ext), ext)
    if b0:
        C0, C1 = _rotate_ext(ctx, C0, C1, b0, keys, level, ops)
    return (ctx.moddown_rescale(C0, level, ops), ctx.moddown_rescale(C1, level, ops)), ops


def lt_bsgs(ctx: Ctx, ct, diags: np.ndarray, keys: dict, n1: int, n2: int, stride: int = 1,
            ops: Ops | None = None, offset0: int = 0):
    """BSGS, Eq. (5): sum_j Rot( sum_i Rot(ct, i) f^_{n1 j + i}, n1 j ) with
    f^_{n1 j + i} = phi_{-n1 j}(f_{n1 j + i}); every rotation un-hoisted.  The
    giant amounts are offset0 + stride n1 j."""
    ops = ops if ops is not None else Ops()
    c0, c1 = ct
    level = c0.shape[0]
    Q = ctx.basis(level, False)
    assert n1 * n2 == diags.shape[0]
    F = _Diags(ctx, diags, level, False)
    cts = [ct]
    for i in range(1, n1):
        cts.append(ctx.rotate(ct, stride * i, _key(ctx, keys, stride * i, level, ops), level, ops))
    res = (np.zeros((level, ctx.N), dtype=np.uint64), np.zeros((level, ctx.N), dtype=np.uint64))
    for j in range(n2):
        r = _outer(ctx, offset0 + stride * n1 * j)
        v0 = np.zeros((level, ctx.N), dtype=np.uint64)
        v1 = np.zeros((level, ctx.N), dtype=np.uint64)
        for i in range(n1):
            fh = F.hat(n1 * j + i, r)
            ops.cw_mult += 2 * level
            v0 = ctx.add(v0, ctx.mul(cts[i][0], fh, Q), Q)
            v1 = ctx.add(v1, ctx.mul(cts[i][1], fh, Q), Q)
        if r:
            v0, v1 = ctx.rotate((v0, v1), r, _key(ctx, keys, r, level, ops), level, ops)
        res = (ctx.add(res[0], v0, Q), ctx.add(res[1], v1, Q))
    return (ctx.rescale(res[0], level, ops), ctx.rescale(res[1], level, ops)), ops


def lt_dh_bsgs(ctx: Ctx, ct, diags: np.ndarray, keys: dict, n1: int, n2: int, stride: int = 1,
               ops: Ops | None = None, offset0: int = 0):
    """DH-BSGS, Algorithm 1 (giant amounts offset0 + stride n1 j)."""
    ops = ops if ops is not None else Ops()
    c0, c1 = ct
    level = c0.shape[0]
    ext = ctx.basis(level, True)
    assert n1 * n2 == diags.shape[0]
    F = _Diags(ctx, diags, level, True)
    d = ctx.decompose(c1, level, ops)                                   # line 1
    a = [ctx.lift(c0, level)]                                           # line 2
    b = [ctx.lift(c1, level)]
    for i in range(1, n1):                                              # lines 3-5
        r = stride * i
        kt = ctx.hoisted_key(_key(ctx, keys, r, level, ops), r)
        x0, x1 = ctx.inner(d, kt, level, ops)
        a.append(ctx.auto_ntt(ctx.add(a[0], x0, ext), r))
        b.append(ctx.auto_ntt(x1, r))
    C0 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
    C1 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
    for j in range(n2):                                                 # lines 7-11
        r = _outer(ctx, offset0 + stride * n1 * j)
        u0 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
        u1 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
        for i in range(n1):
            fh = F.hat(n1 * j + i, r)
            ops.cw_mult += 2 * len(ext)
            u0 = ctx.add(u0, ctx.mul(a[i], fh, ext), ext)
            u1 = ctx.add(u1, ctx.mul(b[i], fh, ext), ext)
        if r:
            u0, u1 = _rotate_ext(ctx, u0, u1, r, keys, level, ops)
        C0 = ctx.add(C0, u0, ext)
        C1 = ctx.add(C1, u1, ext)
    return (ctx.moddown_rescale(C0, level, ops), ctx.moddown_rescale(C1, level, ops)), ops  # line 12


def lt_th_bsgs(ctx: Ctx, ct, diags: np.ndarray, keys: dict, n1: int, n2: int, n3: int,
               stride: int = 1, ops: Ops | None = None, offset0: int = 0):
    """TH-BSGS, Algorithm 2 (n'1 = n1, n'2 = n2, n'3 = n3; outer amounts
    offset0 + stride n1 n2 k)."""
    ops = ops if ops is not None else Ops()
    c0, c1 = ct
    level = c0.shape[0]
    ext = ctx.basis(level, True)
    assert n1 * n2 * n3 == diags.shape[0]
    F = _Diags(ctx, diags, level, True)
    d = [ctx.decompose(c1, level, ops)]                                 # line 1
    a = [None] * (n1 * n2)
    b = [None] * (n1 * n2)
    a[0] = ctx.lift(c0, level)                                          # line 2
    b[0] = ctx.lift(c1, level)
    for i in range(1, n1):                                              # lines 3-7
        r = stride * i
        kt = ctx.hoisted_key(_key(ctx, keys, r, level, ops), r)
        x0, x1 = ctx.inner(d[0], kt, level, ops)
        a[i] = ctx.auto_ntt(ctx.add(a[0], x0, ext), r)
        b[i] = ctx.auto_ntt(x1, r)
        bp = ctx.moddown(b[i], level, ops)
        d.append(ctx.decompose(bp, level, ops))
    for i in range(n1):                                                 # lines 8-11
        for j in range(1, n2):
            r = stride * n1 * j
            kt = ctx.hoisted_key(_key(ctx, keys, r, level, ops), r)
            x0, x1 = ctx.inner(d[i], kt, level, ops)
            a[n1 * j + i] = ctx.auto_ntt(ctx.add(a[i], x0, ext), r)
            b[n1 * j + i] = ctx.auto_ntt(x1, r)

    def sum_products(k, r):
        u0 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
        u1 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
        for i in range(n1 * n2):
            fh = F.hat(n1 * n2 * k + i, r)
            ops.cw_mult += 2 * len(ext)
            u0 = ctx.add(u0, ctx.mul(a[i], fh, ext), ext)
            u1 = ctx.add(u1, ctx.mul(b[i], fh, ext), ext)
        return u0, u1

    C0 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
    C1 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
    for k in range(n3):                                                 # lines 12-18
        r = _outer(ctx, offset0 + stride * n1 * n2 * k)
        u0, u1 = sum_products(k, r)
        if r:
            u0, u1 = _rotate_ext(ctx, u0, u1, r, keys, level, ops)
        C0 = ctx.add(C0, u0, ext)
        C1 = ctx.add(C1, u1, ext)
    return (ctx.moddown_rescale(C0, level, ops), ctx.moddown_rescale(C1, level, ops)), ops  # line 19


def rotation_set(algo: str, D: int, split, stride: int, n_slots: int, offset0: int = 0) -> list:
    """Rotation amounts whose keys each algorithm needs (mod N/2)."""
    if algo == "diag":
        rs = [stride * t for t in range(1, D)] + [offset0]
    elif algo in ("bsgs", "dh"):
        n1, n2 = split[0], split[1]
        rs = [stride * i for i in range(1, n1)] + [offset0 + stride * n1 * j for j in range(n2)]
    elif algo == "th":
        n1, n2, n3 = split
        rs = ([stride * i for i in range(1, n1)] + [stride * n1 * j for j in range(1, n2)]
              + [offset0 + stride * n1 * n2 * k for k in range(n3)])
    else:
        raise ValueError(algo)
    return sorted({r % n_slots for r in rs} - {0})


def fp64_reference(z: np.ndarray, fvals: np.ndarray, stride: int = 1, offset0: int = 0) -> np.ndarray:
    """y[j] = sum_t f_t[j] z[(j + offset0 + stride t) mod n]  (the plain matrix-vector product)."""
    n = z.shape[0]
    y = np.zeros(n, dtype=np.complex128)
    idx = np.arange(n)
    for t in range(fvals.shape[0]):
        y += fvals[t] * z[(idx + offset0 + stride * t) % n]
    return y


def lt_chain(ctx: Ctx, ct, stages, keys: dict):
    """A chain of LTs, one level each (the stages of a factored transform):
    `stages` lists (diags, algo, split, stride, offset0); each stage takes the
    previous stage's output."""
    for diags, algo, split, stride, offset0 in stages:
        ct, _ = run(ctx, algo, ct, diags, keys, split, stride, offset0)
    return ct


def run(ctx: Ctx, algo: str, ct, diags, keys, split=None, stride: int = 1, offset0: int = 0):
    if algo == "diag":
        return lt_diag(ctx, ct, diags, keys, stride, offset0=offset0)
    if algo == "bsgs":
        return lt_bsgs(ctx, ct, diags, keys, split[0], split[1], stride, offset0=offset0)
    if algo == "dh":
        return lt_dh_bsgs(ctx, ct, diags, keys, split[0], split[1], stride, offset0=offset0)
    if algo == "th":
        return lt_th_bsgs(ctx, ct, diags, keys, *split, stride=stride, offset0=offset0)
    raise ValueError(algo)
