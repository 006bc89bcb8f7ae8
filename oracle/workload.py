"""CPU oracle: builds a complete LT problem (secret, keys, ciphertext, encoded
diagonals) from a parameter set and a seed, and evaluates it.

TEST INFRASTRUCTURE ONLY (see oracle/ckks.py).

Input recipe (every random number comes from paper_2605_17222_gb300.synth):
  * secret s: uniform ternary; errors: rounded Gaussian, sigma 3.2
  * input slots z: real and imaginary parts uniform in [-1, 1]
  * matrix: D nonzero diagonals with offsets o_t = offset0 + stride * t, entries
    uniform in [-1, 1]; f_t[j] = F[j][(j + o_t) mod N/2] is sampled directly
  * ciphertext scale 2^40, diagonal scale 2^40; diagonals encoded at the top
    level over all Q and P moduli (the hoisted algorithms multiply in PQ)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from paper_2605_17222_gb300 import synth

from . import dft as _dft
from . import lt as _lt
from .ckks import Ctx


@dataclass
class Problem:
    ctx: Ctx
    seed: int
    level: int
    stride: int
    s: np.ndarray           # ternary secret (int64 coefficients)
    z: np.ndarray           # input slots
    fvals: np.ndarray       # [D][N/2] diagonal values
    diags: np.ndarray       # [D][L + k][N] encoded diagonals (top level, NTT domain)
    ct: tuple               # (c0, c1) at `level`
    keys: dict              # r -> [beta_max][2][L + k][N]
    scale: float
    diag_scale: float
    offset0: int = 0

    @property
    def D(self) -> int:
        return self.fvals.shape[0]

    def out_scale(self) -> float:
        return self.scale * self.diag_scale / self.ctx.q[self.level - 1]

    def expected(self) -> np.ndarray:
        return _lt.fp64_reference(self.z, self.fvals, self.stride, self.offset0)

    def decrypt(self, ct) -> np.ndarray:
        return self.ctx.decrypt(ct, self.s, self.out_scale())


def encode_diagonals(ctx: Ctx, fvals: np.ndarray, scale: float) -> np.ndarray:
    top = ctx.q + ctx.p
    out = np.empty((fvals.shape[0], len(top), ctx.N), dtype=np.uint64)
    for t in range(fvals.shape[0]):
        out[t] = ctx.encode(fvals[t].astype(np.complex128), scale, top)
    return out


def make_problem(param_name: str, seed: int, D: int, level: int | None = None, stride: int = 1,
                 rotations=(), log_scale: int = 40, log_diag_scale: int = 40,
                 ctx: Ctx | None = None, offset0: int = 0) -> Problem:
    ps = synth.param_set(param_name)
    ctx = ctx or Ctx(ps)
    level = level or ctx.L
    scale = float(2 ** log_scale)
    dscale = float(2 ** log_diag_scale)
    s = ctx.secret(seed)
    z = synth.slots(seed, "input", ctx.N // 2)
    fvals = synth.diagonal_values(seed, "diag", D, ctx.N // 2)
    diags = encode_diagonals(ctx, fvals, dscale)
    ct = ctx.encrypt(z, s, level, scale, seed)
    keys = {r: ctx.keygen_rotation(s, r, seed) for r in sorted(set(rotations))}
    return Problem(ctx, seed, level, stride, s, z, fvals, diags, ct, keys, scale, dscale, offset0)


def add_keys(pb: Problem, rotations) -> None:
    for r in sorted(set(rotations)):
        if r not in pb.keys:
            pb.keys[r] = pb.ctx.keygen_rotation(pb.s, r, pb.seed)


@dataclass
class ChainProblem:
    """A ciphertext and the stages of a factored slot DFT (SlotToCoeff or
    CoeffToSlot), each stage's diagonals encoded at the scale of the prime its
    rescale drops, so every stage keeps the ciphertext scale."""
    ctx: Ctx
    seed: int
    level: int
    s: np.ndarray
    z: np.ndarray
    windows: list          # dft.Window per stage
    diags: list            # [D_i][L + k][N] per stage
    splits: list
    ct: tuple
    keys: dict
    scale: float

    def stages(self, algo: str = "th") -> list:
        return [(d, algo, sp, w.stride, w.offset0) for d, sp, w in zip(self.diags, self.splits, self.windows)]

    def expected(self) -> np.ndarray:
        return _dft.apply_windows(self.z, self.windows)

    def out_scale(self) -> float:
        sc = self.scale
        for i in range(len(self.windows)):
            q = self.ctx.q[self.level - 1 - i]
            sc = sc * float(q) / q
        return sc

    def decrypt(self, ct) -> np.ndarray:
        return self.ctx.decrypt(ct, self.s, self.out_scale())


def make_chain_problem(param_name: str, seed: int, kind: str, radices, splits, level: int | None = None,
                       pad: bool = True, amplitude: float = 0.25, log_scale: int = 40,
                       ctx: Ctx | None = None) -> ChainProblem:
    """kind "stc": S_m .. S_1 applied to bit-reversed slots; "cts": S_1^-1 .. S_m^-1.
    `splits` gives each stage's TH split (its keys are generated)."""
    ps = synth.param_set(param_name)
    ctx = ctx or Ctx(ps)
    level = level or ctx.L
    n = ctx.N // 2
    windows = (_dft.slot_to_coeff if kind == "stc" else _dft.coeff_to_slot)(n, radices, pad)
    if len(splits) != len(windows) or level - len(windows) < 1:
        raise ValueError("one split per stage, and a level per stage")
    s = ctx.secret(seed)
    z = amplitude * synth.slots(seed, f"chain/{kind}", n)
    scale = float(2 ** log_scale)
    diags = [encode_diagonals(ctx, w.fvals, float(ctx.q[level - 1 - i])) for i, w in enumerate(windows)]
    ct = ctx.encrypt(z, s, level, scale, seed)
    rots = set()
    for w, sp in zip(windows, splits):
        rots |= set(_lt.rotation_set("th", w.D, sp, w.stride, n, w.offset0))
    keys = {r: ctx.keygen_rotation(s, r, seed) for r in sorted(rots)}
    return ChainProblem(ctx, seed, level, s, z, windows, diags, list(splits), ct, keys, scale)
