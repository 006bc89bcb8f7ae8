"""Seeded synthetic inputs: parameter sets (NTT-friendly primes) and random streams.

This module holds none of the linear-transformation arithmetic.  It only
produces the numbers that both sides consume:

* the modulus chains of the workloads (the paper's Table "HE parameters" gives
  bit widths only; the primes themselves are chosen here: the largest primes
  below 2^w with q = 1 mod 2N, in descending order);
* counter-based random streams (SplitMix64 output function applied to a
  counter, Steele/Lea/Flood 2014), and samplers built on them: uniform
  residues, ternary secrets, rounded Gaussians, uniform slot values and
  uniform matrix diagonals.

Every random number the method needs is drawn here and passed to the
consumer as an input array, so the CPU oracle and the GPU library never have
to agree on a generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


# --------------------------------------------------------------------------- primes
def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases 2..41)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, count: int, two_n: int, exclude=()) -> list[int]:
    """The `count` largest primes below 2^bits with q = 1 (mod two_n), descending."""
    c = ((1 << bits) - 2) // two_n * two_n + 1
    out: list[int] = []
    ex = set(exclude)
    while len(out) < count:
        if c <= two_n:
            raise ValueError("ran out of candidates")
        if c not in ex and is_prime(c):
            out.append(c)
        c -= two_n
    return out


@dataclass(frozen=True)
class ParamSet:
    """One CKKS parameter set: ring degree, Q chain, special primes P, dnum."""

    name: str
    log_n: int
    q: tuple
    p: tuple
    dnum: int
    log_scale: int = 40
    sigma: float = 3.2
    notes: str = field(default="", compare=False)

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def L(self) -> int:  # number of Q limbs at the top level
        return len(self.q)

    @property
    def k(self) -> int:
        return len(self.p)

    @property
    def alpha(self) -> int:
        return -(-self.L // self.dnum)

    @property
    def moduli(self) -> tuple:
        return tuple(self.q) + tuple(self.p)


def make_params(name: str, log_n: int, q_bits: list, p_bits: list, dnum: int,
                notes: str = "") -> ParamSet:
    two_n = 2 << log_n
    q: list[int] = []
    # each entry takes the largest not-yet-used prime of its width
    for bits in q_bits:
        q.append(ntt_primes(bits, 1, two_n, exclude=q)[0])
    p: list[int] = []
    for bits in p_bits:
        p.append(ntt_primes(bits, 1, two_n, exclude=q + p)[0])
    return ParamSet(name, log_n, tuple(q), tuple(p), dnum, notes=notes)


_CACHE: dict = {}


def param_set(name: str) -> ParamSet:
    """Named parameter sets of the workloads.

    toy  : N=2^12, Q = 50b + 3x40b, P = 1x60b, dnum 4 (functional toy, not secure)
    n16  : N=2^16, Q = 55b + 23x40b (24 limbs), P = 4x60b, dnum 6 (alpha 4, beta 6)
    n15  : N=2^15, Q = 50b + 15x40b (16 limbs), P = 3x60b, dnum 4 (alpha 4)
    n14  : N=2^14, Q = 50b + 7x40b (8 limbs), P = 2x60b, dnum 4 (alpha 2)
    setA : the paper's Set-A shape, N=2^13, L+1=5, alpha=5, beta=1, 54-bit words
    setB : the paper's Set-B shape, N=2^15, L+1=16, alpha=8, beta=2, 54-bit words
    n16d8, n14d8, n15d16 : n16 / n14 / n15 with more digits (dnum 8, 8, 16: beta 8, 8, 16),
           the shapes where the staged diagonal kernel's 6-digit key registers do not suffice
    """
    if name in _CACHE:
        return _CACHE[name]
    if name == "toy":
        ps = make_params("toy", 12, [50, 40, 40, 40], [60], 4,
                         "functional toy, not a secure parameter set")
    elif name == "n16":
        ps = make_params("n16", 16, [55] + [40] * 23, [60] * 4, 6)
    elif name == "n15":
        ps = make_params("n15", 15, [50] + [40] * 15, [60] * 3, 4)
    elif name == "n14":  # covers the N = 2^14 transform shape (7 + 7 NTT stages per pass)
        ps = make_params("n14", 14, [50] + [40] * 7, [60] * 2, 4)
    elif name == "setA":
        ps = make_params("setA", 13, [54] * 5, [54] * 5, 1)
    elif name == "setB":
        ps = make_params("setB", 15, [54] * 16, [54] * 8, 2)
    elif name == "n16d8":
        ps = make_params("n16d8", 16, [55] + [40] * 23, [60] * 4, 8)
    elif name == "n14d8":
        ps = make_params("n14d8", 14, [50] + [40] * 7, [60] * 2, 8)
    elif name == "n15d16":
        ps = make_params("n15d16", 15, [50] + [40] * 15, [60] * 3, 16)
    elif name == "tiny":  # unit-test size
        ps = make_params("tiny", 5, [50, 40, 40, 40], [60, 60], 2)
    else:
        raise KeyError(name)
    _CACHE[name] = ps
    return ps


# --------------------------------------------------------------------------- streams
def stream_id(name: str) -> int:
    """64-bit FNV-1a of a stream name (keeps stream identities readable)."""
    h = 0xCBF29CE484222325
    for ch in name.encode():
        h ^= ch
        h = (h * 0x100000001B3) & _MASK
    return h


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def _mix_int(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def u64(seed: int, stream, count: int, offset: int = 0) -> np.ndarray:
    """`count` uniform 64-bit words of stream `stream` (an int or a name).

    Word i is mix(key + (offset + i + 1) * gamma) where key depends only on
    (seed, stream): a counter-based SplitMix64.
    """
    sid = stream_id(stream) if isinstance(stream, str) else int(stream) & _MASK
    key = _mix_int(_mix_int(seed * _GAMMA + 1) ^ sid)
    ctr = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + ctr * np.uint64(_GAMMA)
        return _mix(z)


def uniform_mod(seed: int, stream, moduli, n: int) -> np.ndarray:
    """Array [len(moduli)][n] with row i uniform in [0, moduli[i]) (rejection)."""
    out = np.empty((len(moduli), n), dtype=np.uint64)
    for i, q in enumerate(moduli):
        bits = int(q).bit_length()
        mask = np.uint64((1 << bits) - 1)
        row = np.empty(n, dtype=np.uint64)
        todo = np.arange(n)
        attempt = 0
        while todo.size:
            cand = u64(seed, f"{stream}/{i}/{attempt}", n)[todo] & mask
            ok = cand < np.uint64(q)
            row[todo[ok]] = cand[ok]
            todo = todo[~ok]
            attempt += 1
        out[i] = row
    return out


def ternary(seed: int, stream, n: int) -> np.ndarray:
    """n values uniform in {-1, 0, 1} (2 bits, rejecting 3), as int64."""
    out = np.empty(n, dtype=np.int64)
    todo = np.arange(n)
    attempt = 0
    while todo.size:
        v = (u64(seed, f"{stream}/{attempt}", n)[todo] & np.uint64(3)).astype(np.int64)
        ok = v < 3
        out[todo[ok]] = v[ok] - 1
        todo = todo[~ok]
        attempt += 1
    return out


def _unit(words: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (words >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def gaussian(seed: int, stream, n: int, sigma: float = 3.2) -> np.ndarray:
    """n rounded Gaussians of std sigma (Box-Muller), rejecting |e| > 6 sigma."""
    out = np.empty(n, dtype=np.int64)
    todo = np.arange(n)
    attempt = 0
    while todo.size:
        u1 = _unit(u64(seed, f"{stream}/u1/{attempt}", n)[todo])
        u2 = _unit(u64(seed, f"{stream}/u2/{attempt}", n)[todo])
        r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0, 1]
        e = np.rint(sigma * r * np.cos(2.0 * math.pi * u2)).astype(np.int64)
        ok = np.abs(e) <= 6.0 * sigma
        out[todo[ok]] = e[ok]
        todo = todo[~ok]
        attempt += 1
    return out


def uniform_real(seed: int, stream, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * _unit(u64(seed, stream, n))


def slots(seed: int, stream, n_slots: int) -> np.ndarray:
    """Complex slot vector, real and imaginary parts uniform in [-1, 1]."""
    return (uniform_real(seed, f"{stream}/re", n_slots)
            + 1j * uniform_real(seed, f"{stream}/im", n_slots))


def diagonal_values(seed: int, stream, n_diag: int, n_slots: int) -> np.ndarray:
    """[n_diag][n_slots] real matrix diagonals, entries uniform in [-1, 1].

    Row t holds f_t[j] = F[j][(j + o_t) mod n]: the matrix F is sampled
    through its nonzero diagonals and never materialised.
    """
    return uniform_real(seed, stream, n_diag * n_slots).reshape(n_diag, n_slots)


def uniform_mod_device(seed: int, stream, moduli, n: int, count: int = 1, device="cuda"):
    """[count][len(moduli)][n] int64 device tensor, row i uniform in
    [0, moduli[i]) (torch's seeded generator on the device).  Used for
    throughput runs whose values need only the right shape and range."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed((seed * 0x9E3779B1 + stream_id(stream)) % (1 << 63))
    out = torch.empty((count, len(moduli), n), dtype=torch.int64, device=device)
    for i, q in enumerate(moduli):
        out[:, i].random_(0, int(q), generator=g)
    return out
