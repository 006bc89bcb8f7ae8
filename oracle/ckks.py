"""CPU oracle, CKKS layer: parameters, NTT, automorphisms, encoding, keys,
encryption, decryption and the three key-switching steps.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference the GPU library
is checked against; only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it.  It shares no code with the GPU library.

Paper: Akherati & Zhang, "Triple-Hoisted Baby-Step Giant-Step Linear
Transformation over CKKS Homomorphic Encryption and Hardware Accelerator".
Section II-A (RNS-CKKS) defines every step below:
  * RNS limbs, plaintext x ciphertext product ............ Sec. II-A
  * rescale ............................................... Eq. (1)
  * rotation automorphism phi_r, g = 5 ..................... Eq. (2)
  * key switching: Decompose (ModUp), <d, swk>, ModDown ..... Fig. 1, Eq. (3), Eq. (4)
  * NTT-domain automorphism index map ...................... Eq. (7)
Where the paper is silent the reading taken is stated in the docstring.

Polynomials are numpy uint64 arrays [n_limbs][N]; a "basis" is the list of
moduli of the rows.  Ring elements live in the NTT domain in bit-reversed
order unless a docstring says "coefficients".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import _native as nat


def find_psi(q: int, n: int) -> int:
    """Primitive 2N-th root of unity mod q: psi = x^((q-1)/2N) for the smallest
    x >= 2 with psi^N = -1 (the paper fixes no root; this is the reading)."""
    assert (q - 1) % (2 * n) == 0
    x = 2
    while True:
        psi = pow(x, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi
        x += 1


@dataclass
class Ops:
    """Operation counters (Table "complexity comparisons")."""

    decompose: int = 0
    moddown: int = 0          # polynomials passed through ModDown (merged MDR included)
    ks_products: int = 0      # switching-key inner products <d, swk>
    cw_mult: int = 0          # coefficient-wise limb-polynomial multiplications
    keys: set = field(default_factory=set)
    rescale: int = 0


class Ctx:
    """RNS-CKKS context (Sec. II-A).  L Q-limbs q_0..q_{L-1}, k special
    primes p_0..p_{k-1}, alpha = ceil(L/dnum) limbs per digit."""

    def __init__(self, ps):
        self.ps = ps
        self.log_n = ps.log_n
        self.N = 1 << ps.log_n
        self.q = [int(v) for v in ps.q]
        self.p = [int(v) for v in ps.p]
        self.L = len(self.q)
        self.k = len(self.p)
        self.alpha = -(-self.L // ps.dnum)
        self.beta_max = -(-self.L // self.alpha)
        self.P = math.prod(self.p)
        self.psi = {m: find_psi(m, self.N) for m in self.q + self.p}
        self.lib = nat.lib()

    # ------------------------------------------------------------ bases
    def basis(self, level: int, ext: bool) -> list:
        """Q_level = q_0..q_{level-1}; with ext, followed by p_0..p_{k-1}."""
        return self.q[:level] + (self.p if ext else [])

    def beta(self, level: int) -> int:
        """beta = ceil(level / alpha) digits (Sec. II-A)."""
        return -(-level // self.alpha)

    def digit_range(self, b: int, level: int) -> range:
        """Digit b holds limbs alpha*b .. min(alpha*(b+1), level) - 1.  The
        paper prints the upper end as min(alpha(b+1)-1, L+1); the reading is L
        (the last limb index), i.e. the last digit is partial."""
        return range(self.alpha * b, min(self.alpha * (b + 1), level))

    def galois(self, r: int) -> int:
        """g_r = 5^r mod 2N (Eq. 2); negative r through the order N/2 of 5."""
        return pow(5, r % (self.N // 2), 2 * self.N)

    def ext_rows(self, level: int) -> list:
        """Rows of a top-level extended array (L Q-limbs then k P-limbs) that
        form the extended basis at `level`."""
        return list(range(level)) + list(range(self.L, self.L + self.k))

    # ------------------------------------------------------------ primitives
    def _arr(self, a) -> np.ndarray:
        return np.ascontiguousarray(a, dtype=np.uint64)

    def ntt(self, a, basis) -> np.ndarray:
        out = self._arr(a).copy()
        assert out.shape == (len(basis), self.N)
        qs = nat.u64arr(basis)
        ps = nat.u64arr([self.psi[m] for m in basis])
        self.lib.orc_ntt(nat.ptr(out), len(basis), self.log_n, nat.ptr(qs), nat.ptr(ps))
        return out

    def intt(self, a, basis) -> np.ndarray:
        out = self._arr(a).copy()
        assert out.shape == (len(basis), self.N)
        qs = nat.u64arr(basis)
        ps = nat.u64arr([self.psi[m] for m in basis])
        self.lib.orc_intt(nat.ptr(out), len(basis), self.log_n, nat.ptr(qs), nat.ptr(ps))
        return out

    def _bin(self, fn, a, b, basis) -> np.ndarray:
        a = self._arr(a)
        b = self._arr(b)
        assert a.shape == b.shape == (len(basis), self.N), (a.shape, b.shape, len(basis))
        out = np.empty_like(a)
        qs = nat.u64arr(basis)
        fn(nat.ptr(a), nat.ptr(b), nat.ptr(out), len(basis), self.N, nat.ptr(qs))
        return out

    def mul(self, a, b, basis):
        return self._bin(self.lib.orc_mul, a, b, basis)

    def add(self, a, b, basis):
        return self._bin(self.lib.orc_add, a, b, basis)

    def sub(self, a, b, basis):
        return self._bin(self.lib.orc_sub, a, b, basis)

    def mul_const(self, a, consts, basis):
        a = self._arr(a)
        out = np.empty_like(a)
        c = nat.u64arr([int(v) % m for v, m in zip(consts, basis)])
        qs = nat.u64arr(basis)
        self.lib.orc_mul_const(nat.ptr(a), nat.ptr(c), nat.ptr(out), len(basis), self.N, nat.ptr(qs))
        return out

    def bconv(self, y, src, dst) -> np.ndarray:
        """Eq. (3): sum_j y_j * [Qs/q_j]_t mod t for every target t, where
        y_j = [a^(j) * (Qs/q_j)^-1]_{q_j} has already been formed."""
        y = self._arr(y)
        Qs = math.prod(src)
        tab = nat.u64arr([(Qs // qj) % t for t in dst for qj in src])
        out = np.empty((len(dst), self.N), dtype=np.uint64)
        ts = nat.u64arr(dst)
        self.lib.orc_bconv(nat.ptr(y), len(src), nat.ptr(tab), nat.ptr(out), len(dst), self.N,
                           nat.ptr(ts))
        return out

    def auto_ntt(self, a, r: int) -> np.ndarray:
        """phi_r in the NTT domain (Eq. 7): a gather on the evaluation points."""
        a = self._arr(a)
        out = np.empty_like(a)
        self.lib.orc_auto_ntt(nat.ptr(a), nat.ptr(out), a.shape[0], self.log_n, self.galois(r))
        return out

    def auto_coeff(self, a, r: int, basis) -> np.ndarray:
        """phi_r on coefficients (Eq. 2): a(x) -> a(x^g) mod x^N + 1."""
        a = self._arr(a)
        out = np.empty_like(a)
        qs = nat.u64arr(basis)
        self.lib.orc_auto_coeff(nat.ptr(a), nat.ptr(out), a.shape[0], self.log_n, self.galois(r),
                                nat.ptr(qs))
        return out

    def residues(self, ints: np.ndarray, basis) -> np.ndarray:
        """Signed integer coefficients (int64, or object for big values) -> residues."""
        out = np.empty((len(basis), self.N), dtype=np.uint64)
        if ints.dtype == object:
            for i, m in enumerate(basis):
                out[i] = np.array([int(v) % m for v in ints], dtype=np.uint64)
        else:
            for i, m in enumerate(basis):
                out[i] = np.mod(ints, m).astype(np.uint64)
        return out

    # ------------------------------------------------------------ encoding (Sec. II-A packing)
    def _slot_positions(self):
        """Evaluation-point index l (point zeta^(2l+1), zeta = e^(i pi/N)) of slot j and of its conjugate."""
        n2 = 2 * self.N
        e = np.array([pow(5, j, n2) for j in range(self.N // 2)], dtype=np.int64)
        return (e - 1) // 2, (n2 - e - 1) // 2

    def encode_coeffs(self, z: np.ndarray, scale: float) -> np.ndarray:
        """Canonical-embedding encoding: the real polynomial m with
        m(zeta^(5^j)) = z_j and m(zeta^(-5^j)) = conj(z_j); returns
        round(scale * m) as int64 coefficients.  An FFT evaluates the
        inverse embedding (a library primitive used as one step)."""
        N = self.N
        pos, neg = self._slot_positions()
        V = np.zeros(N, dtype=np.complex128)
        V[pos] = z
        V[neg] = np.conj(z)
        t = np.arange(N)
        b = np.fft.fft(V) / N                      # b_t = m_t zeta^t
        m = (b * np.exp(-1j * np.pi * t / N)).real
        return np.rint(m * scale).astype(np.int64)

    def decode_coeffs(self, m: np.ndarray, scale: float) -> np.ndarray:
        """Inverse of encode_coeffs: evaluate m at zeta^(5^j), divide by scale."""
        N = self.N
        t = np.arange(N)
        b = np.asarray(m, dtype=np.float64) * np.exp(1j * np.pi * t / N)
        V = np.fft.ifft(b) * N                     # V[l] = m(zeta^(2l+1))
        pos, _ = self._slot_positions()
        return V[pos] / scale

    def encode(self, z, scale, basis) -> np.ndarray:
        return self.ntt(self.residues(self.encode_coeffs(z, scale), basis), basis)

    def crt_centered(self, res: np.ndarray, basis) -> np.ndarray:
        """Centered integer from the first two limbs, or the only limb
        (|m| < modulus / 4 asserted)."""
        q0 = basis[0]
        q1 = basis[1] if len(basis) > 1 else 1
        inv = pow(q0, -1, q1) if q1 > 1 else 0
        r0 = [int(v) for v in res[0]]
        r1 = [int(v) for v in res[1]] if q1 > 1 else [0] * self.N
        M = q0 * q1
        out = np.empty(self.N, dtype=object)
        for i in range(self.N):
            x = r0[i] + q0 * (((r1[i] - r0[i]) * inv) % q1)
            if x > M // 2:
                x -= M
            assert abs(x) < M // 4, "plaintext too large for a two-limb decode"
            out[i] = x
        return out

    # ------------------------------------------------------------ keys and encryption
    def secret(self, seed: int):
        from paper_2605_17222_gb300 import synth
        return synth.ternary(seed, "secret", self.N)

    def secret_ntt(self, s: np.ndarray, basis) -> np.ndarray:
        return self.ntt(self.residues(s, basis), basis)

    def keygen_rotation(self, s: np.ndarray, r: int, seed: int) -> np.ndarray:
        """Switching key from phi_r(s) to s, standard (un-hoisted) form.

        The paper does not spell out key formation; the reading is the
        standard hybrid key of the RNS-CKKS literature, with the gadget implied
        by Sec. II-A: for digit b,
            swk_{b,0} = -a_b s + e_b + [j in digit b] [P]_{q_j} phi_r(s),
            swk_{b,1} = a_b,
        over all L + k moduli.  Layout [beta_max][2][L + k][N], NTT domain."""
        from paper_2605_17222_gb300 import synth
        top = self.q + self.p
        g = self.galois(r)
        # phi_r(s) on integer coefficients (signed permutation, Eq. 2)
        s_rot = np.zeros(self.N, dtype=np.int64)
        for t in range(self.N):
            pos = (t * g) % (2 * self.N)
            if pos < self.N:
                s_rot[pos] = s[t]
            else:
                s_rot[pos - self.N] = -s[t]
        S = self.secret_ntt(s, top)
        Sr = self.secret_ntt(s_rot, top)
        key = np.empty((self.beta_max, 2, len(top), self.N), dtype=np.uint64)
        for b in range(self.beta_max):
            a = synth.uniform_mod(seed, f"swk/{r}/{b}/a", top, self.N)
            e = self.ntt(self.residues(synth.gaussian(seed, f"swk/{r}/{b}/e", self.N), top), top)
            k0 = self.sub(e, self.mul(a, S, top), top)
            for j in self.digit_range(b, self.L):
                k0[j] = self.add(k0[j:j + 1],
                                 self.mul_const(Sr[j:j + 1], [self.P % top[j]], [top[j]]),
                                 [top[j]])[0]
            key[b, 0] = k0
            key[b, 1] = a
        return key

    def key_at_level(self, key: np.ndarray, level: int) -> np.ndarray:
        """Drop Q limbs >= level and digits >= beta(level)."""
        return np.ascontiguousarray(key[: self.beta(level)][:, :, self.ext_rows(level)])

    def encrypt(self, z, s: np.ndarray, level: int, scale: float, seed: int, stream="ct"):
        """Symmetric encryption: c1 = a, c0 = -a s + m + e over Q_level (NTT)."""
        from paper_2605_17222_gb300 import synth
        B = self.basis(level, False)
        m = self.encode(z, scale, B)
        a = synth.uniform_mod(seed, f"{stream}/a", B, self.N)
        e = self.ntt(self.residues(synth.gaussian(seed, f"{stream}/e", self.N), B), B)
        S = self.secret_ntt(s, B)
        c0 = self.add(self.sub(e, self.mul(a, S, B), B), m, B)
        return (c0, a)

    def decrypt_coeffs(self, ct, s: np.ndarray):
        c0, c1 = ct
        level = c0.shape[0]
        B = self.basis(level, False)
        S = self.secret_ntt(s, B)
        m = self.intt(self.add(c0, self.mul(c1, S, B), B), B)
        return self.crt_centered(m, B)

    def decrypt(self, ct, s: np.ndarray, scale: float) -> np.ndarray:
        m = self.decrypt_coeffs(ct, s)
        return self.decode_coeffs(np.array([float(v) for v in m]), scale)

    # ------------------------------------------------------------ key switching (Fig. 1)
    def decompose(self, c, level: int, ops: Ops | None = None) -> list:
        """Decompose(c, alpha, beta, Q, P) (Fig. 1; ModUp by Eq. 3).

        For each digit b with limbs j in b and Q_b = prod q_j: INTT the limbs,
        y_j = [c^(j) (Q_b/q_j)^-1]_{q_j}, then for every other modulus t of
        Q_level u P, d_b^(t) = sum_j y_j [Q_b/q_j]_t mod t (fast basis
        conversion, used literally: no exact correction); for t in b,
        d_b^(t) = c^(t).  NTT the new limbs.  Returns beta arrays over the
        extended basis (Q limbs first, then P limbs)."""
        if ops is not None:
            ops.decompose += 1
        Q = self.basis(level, False)
        ext = self.basis(level, True)
        coeff = self.intt(c, Q)
        digits = []
        for b in range(self.beta(level)):
            rng = self.digit_range(b, level)
            src = [Q[j] for j in rng]
            Qb = math.prod(src)
            y = self.mul_const(coeff[rng.start:rng.stop], [pow(Qb // qj, -1, qj) for qj in src], src)
            tgt_rows = [t for t in range(len(ext)) if t not in rng]
            tgt = [ext[t] for t in tgt_rows]
            conv = self.ntt(self.bconv(y, src, tgt), tgt)
            d = np.empty((len(ext), self.N), dtype=np.uint64)
            d[rng.start:rng.stop] = c[rng.start:rng.stop]
            d[tgt_rows] = conv
            digits.append(d)
        return digits

    def inner(self, digits: list, key_l: np.ndarray, level: int, ops: Ops | None = None):
        """<d, swk> = sum_b d_b (swk_{b,0}, swk_{b,1}) mod PQ (Sec. II-A)."""
        ext = self.basis(level, True)
        if ops is not None:
            ops.ks_products += 1
            ops.cw_mult += 2 * len(digits) * len(ext)
        x0 = np.zeros((len(ext), self.N), dtype=np.uint64)
        x1 = np.zeros((len(ext), self.N), dtype=np.uint64)
        for b, d in enumerate(digits):
            x0 = self.add(x0, self.mul(d, key_l[b, 0], ext), ext)
            x1 = self.add(x1, self.mul(d, key_l[b, 1], ext), ext)
        return x0, x1

    def moddown(self, x, level: int, ops: Ops | None = None) -> np.ndarray:
        """ModDown, Eq. (4): P^-1 (x^(Q) - BConv(x^(P), P, Q)) mod q_j."""
        if ops is not None:
            ops.moddown += 1
        Q = self.basis(level, False)
        xP = self.intt(x[level:], self.p)
        y = self.mul_const(xP, [pow(self.P // pi, -1, pi) for pi in self.p], self.p)
        conv = self.ntt(self.bconv(y, self.p, Q), Q)
        return self.mul_const(self.sub(x[:level], conv, Q), [pow(self.P, -1, qj) for qj in Q], Q)

    def rescale(self, x, level: int, ops: Ops | None = None) -> np.ndarray:
        """Rescale, Eq. (1), literally in the coefficient domain:
        [q_last^-1 (c^(j) - c^(last))]_{q_j}, c^(last) taken in [0, q_last)."""
        if ops is not None:
            ops.rescale += 1
        Q = self.basis(level, False)
        ql = Q[-1]
        coeff = self.intt(x, Q)
        last = coeff[level - 1]
        out = np.empty((level - 1, self.N), dtype=np.uint64)
        for j in range(level - 1):
            qj = Q[j]
            inv = pow(ql, -1, qj)
            cj = [int(v) for v in coeff[j]]
            lv = [int(v) for v in last]
            out[j] = np.array([(inv * (a - b)) % qj for a, b in zip(cj, lv)], dtype=np.uint64)
        return self.ntt(out, Q[:-1])

    def moddown_rescale(self, x, level: int, ops: Ops | None = None) -> np.ndarray:
        """ModDown merged with rescale (Alg. 2 line 19, Sec. III).

        The paper cites the merge without its construction; the reading is
        Eq. (4) with the source basis B' = {q_{level-1}, p_0..p_{k-1}} and
        P' = q_{level-1} P, producing limbs q_0..q_{level-2}.  With k = 0 it
        is exactly Eq. (1)."""
        if ops is not None:
            ops.moddown += 1
        Q = self.basis(level, False)
        out_b = Q[:-1]
        src = [Q[-1]] + self.p
        Pp = math.prod(src)
        xs = self.intt(x[level - 1:], src)
        y = self.mul_const(xs, [pow(Pp // b, -1, b) for b in src], src)
        conv = self.ntt(self.bconv(y, src, out_b), out_b)
        return self.mul_const(self.sub(x[:level - 1], conv, out_b), [pow(Pp, -1, qj) for qj in out_b], out_b)

    def lift(self, c, level: int) -> np.ndarray:
        """P * c mod PQ (Alg. 1/2 line 2): Q limbs times [P]_{q_j}; P limbs 0."""
        Q = self.basis(level, False)
        out = np.zeros((level + self.k, self.N), dtype=np.uint64)
        out[:level] = self.mul_const(c, [self.P % qj for qj in Q], Q)
        return out

    def hoisted_key(self, key_l: np.ndarray, r: int) -> np.ndarray:
        """swk~_r = phi_{-r}(swk_r) (Alg. 1/2 inputs), applied to every limb."""
        out = np.empty_like(key_l)
        for b in range(key_l.shape[0]):
            for c in range(2):
                out[b, c] = self.auto_ntt(key_l[b, c], -r)
        return out

    def rotate(self, ct, r: int, key_l: np.ndarray, level: int, ops: Ops | None = None):
        """Ciphertext rotation by r slots, un-hoisted (Fig. 1): phi_r on both
        polynomials, then Decompose, <d, swk_r>, ModDown of both outputs."""
        c0, c1 = ct
        Q = self.basis(level, False)
        c0r = self.auto_ntt(c0, r)
        c1r = self.auto_ntt(c1, r)
        d = self.decompose(c1r, level, ops)
        x0, x1 = self.inner(d, key_l, level, ops)
        return (self.add(c0r, self.moddown(x0, level, ops), Q), self.moddown(x1, level, ops))
