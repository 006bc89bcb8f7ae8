/*
 * CPU oracle for the CKKS homomorphic linear transformation: primitive ring
 * operations on RNS residue polynomials.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference against
 * which the GPU library is checked.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the GPU library.
 *
 * Conventions (stated once):
 *   - A polynomial over a basis of nl moduli is nl consecutive rows ("limbs")
 *     of N uint64 words; row i holds residues mod q[i], canonical in [0, q[i]).
 *   - Every modular product is computed as ((unsigned __int128)a*b) % q.
 *   - NTT domain, bit-reversed layout: word s of a limb holds a(psi^(2*brv(s)+1))
 *     where psi is a primitive 2N-th root of unity mod q and brv reverses
 *     log2(N) bits.  The paper keeps NTT outputs in bit-reversed order
 *     (Sec. V, permutation circuit) and evaluates automorphisms in that order.
 *   - OpenMP parallelism is over independent limbs only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}
/* a, b canonical in [0, q), q < 2^63 */
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
static uint32_t brv(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

uint32_t orc_bitrev(uint32_t x, int bits) { return brv(x, bits); }
uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }
uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t q) { return powmod(a, e, q); }

/* Cyclic DFT of length 2^logn over Z_q with root w, natural order in and out:
 * X[l] = sum_t x[t] w^(l t).  Textbook iterative radix-2 FFT (bit-reversal
 * copy, then log n butterfly levels). */
static void cyclic_dft(uint64_t* a, int logn, uint64_t w, uint64_t q) {
    const uint32_t n = 1u << logn;
    uint64_t* x = (uint64_t*)malloc(sizeof(uint64_t) * n);
    for (uint32_t i = 0; i < n; i++) x[brv(i, logn)] = a[i];
    for (int s = 1; s <= logn; s++) {
        const uint32_t m = 1u << s;
        const uint64_t wm = powmod(w, n / m, q);
        for (uint32_t k = 0; k < n; k += m) {
            uint64_t wj = 1;
            for (uint32_t j = 0; j < m / 2; j++) {
                uint64_t t = mulmod(wj, x[k + j + m / 2], q);
                uint64_t u = x[k + j];
                x[k + j] = addmod(u, t, q);
                x[k + j + m / 2] = submod(u, t, q);
                wj = mulmod(wj, wm, q);
            }
        }
    }
    memcpy(a, x, sizeof(uint64_t) * n);
    free(x);
}

/* Negacyclic NTT of every limb, in place (Sec. II-A: products in R_q are
 * coefficient-wise in the NTT domain).  A(psi^(2l+1)) = sum_t (a_t psi^t) w^(lt)
 * with w = psi^2, so: twist by psi^t, cyclic DFT, then store in bit-reversed
 * order. */
void orc_ntt(uint64_t* a, int nl, int logn, const uint64_t* q, const uint64_t* psi) {
    const uint32_t n = 1u << logn;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < nl; i++) {
        uint64_t* x = a + (size_t)i * n;
        const uint64_t qi = q[i], ps = psi[i];
        uint64_t pw = 1;
        for (uint32_t t = 0; t < n; t++) {
            x[t] = mulmod(x[t], pw, qi);
            pw = mulmod(pw, ps, qi);
        }
        cyclic_dft(x, logn, mulmod(ps, ps, qi), qi);
        uint64_t* y = (uint64_t*)malloc(sizeof(uint64_t) * n);
        for (uint32_t s = 0; s < n; s++) y[s] = x[brv(s, logn)];
        memcpy(x, y, sizeof(uint64_t) * n);
        free(y);
    }
}

/* Inverse of orc_ntt: undo the bit-reversed order, inverse cyclic DFT with
 * w^-1 and 1/N, then untwist by psi^-t. */
void orc_intt(uint64_t* a, int nl, int logn, const uint64_t* q, const uint64_t* psi) {
    const uint32_t n = 1u << logn;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < nl; i++) {
        uint64_t* x = a + (size_t)i * n;
        const uint64_t qi = q[i];
        const uint64_t psi_inv = powmod(psi[i], 2 * (uint64_t)n - 1, qi);
        uint64_t* y = (uint64_t*)malloc(sizeof(uint64_t) * n);
        for (uint32_t s = 0; s < n; s++) y[brv(s, logn)] = x[s];
        cyclic_dft(y, logn, mulmod(psi_inv, psi_inv, qi), qi);
        const uint64_t n_inv = powmod(n % qi, qi - 2, qi);
        uint64_t pw = 1;
        for (uint32_t t = 0; t < n; t++) {
            x[t] = mulmod(mulmod(y[t], n_inv, qi), pw, qi);
            pw = mulmod(pw, psi_inv, qi);
        }
        free(y);
    }
}

/* out = a * b coefficient-wise (PE mode CWPM, Sec. V). */
void orc_mul(const uint64_t* a, const uint64_t* b, uint64_t* out, int nl, int n, const uint64_t* q) {
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (int t = 0; t < n; t++) {
            size_t o = (size_t)i * n + t;
            out[o] = mulmod(a[o], b[o], q[i]);
        }
}

/* out = a + b, a - b. */
void orc_add(const uint64_t* a, const uint64_t* b, uint64_t* out, int nl, int n, const uint64_t* q) {
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (int t = 0; t < n; t++) {
            size_t o = (size_t)i * n + t;
            out[o] = addmod(a[o], b[o], q[i]);
        }
}
void orc_sub(const uint64_t* a, const uint64_t* b, uint64_t* out, int nl, int n, const uint64_t* q) {
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (int t = 0; t < n; t++) {
            size_t o = (size_t)i * n + t;
            out[o] = submod(a[o], b[o], q[i]);
        }
}

/* out = c[i] * a, one constant per limb (PE mode CM). */
void orc_mul_const(const uint64_t* a, const uint64_t* c, uint64_t* out, int nl, int n, const uint64_t* q) {
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (int t = 0; t < n; t++) {
            size_t o = (size_t)i * n + t;
            out[o] = mulmod(a[o], c[i] % q[i], q[i]);
        }
}

/* Fast basis conversion, Eq. (3): given y_j = [a^(j) * qhat_j^-1]_{q_j} for the
 * nsrc source moduli, out^(t) = sum_j y_j * [qhat_j]_{t} mod t for each target.
 * qhat_mod_t is [ntgt][nsrc]. */
void orc_bconv(const uint64_t* y, int nsrc, const uint64_t* qhat_mod_t, uint64_t* out, int ntgt,
               int n, const uint64_t* t_mod) {
#pragma omp parallel for
    for (int i = 0; i < ntgt; i++) {
        const uint64_t t = t_mod[i];
        for (int c = 0; c < n; c++) {
            uint64_t s = 0;
            for (int j = 0; j < nsrc; j++)
                s = addmod(s, mulmod(y[(size_t)j * n + c] % t, qhat_mod_t[(size_t)i * nsrc + j] % t, t), t);
            out[(size_t)i * n + c] = s;
        }
    }
}

/* Automorphism phi_g in the coefficient domain, Eq. (2): a(x) -> a(x^g) mod x^N+1.
 * Coefficient t moves to t*g mod 2N and changes sign when that is >= N. */
void orc_auto_coeff(const uint64_t* a, uint64_t* out, int nl, int logn, uint64_t g, const uint64_t* q) {
    const uint64_t n = 1ull << logn;
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (uint64_t t = 0; t < n; t++) {
            uint64_t pos = (t * g) % (2 * n);
            uint64_t v = a[(size_t)i * n + t];
            if (pos < n) out[(size_t)i * n + pos] = v;
            else out[(size_t)i * n + pos - n] = (q[i] - v) % q[i];
        }
}

/* Automorphism phi_g in the NTT domain, Eq. (7), bit-reversed layout.
 * (phi_g a)(psi^(2l+1)) = a(psi^(g(2l+1))), so evaluation point l takes the
 * value of point l' = ((g(2l+1) mod 2N) - 1)/2: a gather. */
void orc_auto_ntt(const uint64_t* a, uint64_t* out, int nl, int logn, uint64_t g) {
    const uint64_t n = 1ull << logn;
#pragma omp parallel for
    for (int i = 0; i < nl; i++)
        for (uint64_t s = 0; s < n; s++) {
            uint64_t l = brv((uint32_t)s, logn);
            uint64_t lp = (((g % (2 * n)) * (2 * l + 1)) % (2 * n) - 1) / 2;
            out[(size_t)i * n + s] = a[(size_t)i * n + brv((uint32_t)lp, logn)];
        }
}
