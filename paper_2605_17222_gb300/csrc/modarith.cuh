// Modular arithmetic on uint64 RNS residues for sm_103a.
//
// The paper's PE modes (Sec. V: CM, CWPM, CM-ACC, CWPM-ACC, CWPA-CM) all reduce
// to three device primitives here:
//   * Shoup multiplication by a constant w with precomputed w' = floor(w 2^64 / q)
//     (twiddles, per-limb constants);
//   * a lazy 128-bit multiply-accumulate (mad.lo.cc / madc.hi), reduced once
//     at the end of an inner product;
//   * Barrett reduction of a 128-bit value with mu = floor(2^128 / q).
// Every modulus is below 2^60, so a product is below 2^120 and up to 256
// products fit one 128-bit accumulator.  Outputs are canonical in [0, q).
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef uint32_t u32;

struct ModC {
    u64 q;
    u64 mu_hi;  // floor(2^128 / q) >> 64
    u64 mu_lo;  // floor(2^128 / q) mod 2^64
};

struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}

// a * w mod q for w < q, wp = floor(w * 2^64 / q); valid for any a < 2^64 and q < 2^63.
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wp, u64 q) {
    u64 t = __umul64hi(a, wp);
    u64 r = a * w - t * q;
    return r >= q ? r - q : r;
}

// acc += a * b.  The four 32x32 partial products are added into the four
// 32-bit words of the accumulator along explicit carry chains: ten 32-bit
// multiply-add instructions, cheaper than the 64-bit mad.lo/madc.hi forms.
// The caller keeps the 128-bit sum from overflowing.
__device__ __forceinline__ void mac128(U128& acc, u64 a, u64 b) {
    asm("{\n\t.reg .u32 a0, a1, a2, a3, x0, x1, y0, y1;\n\t"
        "mov.b64 {a0, a1}, %0;\n\t"
        "mov.b64 {a2, a3}, %1;\n\t"
        "mov.b64 {x0, x1}, %2;\n\t"
        "mov.b64 {y0, y1}, %3;\n\t"
        "mad.lo.cc.u32 a0, x0, y0, a0;\n\t"
        "madc.hi.cc.u32 a1, x0, y0, a1;\n\t"
        "madc.lo.cc.u32 a2, x1, y1, a2;\n\t"
        "madc.hi.u32 a3, x1, y1, a3;\n\t"
        "mad.lo.cc.u32 a1, x0, y1, a1;\n\t"
        "madc.hi.cc.u32 a2, x0, y1, a2;\n\t"
        "addc.u32 a3, a3, 0;\n\t"
        "mad.lo.cc.u32 a1, x1, y0, a1;\n\t"
        "madc.hi.cc.u32 a2, x1, y0, a2;\n\t"
        "addc.u32 a3, a3, 0;\n\t"
        "mov.b64 %0, {a0, a1};\n\t"
        "mov.b64 %1, {a2, a3};\n\t}"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(a), "l"(b));
}

// A 96-bit accumulator (low 64 bits, high 32 bits) for products of operands
// below 2^41.
struct U96 {
    u64 lo;
    u32 hi;
};

// acc += a * b for a, b < 2^41; the caller keeps the sum below 2^96.  With
// a = a1 2^32 + a0 and b = b1 2^32 + b0 (a1, b1 < 2^9), a1 b1 is below 2^18
// and the high halves of a0 b1 and a1 b0 below 2^9, so the top word takes
// them with no carry out of it: seven 32-bit multiply-adds along three short
// carry chains instead of mac128's ten.
__device__ __forceinline__ void mac96(U96& acc, u64 a, u64 b) {
    asm("{\n\t.reg .u32 w0, w1, x0, x1, y0, y1;\n\t"
        "mov.b64 {w0, w1}, %0;\n\t"
        "mov.b64 {x0, x1}, %2;\n\t"
        "mov.b64 {y0, y1}, %3;\n\t"
        "mad.lo.cc.u32 w0, x0, y0, w0;\n\t"
        "madc.hi.cc.u32 w1, x0, y0, w1;\n\t"
        "madc.lo.u32 %1, x1, y1, %1;\n\t"
        "mad.lo.cc.u32 w1, x0, y1, w1;\n\t"
        "madc.hi.u32 %1, x0, y1, %1;\n\t"
        "mad.lo.cc.u32 w1, x1, y0, w1;\n\t"
        "madc.hi.u32 %1, x1, y0, %1;\n\t"
        "mov.b64 %0, {w0, w1};\n\t}"
        : "+l"(acc.lo), "+r"(acc.hi)
        : "l"(a), "l"(b));
}

__device__ __forceinline__ void add96(U96& acc, u64 v) {
    asm("{\n\t.reg .u32 w0, w1, v0, v1;\n\t"
        "mov.b64 {w0, w1}, %0;\n\t"
        "mov.b64 {v0, v1}, %2;\n\t"
        "add.cc.u32 w0, w0, v0;\n\t"
        "addc.cc.u32 w1, w1, v1;\n\t"
        "addc.u32 %1, %1, 0;\n\t"
        "mov.b64 %0, {w0, w1};\n\t}"
        : "+l"(acc.lo), "+r"(acc.hi)
        : "l"(v));
}

__device__ __forceinline__ void add128(U128& acc, u64 v) {
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, 0;"
        : "+l"(acc.lo), "+l"(acc.hi)
        : "l"(v));
}

// x mod q for any 128-bit x (q < 2^62).  The quotient estimate
//   qe = x1*m1 + hi(x1*m0) + hi(x0*m1)            (mod 2^64)
// drops the low partial products, so it is below floor(x/q) by at most 3 and
// x - qe*q < 4q fits 64 bits.
__device__ __forceinline__ u64 reduce128_lazy(U128 x, const ModC& m) {  // x mod q up to 3q, in [0, 4q)
    const u64 qe = x.hi * m.mu_hi + __umul64hi(x.hi, m.mu_lo) + __umul64hi(x.lo, m.mu_hi);
    return x.lo - qe * m.q;
}
__device__ __forceinline__ u64 reduce128(U128 x, const ModC& m) {
    u64 r = reduce128_lazy(x, m);
    r = r >= 2 * m.q ? r - 2 * m.q : r;
    r = r >= m.q ? r - m.q : r;
    return r;
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModC& m) {
    U128 p{a * b, __umul64hi(a, b)};
    return reduce128(p, m);
}

// Source index of the NTT-domain automorphism x -> x^g in bit-reversed
// storage (Eq. 7): output word s reads word brv(((g (2 brv(s) + 1)) mod 2N - 1) / 2).
// 2N divides 2^32, so the product may wrap.
__device__ __forceinline__ u32 auto_src(u32 s, u32 g, u32 log_n) {
    const u32 sh = 32u - log_n;
    u32 l = __brev(s) >> sh;
    u32 e = (g * (2u * l + 1u)) & ((2u << log_n) - 1u);
    return __brev((e - 1u) >> 1) >> sh;
}
