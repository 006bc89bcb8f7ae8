// Key-switching inner product (K4) and plaintext-diagonal multiply-accumulate
// (K6) kernels, sm_103a.
//
// Both kernels read their ring elements in the NTT domain with the hoisted
// automorphism fused in as an index gather: Algorithms 1-2 rotate the
// switching key, swk~_r = phi_{-r}(swk_r), and apply phi_r after the inner
// product; since phi_r is a pure permutation of NTT-domain words,
//     phi_r(x + <d, phi_{-r}(swk)>) = phi_r(x) + <phi_r(d), swk>
// holds word for word, so the standard key is streamed once, in order, and
// the digits are gathered.  In bit-reversed storage the gather maps every
// aligned run of 32 words onto one aligned run of 32 words (Eq. 8), so a
// warp's gathered load touches exactly the same 256 bytes as a plain load.
//
// Sums of products stay in 128-bit accumulators (mad.lo.cc / madc.hi) and are
// reduced once (PE modes CWPM-ACC / CM-ACC of Sec. V, done lazily).
#include "kernels.h"

namespace ckks {
namespace {

constexpr int THREADS = 256;

// ------------------------------------------------------------------ K4
__global__ void __launch_bounds__(THREADS) k_ks_inner(const __grid_constant__ KsArgs a) {
    const u32 N = 1u << a.log_n;
    const u32 s = blockIdx.x * THREADS + threadIdx.x;
    const u32 t = blockIdx.y;
    if (s >= N) return;
    const u32 kp = a.ext - a.level;
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const ModC m = a.mods[gmod];
    const u32 src = a.gal ? auto_src(s, a.gal, a.log_n) : s;
    const size_t key_b = 2ull * (a.L + kp) * N;
    U128 acc0{0, 0}, acc1{0, 0};
    for (u32 b = 0; b < a.beta; b++) {
        const u64 d = a.digits[((size_t)b * a.ext + t) * N + src];
        const u64* kb = a.key + b * key_b + (size_t)gmod * N + s;
        mac128(acc0, d, kb[0]);
        mac128(acc1, d, kb[(size_t)(a.L + kp) * N]);
    }
    if (a.x0_mode == 1) {
        add128(acc0, a.x0[(size_t)t * N + src]);
    } else if (a.x0_mode == 2 && t < a.level) {
        add128(acc0, mul_shoup(a.x0[(size_t)t * N + src], a.lift_c[gmod], a.lift_sh[gmod], m.q));
    }
    u64 r0 = reduce128(acc0, m), r1 = reduce128(acc1, m);
    const size_t o = (size_t)t * N + s;
    if (a.accumulate) {
        r0 = add_mod(r0, a.out0[o], m.q);
        r1 = add_mod(r1, a.out1[o], m.q);
    }
    a.out0[o] = r0;
    a.out1[o] = r1;
}

// ------------------------------------------------------------------ K6
// For one word s of limb t and K3 giant indices k (a chunk of the n3 outer
// rotations) this computes
//   U_{c,k}[s] = sum_{j < n2} sum_{i < n1} pair_c(i, j)[s] * f_{n1 n2 k + n1 j + i}[h_k(s)]
// where h_k is the gather of phi_{-n1 n2 k} (the pre-rotated diagonal
// f^ = phi_{-n1 n2 k}(f), Alg. 2 input) and
//   pair(i, 0) = (A_i, B_i)                                    (Alg. 2 lines 2-5)
//   pair(i, j) = phi_{n1 j}(A_i + <D_i, swk~_0>, <D_i, swk~_1>) (Alg. 2 lines 9-10)
// so Alg. 2 lines 8-14 (Phases 3 and 4 of Sec. IV) run without writing the
// n1*n2 rotated ciphertexts to HBM.  DH-BSGS is the case n2 = 1, the diagonal
// method n1 = 1, BSGS n2 = 1 over Q only.
constexpr int MAXB = 8;  // digits handled unrolled; larger beta runs a plain loop

template <int K3>
__global__ void __launch_bounds__(THREADS, 2) k_diag_mac(const __grid_constant__ DiagMacArgs a) {
    // this giant index's switching-key words for the thread's own position,
    // parked in thread-private shared-memory slots (no barrier needed)
    __shared__ u64 skey[2 * MAXB * THREADS];
    const u32 N = 1u << a.log_n;
    const u32 s = blockIdx.x * THREADS + threadIdx.x;
    const u32 t = blockIdx.y;
    if (s >= N) return;
    const u32 k_first = blockIdx.z * K3;
    const u32 k_count = min((u32)K3, a.n3 - k_first);
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const u32 drow = t < a.level ? t : a.diag_level + (t - a.level);
    const ModC m = a.mods[gmod];
    const size_t dstride = (size_t)(a.diag_level + a.k_p) * N;
    const size_t key_b = 2ull * (a.L + a.k_p) * N;
    const size_t key_c = (size_t)(a.L + a.k_p) * N;
    const size_t dig_b = (size_t)a.ext * N;
    const size_t tN = (size_t)t * N;
    const u32 n1n2 = a.n1 * a.n2;
    const bool lift_limb = a.lift0 && t < a.level;
    const u64 lc = lift_limb ? a.lift_c[gmod] : 0, lsh = lift_limb ? a.lift_sh[gmod] : 0;
    const u32 beta = a.beta;
    const bool small_beta = beta <= MAXB;
    u64* sk = skey + threadIdx.x;

    const u64* fb[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        const u32 kc = k_first + min((u32)kk, k_count - 1);  // lanes past the chunk mirror its last index
        const u32 g = a.gal_diag[kc];
        fb[kk] = a.diags + (size_t)(n1n2 * kc) * dstride + (size_t)drow * N + (g ? auto_src(s, g, a.log_n) : s);
    }
    U128 acc0[K3], acc1[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) acc0[kk] = acc1[kk] = U128{0, 0};
    u32 terms = 0;

    for (u32 j = 0; j < a.n2; j++) {
        const u32 src = j ? auto_src(s, a.gal_mid[j], a.log_n) : s;
        const u64* key = j ? a.keys[j] + (size_t)gmod * N + s : nullptr;
        if (j && small_beta) {
#pragma unroll
            for (int b = 0; b < MAXB; b++) {
                if (b < (int)beta) {
                    sk[(2 * b) * THREADS] = key[b * key_b];
                    sk[(2 * b + 1) * THREADS] = key[b * key_b + key_c];
                }
            }
        }
        for (u32 i = 0; i < a.n1; i++) {
            const bool lifted = (i == 0) && a.lift0;
            // issue every independent load of this (i, j) before any arithmetic
            const size_t didx = (size_t)(a.n1 * j + i) * dstride;
            u64 f[K3];
#pragma unroll
            for (int kk = 0; kk < K3; kk++) f[kk] = kk < (int)k_count ? fb[kk][didx] : 0;
            u64 av, bv;
            if (j == 0) {
                if (lifted) {
                    av = lift_limb ? mul_shoup(a.A[0][tN + s], lc, lsh, m.q) : 0;
                    bv = lift_limb ? mul_shoup(a.B[0][tN + s], lc, lsh, m.q) : 0;
                } else {
                    av = a.A[i][tN + s];
                    bv = a.B[i][tN + s];
                }
            } else {
                const u64* D = a.Dg[i] + tN + src;
                const u64 xa = (!lifted || lift_limb) ? a.A[i][tN + src] : 0;
                U128 x0{0, 0}, x1{0, 0};
                if (small_beta) {
                    u64 d[MAXB];
#pragma unroll
                    for (int b = 0; b < MAXB; b++) d[b] = b < (int)beta ? D[b * dig_b] : 0;
#pragma unroll
                    for (int b = 0; b < MAXB; b++) {
                        if (b < (int)beta) {
                            mac128(x0, d[b], sk[(2 * b) * THREADS]);
                            mac128(x1, d[b], sk[(2 * b + 1) * THREADS]);
                        }
                    }
                } else {
                    for (u32 b = 0; b < beta; b++) {
                        const u64 dv = D[b * dig_b];
                        mac128(x0, dv, key[b * key_b]);
                        mac128(x1, dv, key[b * key_b + key_c]);
                    }
                }
                add128(x0, lifted ? mul_shoup(xa, lc, lsh, m.q) : xa);
                av = reduce128(x0, m);
                bv = reduce128(x1, m);
            }
#pragma unroll
            for (int kk = 0; kk < K3; kk++) {
                if (kk < (int)k_count) {
                    mac128(acc0[kk], av, f[kk]);
                    mac128(acc1[kk], bv, f[kk]);
                }
            }
            if (++terms == 128) {
                terms = 0;
#pragma unroll
                for (int kk = 0; kk < K3; kk++) {
                    acc0[kk] = U128{reduce128(acc0[kk], m), 0};
                    acc1[kk] = U128{reduce128(acc1[kk], m), 0};
                }
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        if (kk < (int)k_count) {
            a.U0[k_first + kk][tN + s] = reduce128(acc0[kk], m);
            a.U1[k_first + kk][tN + s] = reduce128(acc1[kk], m);
        }
    }
}

}  // namespace

void launch_ks_inner(const KsArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    ProfScope ps(K_KS_INNER, st);
    k_ks_inner<<<dim3((N + THREADS - 1) / THREADS, a.ext), THREADS, 0, st>>>(a);
    count_launch();
}

void launch_diag_mac(const DiagMacArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    u32 k3 = 1;
    while (k3 < a.n3 && k3 < (u32)DM_MAX_K3) k3 *= 2;
    const dim3 grid((N + THREADS - 1) / THREADS, a.ext, (a.n3 + k3 - 1) / k3);
    ProfScope ps(K_DIAG_MAC, st);
    switch (k3) {
        case 1: k_diag_mac<1><<<grid, THREADS, 0, st>>>(a); break;
        case 2: k_diag_mac<2><<<grid, THREADS, 0, st>>>(a); break;
        case 4: k_diag_mac<4><<<grid, THREADS, 0, st>>>(a); break;
        default: k_diag_mac<8><<<grid, THREADS, 0, st>>>(a); break;
    }
    count_launch();
}

}  // namespace ckks
