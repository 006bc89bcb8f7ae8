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

#include <algorithm>
#include <atomic>
#include <cstdlib>

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
    const size_t plane = (size_t)(a.L + kp) * N;  // key words per digit (interleaved components)
    U128 acc0{0, 0}, acc1{0, 0};
    for (u32 b = 0; b < a.beta; b++) {
        const u64 d = a.digits[((size_t)b * a.ext + t) * N + src];
        const ulonglong2 kv = ((const ulonglong2*)a.key)[b * plane + (size_t)gmod * N + s];
        mac128(acc0, d, kv.x);
        mac128(acc1, d, kv.y);
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

// ------------------------------------------------------------------ K4, all giant indices at once
__global__ void __launch_bounds__(THREADS) k_ks_multi(const __grid_constant__ KsMultiArgs a) {
    const u32 N = 1u << a.log_n;
    const u32 s = blockIdx.x * THREADS + threadIdx.x;
    const u32 t = blockIdx.y;
    if (s >= N) return;
    const u32 kp = a.ext - a.level;
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const ModC m = a.mods[gmod];
    const size_t plane = (size_t)(a.L + kp) * N;  // key words per digit (interleaved components)
    const size_t o = (size_t)t * N + s;
    U128 acc0{a.out0[o], 0}, acc1{a.out1[o], 0};
    for (u32 k = 0; k < a.count; k++) {
        const u32 src = auto_src(s, a.gal[k], a.log_n);
        const u64* D = a.digits[k] + (size_t)t * N + src;
        const ulonglong2* K = (const ulonglong2*)a.keys[k] + (size_t)gmod * N + s;
        add128(acc0, a.x0[k][(size_t)t * N + src]);
        for (u32 b = 0; b < a.beta; b++) {
            const u64 d = D[(size_t)b * a.ext * N];
            const ulonglong2 kv = K[b * plane];
            mac128(acc0, d, kv.x);
            mac128(acc1, d, kv.y);
        }
        // keep the running sums bounded: one partial reduction per giant index
        acc0 = U128{reduce128_lazy(acc0, m), 0};
        acc1 = U128{reduce128_lazy(acc1, m), 0};
    }
    a.out0[o] = reduce128(acc0, m);
    a.out1[o] = reduce128(acc1, m);
}

// ------------------------------------------------------------------ K4, many independent products
__global__ void __launch_bounds__(THREADS) k_ks_batch(const __grid_constant__ KsBatchArgs a) {
    const u32 N = 1u << a.log_n;
    const KsBatchEntry& E = a.e[blockIdx.x % a.count];
    const u32 s = (blockIdx.x / a.count) * THREADS + threadIdx.x;
    const u32 t = blockIdx.y;
    if (s >= N) return;
    const u32 kp = a.ext - a.level;
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const ModC m = a.mods[gmod];
    const u32 src = E.gal ? auto_src(s, E.gal, a.log_n) : s;
    const size_t plane = (size_t)(a.L + kp) * N;  // key words per digit (interleaved components)
    U128 acc0{0, 0}, acc1{0, 0};
    for (u32 b = 0; b < a.beta; b++) {
        const u64 d = E.digits[((size_t)b * a.ext + t) * N + src];
        const ulonglong2 kv = ((const ulonglong2*)E.key)[b * plane + (size_t)gmod * N + s];
        mac128(acc0, d, kv.x);
        mac128(acc1, d, kv.y);
    }
    if (t < a.level) add128(acc0, mul_shoup(E.x0[(size_t)t * N + src], a.lift_c[gmod], a.lift_sh[gmod], m.q));
    const size_t o = (size_t)t * N + s;
    E.out0[o] = reduce128(acc0, m);
    E.out1[o] = reduce128(acc1, m);
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
    const u32 bidx = blockIdx.x % a.batch;
    const u32 s = (blockIdx.x / a.batch) * THREADS + threadIdx.x;
    const size_t oab = bidx * a.bs_ab, odg = bidx * a.bs_dg, ou = bidx * a.bs_u;
    const u64* A0 = a.lift0 ? a.c0[bidx] : a.A[0];
    const u64* B0 = a.lift0 ? a.c1[bidx] : a.B[0];
    const u32 t = blockIdx.y;
    if (s >= N) return;
    const u32 k_first = blockIdx.z * K3;
    const u32 k_count = min((u32)K3, a.n3 - k_first);
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const u32 drow = t < a.level ? t : a.diag_level + (t - a.level);
    const ModC m = a.mods[gmod];
    const size_t dstride = (size_t)(a.diag_level + a.k_p) * N;
    const size_t plane = (size_t)(a.L + a.k_p) * N;  // key words per digit (interleaved components)
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
        const ulonglong2* key = j ? (const ulonglong2*)a.keys[j] + (size_t)gmod * N + s : nullptr;
        if (j && small_beta) {
#pragma unroll
            for (int b = 0; b < MAXB; b++) {
                if (b < (int)beta) {
                    const ulonglong2 kv = key[b * plane];
                    sk[(2 * b) * THREADS] = kv.x;
                    sk[(2 * b + 1) * THREADS] = kv.y;
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
                    av = lift_limb ? mul_shoup(A0[tN + s], lc, lsh, m.q) : 0;
                    bv = lift_limb ? mul_shoup(B0[tN + s], lc, lsh, m.q) : 0;
                } else {
                    av = (i ? a.A[i] + oab : A0)[tN + s];
                    bv = (i ? a.B[i] + oab : B0)[tN + s];
                }
            } else {
                const u64* D = a.Dg[i] + odg + tN + src;
                const u64 xa = (!lifted || lift_limb) ? (i ? a.A[i] + oab : A0)[tN + src] : 0;
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
                        const ulonglong2 kv = key[b * plane];
                        mac128(x0, dv, kv.x);
                        mac128(x1, dv, kv.y);
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
            a.U0[k_first + kk][ou + tN + s] = reduce128(acc0[kk], m);
            a.U1[k_first + kk][ou + tN + s] = reduce128(acc1[kk], m);
        }
    }
}

// ------------------------------------------------------------------ K6, staged through shared memory by TMA
// Same computation as k_diag_mac, organised around Eq. (8): in bit-reversed
// storage every automorphism maps an aligned run of RUN words onto one
// aligned run of RUN words.  A CTA owns one run of RUN positions of limb t, so
// every operand of one (i, j) step is a handful of contiguous RUN-word source
// runs: K3 diagonal runs, beta digit runs and the A run (B too at j = 0), plus
// 2*beta key runs per giant index j.  One thread copies them into shared
// memory with bulk (TMA) copies, cp.async.bulk, completing on an mbarrier, one
// step ahead of the computation (ring of DM_NS stage buffers; keys
// double-buffered by the parity of j).  The CTA then computes the step from
// shared memory, applying the in-run permutation.
//
// Every wait is bounded.  A wait that gives up sets *a.err and the whole CTA
// leaves the loop together (the decision goes through __syncthreads_or); the
// producer then waits, bounded again, for the copies it has in flight before
// the CTA exits.
constexpr u64 DM_WAIT_NS = 1000000000ull;              // a wait gives up after 1 s

__device__ __forceinline__ u64 global_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, u32 parity, u64 limit_ns = DM_WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const u64 t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int K3, int RUN, int NS, int KB>
__global__ void __launch_bounds__(RUN, 1) k_diag_mac_staged(const __grid_constant__ DiagMacArgs a) {
    extern __shared__ __align__(128) u64 smem[];
    __shared__ __align__(8) u64 full_bar[NS];
    const u32 N = 1u << a.log_n;
    const u32 l = threadIdx.x;
    const u32 bidx = blockIdx.x % a.batch;
    const u32 run = blockIdx.x / a.batch;
    const u32 s = run * RUN + l;
    const size_t oab = bidx * a.bs_ab, odg = bidx * a.bs_dg, ou = bidx * a.bs_u;
    const u64* A0 = a.lift0 ? a.c0[bidx] : a.A[0];
    const u64* B0 = a.lift0 ? a.c1[bidx] : a.B[0];
    const u32 t = blockIdx.y;
    const u32 k_first = blockIdx.z * K3;
    const u32 k_count = min((u32)K3, a.n3 - k_first);
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const u32 drow = t < a.level ? t : a.diag_level + (t - a.level);
    const ModC m = a.mods[gmod];
    const size_t dstride = (size_t)(a.diag_level + a.k_p) * N;
    const size_t plane = (size_t)(a.L + a.k_p) * N;  // key words per digit (interleaved components)
    const size_t dig_b = (size_t)a.ext * N;
    const size_t tN = (size_t)t * N;
    const u32 n1 = a.n1, n2 = a.n2, n1n2 = n1 * n2;
    const u32 beta = n2 > 1 ? a.beta : 0;  // <= KB (host checks)
    const bool lift_limb = a.lift0 && t < a.level;
    const u64 lc = lift_limb ? a.lift_c[gmod] : 0, lsh = lift_limb ? a.lift_sh[gmod] : 0;
    constexpr u32 RB = RUN * 8;  // bytes per run
    const bool fold = m.q < (1ull << 41) && beta <= 8;
    const u64 c63 = fold ? (1ull << 63) % m.q : 0, c64 = fold ? (0 - m.q) % m.q : 0;  // 2^63, 2^64 mod q

    // shared memory: NS stages of [K3 diag | beta digit | A | B] runs
    const u32 stage_runs = K3 + beta + 2;

    // per-thread in-run positions of the diagonal gathers (constant over the loop)
    u32 pd[K3];
    u32 hrun[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        const u32 kc = k_first + min((u32)kk, k_count - 1);
        const u32 g = a.gal_diag[kc];
        const u32 base = g ? auto_src(run * RUN, g, a.log_n) : run * RUN;
        hrun[kk] = base / RUN;
        pd[kk] = (g ? auto_src(s, g, a.log_n) : s) - hrun[kk] * RUN;
    }

    // Producer (thread 0): copies of step `it` = j * n1 + i into stage it % NS.
    // Runs, in order: k_count diagonal runs; at j = 0 the A and B runs; at j > 0
    // the beta digit runs and the A run.  A and B are skipped for the lifted
    // ciphertext on P limbs (zero words).
    // source run of the middle-layer gather for every j (Eq. 8 maps an aligned
    // run onto one aligned run), computed once by the whole CTA
    u32* srun_of = (u32*)(smem + (size_t)NS * stage_runs * RUN);
    for (u32 jj = l; jj < n2; jj += RUN) srun_of[jj] = jj ? auto_src(run * RUN, a.gal_mid[jj], a.log_n) / RUN : run;

    auto issue = [&](u32 it) {
        if (it >= n1n2 || it == a.starve_step) return;
        const u32 j = n1 == 1 ? it : it / n1, i = n1 == 1 ? 0u : it % n1;
        u64* st = smem + (size_t)(it % NS) * stage_runs * RUN;
        u64* bar = &full_bar[it % NS];
        const bool lifted = (i == 0) && a.lift0;
        const bool copy_a = !lifted || lift_limb;
        const u32 srun = srun_of[j];
        const u32 n_ab = j == 0 ? (copy_a ? 2u : 0u) : (copy_a ? 1u : 0u);
        const u32 n_dig = j == 0 ? 0u : beta;
        mbar_expect_tx(bar, (k_count + n_dig + n_ab) * RB);
        const size_t didx = (size_t)(n1 * j + i) * dstride + (size_t)drow * N;
#pragma unroll
        for (int kk = 0; kk < K3; kk++)
            if (kk < (int)k_count)
                tma_load_1d(st + (size_t)kk * RUN,
                            a.diags + (size_t)(n1n2 * (k_first + kk)) * dstride + didx + (size_t)hrun[kk] * RUN, RB,
                            bar);
        for (u32 b = 0; b < n_dig; b++)
            tma_load_1d(st + (size_t)(K3 + b) * RUN, a.Dg[i] + odg + b * dig_b + tN + (size_t)srun * RUN, RB, bar);
        const u64* Ai = i ? a.A[i] + oab : A0;
        const u64* Bi = i ? a.B[i] + oab : B0;
        if (n_ab >= 1) tma_load_1d(st + (size_t)(K3 + beta) * RUN, Ai + tN + (size_t)srun * RUN, RB, bar);
        if (n_ab == 2) tma_load_1d(st + (size_t)(K3 + beta + 1) * RUN, Bi + tN + (size_t)srun * RUN, RB, bar);
    };

    if (l == 0) {
#pragma unroll
        for (int b = 0; b < NS; b++) mbar_init(&full_bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (l == 0)
        for (int p = 0; p < NS - 1; p++) issue(p);

    U128 acc0[K3], acc1[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) acc0[kk] = acc1[kk] = U128{0, 0};
    u32 terms = 0;
    u32 issued = NS - 1;  // steps the producer has issued (meaningful in thread 0)
    u32 failed_at = n1n2;  // the step whose wait gave up (n1n2: none)
    const u64 wait_ns = a.wait_ns ? a.wait_ns : DM_WAIT_NS;
    u64 k0[KB], k1[KB];  // switching-key words of the current giant index at this thread's position
    u32 pm = 0;          // in-run source position of the middle-layer gather of the current j

    for (u32 it = 0; it < n1n2; it++) {
        const u32 j = n1 == 1 ? it : it / n1, i = n1 == 1 ? 0u : it % n1;
        if (j > 0 && i == 0) {
            // a new giant index: its key words (not gathered) come straight from
            // global memory; the loads overlap the wait for the stage below
            const ulonglong2* ks = (const ulonglong2*)a.keys[j] + (size_t)gmod * N + s;
#pragma unroll
            for (int b = 0; b < KB; b++) {
                const ulonglong2 kv = b < (int)beta ? ks[b * plane] : make_ulonglong2(0, 0);
                k0[b] = kv.x;
                k1[b] = kv.y;
            }
            pm = auto_src(s, a.gal_mid[j], a.log_n) % RUN;
        }
        const bool ok = mbar_wait_bounded(&full_bar[it % NS], (it / NS) & 1, wait_ns);
        // everyone has finished step it-1 (its buffer is free) and agrees on success
        if (__syncthreads_or(!ok)) {
            failed_at = it;
            break;
        }
        if (l == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(it + NS - 1);
            issued = it + NS;
        }
        const u64* st = smem + (size_t)(it % NS) * stage_runs * RUN;
        const bool lifted = (i == 0) && a.lift0;
        u64 av, bv;
        if (j == 0) {
            if (lifted) {
                av = lift_limb ? mul_shoup(st[(K3 + beta) * RUN + l], lc, lsh, m.q) : 0;
                bv = lift_limb ? mul_shoup(st[(K3 + beta + 1) * RUN + l], lc, lsh, m.q) : 0;
            } else {
                av = st[(K3 + beta) * RUN + l];
                bv = st[(K3 + beta + 1) * RUN + l];
            }
        } else {
            U128 x0{0, 0}, x1{0, 0};
#pragma unroll
            for (int b = 0; b < KB; b++) {
                if (b < (int)beta) {
                    const u64 d = st[(K3 + b) * RUN + pm];
                    mac128(x0, d, k0[b]);
                    mac128(x1, d, k1[b]);
                }
            }
            if (lifted) {
                if (lift_limb) add128(x0, mul_shoup(st[(K3 + beta) * RUN + pm], lc, lsh, m.q));
            } else {
                add128(x0, st[(K3 + beta) * RUN + pm]);
            }
            // partial reductions are enough to feed the products: below 4q < 2^62
            // in general; for q < 2^41 (and beta <= 8, so x < 2^85) a fold
            //   (x mod 2^63) + [bit 63] (2^63 mod q) + x_hi (2^64 mod q)  <  2^64
            // is congruent to x, and 64 of its products with a word below q stay
            // below 2^128 in the accumulators
            if (fold) {
                av = (x0.lo & ~(1ull << 63)) + ((x0.lo >> 63) ? c63 : 0) + x0.hi * c64;
                bv = (x1.lo & ~(1ull << 63)) + ((x1.lo >> 63) ? c63 : 0) + x1.hi * c64;
            } else {
                av = reduce128_lazy(x0, m);
                bv = reduce128_lazy(x1, m);
            }
        }
#pragma unroll
        for (int kk = 0; kk < K3; kk++) {
            if (kk < (int)k_count) {
                const u64 f = st[kk * RUN + pd[kk]];
                mac128(acc0[kk], av, f);
                mac128(acc1[kk], bv, f);
            }
        }
        if (++terms == 64) {  // 64 products below 2^122 each fit the accumulators
            terms = 0;
#pragma unroll
            for (int kk = 0; kk < K3; kk++) {
                acc0[kk] = U128{reduce128(acc0[kk], m), 0};
                acc1[kk] = U128{reduce128(acc1[kk], m), 0};
            }
        }
    }
    if (failed_at < n1n2) {
        // drain: the producer waits (bounded, default limit) for the steps it
        // issued that were not consumed, failed_at .. issued - 1.  Every step
        // before failed_at completed and was consumed; their stages have been
        // reused or never will be, so waiting on them would only run out.
        // A starved step has no copies in flight.
        if (l == 0) {
            for (u32 it = failed_at; it < min(issued, n1n2); it++)
                if (it != a.starve_step) mbar_wait_bounded(&full_bar[it % NS], (it / NS) & 1);
            atomicExch(a.err, 1u);
        }
        return;
    }
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        if (kk < (int)k_count) {
            a.U0[k_first + kk][ou + tN + s] = reduce128(acc0[kk], m);
            a.U1[k_first + kk][ou + tN + s] = reduce128(acc1[kk], m);
        }
    }
}

// Failure-detection self-test: one thread waits on an mbarrier that nothing
// will complete, with the same bounded wait the staged kernels use (limit
// given in ns), and records the give-up in *err.
__global__ void k_wait_selftest(u32* err, u64 limit_ns) {
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const u64 t0 = global_ns();
    bool ok = false;
    while (!(ok = mbar_try_wait(&bar, 0)))
        if (global_ns() - t0 > limit_ns) break;
    if (!ok) atomicExch(err, 1u);
}

// ------------------------------------------------------------------ K6, warp-specialised
// The same computation again, with the copies issued by a warp of their own.
// A CTA has RUN compute threads (one position each) and one producer warp.
// Every operand of a step, the middle layer's switching-key runs included,
// arrives in a shared-memory stage by bulk copies; the ring has NS stages,
// ordered by two mbarriers per stage and no CTA-wide barrier in the loop:
//   full[s]  : the producer's expect_tx; the stage's copies complete it.
//   empty[s] : one arrival per compute warp once the warp has read the stage;
//              the producer waits on it before it refills the stage.
// A compute warp therefore never waits for another compute warp, and the
// producer never waits inside a compute warp's step.
//
// Every wait is bounded (compute: wait_ns, default 1 s; producer: 1 s) and
// also gives up as soon as the CTA's abort flag is raised.  A warp whose wait
// gives up raises the flag and leaves its loop (all its lanes together); the
// producer stops issuing.  Each thread then reaches one final named barrier
// exactly once; after it, if the flag is up, the producer waits (1 s limit)
// for the last copies it issued into each stage -- a stage is only refilled
// after every warp consumed it, so at most one phase of each full barrier is
// pending -- sets *err, and the CTA writes no output.
__device__ __forceinline__ void nbar_sync(u32 id, u32 count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(u64* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_abortable(u64* bar, u32 parity, u64 limit_ns, const volatile u32* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const u64 t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (*abort || global_ns() - t0 > limit_ns) return false;
    return true;
}

template <int K3, int RUN, int NS, int BETA>
struct WsLayout {
    // one stage, in words: K3 diagonal runs | BETA digit runs | A run | B run | BETA key runs (word pairs)
    static constexpr u32 OFF_DIG = K3 * RUN;
    static constexpr u32 OFF_A = (K3 + BETA) * RUN;
    static constexpr u32 OFF_B = OFF_A + RUN;
    static constexpr u32 OFF_KEY = OFF_B + RUN;
    static constexpr u32 STAGE = OFF_KEY + 2 * BETA * RUN;
    static constexpr size_t bytes(u32 n2) { return 8ull * STAGE * NS + ((4ull * n2 + 15) & ~15ull); }
};

// What the compute threads of k_diag_mac_ws share.
struct WsCtx {
    const DiagMacArgs& a;
    const u64* smem;
    u64* full_bar;
    u64* empty_bar;
    volatile u32* abort;
    u32 s, l, n1, n2, beta, k_first, k_count;
    size_t tN, ou;
    bool lift_limb, c0_lifted;
    u64 lc, lsh;
    ModC m;
};

template <bool SMALL>
struct WsAcc;
template <>
struct WsAcc<true> {  // operands below 2^41: three-word sums (mac96)
    U96 v;
    __device__ __forceinline__ void zero() { v = U96{0, 0}; }
    __device__ __forceinline__ void mac(u64 x, u64 y) { mac96(v, x, y); }
    __device__ __forceinline__ void add(u64 x) { add96(v, x); }
    __device__ __forceinline__ U128 wide() const { return U128{v.lo, v.hi}; }
    __device__ __forceinline__ void set(u64 x) { v = U96{x, 0}; }
};
template <>
struct WsAcc<false> {  // any residue below 2^60: four-word sums (mac128)
    U128 v;
    __device__ __forceinline__ void zero() { v = U128{0, 0}; }
    __device__ __forceinline__ void mac(u64 x, u64 y) { mac128(v, x, y); }
    __device__ __forceinline__ void add(u64 x) { add128(v, x); }
    __device__ __forceinline__ U128 wide() const { return v; }
    __device__ __forceinline__ void set(u64 x) { v = U128{x, 0}; }
};

// The compute threads' step loop of k_diag_mac_ws (see there) and the output.
// SMALL (2^32 < q < 2^41, beta <= 8): every operand is below 2^41, the
// middle-layer sum x = sum_b d_b k_b + A is below 2^85, and it is brought
// into [0, 3q) (a fold below 2^64, then a quotient estimate with the 32-bit
// mu = floor(2^64 / q)) so that 64 outer products with a word below q stay
// below 2^96: mac96 throughout.  Otherwise 128-bit sums, reduced lazily.
template <int K3, int RUN, int NS, int BETA, bool SMALL>
__device__ __forceinline__ void ws_compute(const WsCtx& c) {
    using LY = WsLayout<K3, RUN, NS, BETA>;
    constexpr u32 FULL = 0xffffffffu;
    const DiagMacArgs& a = c.a;
    const u32 l = c.l, s = c.s, n1 = c.n1, n2 = c.n2, n1n2 = n1 * n2, beta = c.beta;
    const ModC m = c.m;
    const u64 wait_ns = a.wait_ns ? a.wait_ns : DM_WAIT_NS;
    const bool fold = m.q < (1ull << 41) && beta <= 8;
    const u64 c63 = fold ? (1ull << 63) % m.q : 0, c64 = fold ? (0 - m.q) % m.q : 0;  // 2^63, 2^64 mod q
    const u32 mu32 = (u32)m.mu_hi;  // floor(2^64 / q) (SMALL: below 2^32)
    u32 pd[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        const u32 kc = c.k_first + min((u32)kk, c.k_count - 1);
        const u32 g = a.gal_diag[kc];
        const u32 run = s / RUN;
        const u32 hr = (g ? auto_src(run * RUN, g, a.log_n) : run * RUN) / RUN;
        pd[kk] = (g ? auto_src(s, g, a.log_n) : s) - hr * RUN;
    }
    WsAcc<SMALL> acc0[K3], acc1[K3];
#pragma unroll
    for (int kk = 0; kk < K3; kk++) acc0[kk].zero(), acc1[kk].zero();
    u32 terms = 0;
    for (u32 it = 0; it < n1n2; it++) {
        const u32 sidx = it % NS;
        // the warp decides together, so that its lanes stay converged
        if (!__all_sync(FULL, mbar_wait_abortable(&c.full_bar[sidx], (it / NS) & 1, wait_ns, c.abort))) {
            *c.abort = 1u;
            break;
        }
        const u32 j = n1 == 1 ? it : it / n1, i = n1 == 1 ? 0u : it % n1;
        const bool lifted = (i == 0) && a.lift0;
        const u64* st = c.smem + (size_t)sidx * LY::STAGE;
        u64 av, bv;
        if (j == 0) {
            if (lifted) {
                if (c.lift_limb) {
                    const u64 x = st[LY::OFF_A + l];
                    av = c.c0_lifted ? x : mul_shoup(x, c.lc, c.lsh, m.q);
                    bv = mul_shoup(st[LY::OFF_B + l], c.lc, c.lsh, m.q);
                } else {
                    av = bv = 0;
                }
            } else {
                av = st[LY::OFF_A + l];
                bv = st[LY::OFF_B + l];
            }
        } else {
            const u32 pm = auto_src(s, a.gal_mid[j], a.log_n) % RUN;
            WsAcc<SMALL> x0, x1;
            x0.zero();
            x1.zero();
            const ulonglong2* kp = (const ulonglong2*)(st + LY::OFF_KEY) + l;
#pragma unroll
            for (int b = 0; b < BETA; b++) {
                if (b < (int)beta) {
                    const u64 d = st[LY::OFF_DIG + b * RUN + pm];
                    const ulonglong2 kv = kp[b * RUN];
                    x0.mac(d, kv.x);
                    x1.mac(d, kv.y);
                }
            }
            if (lifted) {
                if (c.lift_limb) {
                    const u64 x = st[LY::OFF_A + pm];
                    x0.add(c.c0_lifted ? x : mul_shoup(x, c.lc, c.lsh, m.q));
                }
            } else {
                x0.add(st[LY::OFF_A + pm]);
            }
            // partial reductions feed the products (see k_diag_mac_staged)
            const U128 w0 = x0.wide(), w1 = x1.wide();
            if (fold) {
                av = (w0.lo & ~(1ull << 63)) + ((w0.lo >> 63) ? c63 : 0) + w0.hi * c64;
                bv = (w1.lo & ~(1ull << 63)) + ((w1.lo >> 63) ? c63 : 0) + w1.hi * c64;
                if constexpr (SMALL) {  // below 2^64 -> [0, 3q)
                    const u64 qa = ((u64)(u32)(av >> 32) * mu32 + __umulhi((u32)av, mu32)) >> 32;
                    const u64 qb = ((u64)(u32)(bv >> 32) * mu32 + __umulhi((u32)bv, mu32)) >> 32;
                    av -= qa * m.q;
                    bv -= qb * m.q;
                }
            } else {
                av = reduce128_lazy(w0, m);
                bv = reduce128_lazy(w1, m);
            }
        }
        u64 f[K3];
#pragma unroll
        for (int kk = 0; kk < K3; kk++) f[kk] = kk < (int)c.k_count ? st[kk * RUN + pd[kk]] : 0;
        __syncwarp();
        if ((l & 31) == 0) mbar_arrive(&c.empty_bar[sidx]);  // the warp has read stage sidx
#pragma unroll
        for (int kk = 0; kk < K3; kk++) {
            if (kk < (int)c.k_count) {
                acc0[kk].mac(av, f[kk]);
                acc1[kk].mac(bv, f[kk]);
            }
        }
        if (++terms == 64) {  // 64 products fit the accumulators (2^122 each, or 2^83 on the 96-bit path)
            terms = 0;
#pragma unroll
            for (int kk = 0; kk < K3; kk++) {
                acc0[kk].set(reduce128(acc0[kk].wide(), m));
                acc1[kk].set(reduce128(acc1[kk].wide(), m));
            }
        }
    }
    nbar_sync(1, RUN + 32);  // every thread of the CTA reaches this once; then one decision for all
    if (*c.abort) return;
#pragma unroll
    for (int kk = 0; kk < K3; kk++) {
        if (kk < (int)c.k_count) {
            a.U0[c.k_first + kk][c.ou + c.tN + s] = reduce128(acc0[kk].wide(), m);
            a.U1[c.k_first + kk][c.ou + c.tN + s] = reduce128(acc1[kk].wide(), m);
        }
    }
}

template <int K3, int RUN, int NS, int BETA, int MINB>
__global__ void __launch_bounds__(RUN + 32, MINB) k_diag_mac_ws(const __grid_constant__ DiagMacArgs a) {
    using LY = WsLayout<K3, RUN, NS, BETA>;
    constexpr u32 NT = RUN + 32;  // threads of the CTA
    constexpr u32 RB = RUN * 8;   // bytes per run
    constexpr u32 FULL = 0xffffffffu;
    extern __shared__ __align__(128) u64 smem[];
    __shared__ __align__(8) u64 full_bar[NS];
    __shared__ __align__(8) u64 empty_bar[NS];
    __shared__ u32 abort_flag;
    const u32 N = 1u << a.log_n;
    const u32 l = threadIdx.x;
    const u32 bidx = blockIdx.x % a.batch;
    const u32 run = blockIdx.x / a.batch;
    const size_t oab = bidx * a.bs_ab, odg = bidx * a.bs_dg, ou = bidx * a.bs_u;
    const u32 t = blockIdx.y;
    const u32 k_first = blockIdx.z * K3;
    const u32 k_count = min((u32)K3, a.n3 - k_first);
    const u32 gmod = t < a.level ? t : a.L + (t - a.level);
    const u32 drow = t < a.level ? t : a.diag_level + (t - a.level);
    const ModC m = a.mods[gmod];
    const size_t dstride = (size_t)(a.diag_level + a.k_p) * N;
    const size_t plane = (size_t)(a.L + a.k_p) * N;  // key pairs per digit
    const size_t dig_b = (size_t)a.ext * N;
    const size_t tN = (size_t)t * N;
    const u32 n1 = a.n1, n2 = a.n2, n1n2 = n1 * n2;
    const u32 beta = n2 > 1 ? a.beta : 0;  // <= BETA (host checks)
    const bool lift_limb = a.lift0 && t < a.level;
    const u64* c0l = a.c0l[bidx];
    u32* srun_of = (u32*)(smem + (size_t)NS * LY::STAGE);
    for (u32 jj = l; jj < n2; jj += NT) srun_of[jj] = jj ? auto_src(run * RUN, a.gal_mid[jj], a.log_n) / RUN : run;
    if (l == 0) {
#pragma unroll
        for (int b = 0; b < NS; b++) {
            mbar_init(&full_bar[b], 1);
            mbar_init(&empty_bar[b], RUN / 32);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    volatile u32* abort = &abort_flag;

    if (l >= RUN) {
        // ------------------------------------------------------------ producer warp
        const u32 ln = l - RUN;
        const u64* A0 = a.lift0 ? (c0l ? c0l : a.c0[bidx]) : a.A[0];
        const u64* B0 = a.lift0 ? a.c1[bidx] : a.B[0];
        // lane c < K3 keeps the source run of diagonal c's gather
        u32 hrun = 0;
        if (ln < (u32)K3) {
            const u32 kc = k_first + min(ln, k_count - 1);
            const u32 g = a.gal_diag[kc];
            hrun = (g ? auto_src(run * RUN, g, a.log_n) : run * RUN) / RUN;
        }
        u32 last[NS];  // the last step issued into each stage (lane 0)
#pragma unroll
        for (int b = 0; b < NS; b++) last[b] = ~0u;
        for (u32 it = 0; it < n1n2; it++) {
            const u32 sidx = it % NS;
            bool go = true;
            if (ln == 0) {
                if (it >= NS && !mbar_wait_abortable(&empty_bar[sidx], ((it - NS) / NS) & 1, DM_WAIT_NS, abort))
                    *abort = 1u;  // every compute warp has read step it - NS, or giving up
                go = !*abort;
            }
            if (!__shfl_sync(FULL, go, 0)) break;
            if (it == a.starve_step) continue;  // test hook: this step is never issued
            const u32 j = n1 == 1 ? it : it / n1, i = n1 == 1 ? 0u : it % n1;
            const bool lifted = (i == 0) && a.lift0;
            const bool copy_a = !lifted || lift_limb;
            const u32 n_ab = j == 0 ? (copy_a ? 2u : 0u) : (copy_a ? 1u : 0u);
            const u32 n_dig = j == 0 ? 0u : beta;
            u64* st = smem + (size_t)sidx * LY::STAGE;
            u64* bar = &full_bar[sidx];
            if (ln == 0) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_expect_tx(bar, (k_count + 3 * n_dig + n_ab) * RB);
                last[sidx] = it;
            }
            __syncwarp();
            // one copy per lane: diagonals, digits, A (and B), keys
            const u32 srun = srun_of[j];
            const u32 c = ln;
            if (c < k_count) {
                const size_t didx = (size_t)(n1 * j + i) * dstride + (size_t)drow * N;
                tma_load_1d(st + (size_t)c * RUN,
                            a.diags + (size_t)(n1n2 * (k_first + c)) * dstride + didx + (size_t)hrun * RUN, RB, bar);
            } else if (c >= (u32)K3 && c < (u32)K3 + n_dig) {
                const u32 b = c - K3;
                tma_load_1d(st + LY::OFF_DIG + (size_t)b * RUN, a.Dg[i] + odg + b * dig_b + tN + (size_t)srun * RUN,
                            RB, bar);
            } else if (c == (u32)(K3 + BETA) && n_ab >= 1) {
                const u64* Ai = i ? a.A[i] + oab : A0;
                tma_load_1d(st + LY::OFF_A, Ai + tN + (size_t)srun * RUN, RB, bar);
            } else if (c == (u32)(K3 + BETA + 1) && n_ab == 2) {
                const u64* Bi = i ? a.B[i] + oab : B0;
                tma_load_1d(st + LY::OFF_B, Bi + tN + (size_t)srun * RUN, RB, bar);
            } else if (c >= (u32)(K3 + BETA + 2) && c < (u32)(K3 + BETA + 2) + n_dig) {
                const u32 b = c - (K3 + BETA + 2);
                tma_load_1d(st + LY::OFF_KEY + (size_t)b * 2 * RUN,
                            a.keys[j] + 2 * ((size_t)b * plane + (size_t)gmod * N + (size_t)run * RUN), 2 * RB, bar);
            }
        }
        nbar_sync(1, NT);  // every thread of the CTA reaches this once
        if (*abort && ln == 0) {
            // drain: the last phase issued into each stage (the earlier ones completed and were consumed)
#pragma unroll
            for (int b = 0; b < NS; b++)
                if (last[b] != ~0u) mbar_wait_bounded(&full_bar[b], (last[b] / NS) & 1);
            atomicExch(a.err, 1u);
        }
        return;
    }

    // ---------------------------------------------------------------- compute threads
    const u32 s = run * RUN + l;
    const u64 lc = lift_limb ? a.lift_c[gmod] : 0, lsh = lift_limb ? a.lift_sh[gmod] : 0;
    const WsCtx c{a, smem, full_bar, empty_bar, abort, s, l, n1, n2, beta, k_first, k_count, tN, ou, lift_limb,
                  c0l != nullptr, lc, lsh, m};
    // moduli 2^32 < q < 2^41 (every 40-bit prime): 96-bit accumulators; wider ones: 128-bit
    if (m.q > (1ull << 32) && m.q < (1ull << 41) && beta <= 8) ws_compute<K3, RUN, NS, BETA, true>(c);
    else ws_compute<K3, RUN, NS, BETA, false>(c);
}

// P x on the Q limbs (Alg. 2 line 2), for every polynomial of a batch.
struct LiftArgs {
    const u64* in[DM_MAX_B];
    u64* out[DM_MAX_B];
};
__global__ void k_lift(const ModC* __restrict__ mods, const u64* __restrict__ lift_c, const u64* __restrict__ lift_sh,
                       const __grid_constant__ LiftArgs p, u32 log_n) {
    const u32 N = 1u << log_n;
    const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 t = blockIdx.y, i = blockIdx.z;
    if (s >= N) return;
    const size_t o = (size_t)t * N + s;
    p.out[i][o] = mul_shoup(p.in[i][o], lift_c[t], lift_sh[t], mods[t].q);
}

constexpr size_t DM_SMEM_MAX = 226 * 1024;  // dynamic part; the mbarriers take a few static bytes

template <int K3, int RUN, int NS, int KB>
bool try_staged(const DiagMacArgs& a, cudaStream_t st) {
    const size_t beta = a.n2 > 1 ? a.beta : 0;
    const size_t sm = 8ull * RUN * NS * (K3 + beta + 2) + ((4ull * a.n2 + 15) & ~15ull);  // stages + srun table
    const u32 N = 1u << a.log_n;
    if (sm > DM_SMEM_MAX || N % RUN || beta > (size_t)KB) return false;
    // The dynamic shared-memory limit is a per-device function attribute: set
    // it once per device (threads may race to set it; the call is idempotent).
    // A device that refuses it falls back to the next variant, and the error
    // the refusal left is cleared so that a later status check does not see it.
    static std::atomic<uint64_t> attr_set{0}, attr_bad{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    const uint64_t bit = 1ull << dev;
    if (attr_bad.load(std::memory_order_relaxed) & bit) return false;
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        if (cudaFuncSetAttribute(k_diag_mac_staged<K3, RUN, NS, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)DM_SMEM_MAX) != cudaSuccess) {
            cudaGetLastError();
            attr_bad.fetch_or(bit, std::memory_order_relaxed);
            return false;
        }
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    const dim3 grid((N / RUN) * a.batch, a.ext, (a.n3 + K3 - 1) / K3);
    k_diag_mac_staged<K3, RUN, NS, KB><<<grid, RUN, sm, st>>>(a);
    return true;
}

template <int K3, int RUN, int NS, int BETA, int MINB = 1>
bool try_ws(const DiagMacArgs& a, cudaStream_t st) {
    using LY = WsLayout<K3, RUN, NS, BETA>;
    const u32 beta = a.n2 > 1 ? a.beta : 0;
    const size_t sm = LY::bytes(a.n2);
    const u32 N = 1u << a.log_n;
    if (sm > DM_SMEM_MAX || N % RUN || beta > (u32)BETA) return false;
    static std::atomic<uint64_t> attr_set{0}, attr_bad{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    const uint64_t bit = 1ull << dev;
    if (attr_bad.load(std::memory_order_relaxed) & bit) return false;
    if (!(attr_set.load(std::memory_order_acquire) & bit)) {
        if (cudaFuncSetAttribute(k_diag_mac_ws<K3, RUN, NS, BETA, MINB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DM_SMEM_MAX) != cudaSuccess) {
            cudaGetLastError();
            attr_bad.fetch_or(bit, std::memory_order_relaxed);
            return false;
        }
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    const dim3 grid((N / RUN) * a.batch, a.ext, (a.n3 + K3 - 1) / K3);
    k_diag_mac_ws<K3, RUN, NS, BETA, MINB><<<grid, RUN + 32, sm, st>>>(a);
    return true;
}

// Which K6 form runs: the warp-specialised one when it fits (0), else the
// CTA-barrier staged one; CKKS_K6_FORM=1 forces the latter (comparisons).
static int k6_form() {
    static const int f = [] {
        const char* e = getenv("CKKS_K6_FORM");
        return e ? atoi(e) : 0;
    }();
    return f;
}

// Tile of the warp-specialised K6: positions per CTA.  More CTAs per SM give
// more independent stage rings, which is what the compute warps wait on:
// with four or fewer outer indices per CTA the default is 128 positions and
// four CTAs per SM (measured against two of 256 and one of 512 at the N = 2^16
// splits: 4% and 9% faster), tile_run = 256 or 512 on request; with eight
// outer accumulators per thread (register budget) 128 positions and two CTAs
// per SM by default (2% faster than one of 256), 256 on request.
template <int K3>
bool launch_ws(const DiagMacArgs& a, cudaStream_t st) {
    const bool mid = a.n2 > 1;
    if constexpr (K3 >= 8) {
        if (a.tile_run == 256) return mid ? try_ws<K3, 256, 2, 6>(a, st) : try_ws<K3, 256, 4, 0>(a, st);
        return mid ? try_ws<K3, 128, 2, 6, 2>(a, st) : try_ws<K3, 128, 4, 0, 2>(a, st);
    } else {
        if (a.tile_run == 512) return mid ? try_ws<K3, 512, 2, 6>(a, st) : try_ws<K3, 512, 4, 0>(a, st);
        if (a.tile_run == 256) return mid ? try_ws<K3, 256, 2, 6, 2>(a, st) : try_ws<K3, 256, 4, 0, 2>(a, st);
        return mid ? try_ws<K3, 128, 2, 6, 4>(a, st) : try_ws<K3, 128, 4, 0, 4>(a, st);
    }
}

template <int K3>
bool launch_staged(const DiagMacArgs& a, cudaStream_t st) {
    if (k6_form() == 0 && launch_ws<K3>(a, st)) return true;
    return try_staged<K3, 512, 4, 6>(a, st) || try_staged<K3, 512, 3, 6>(a, st) || try_staged<K3, 256, 4, 6>(a, st);
}

}  // namespace

// Switching keys are stored with their two components interleaved per word:
// in [beta_max][2][L+k][N] -> out [beta_max][L+k][N] of (component 0, component 1).
__global__ void k_interleave_key(const u64* __restrict__ in, ulonglong2* __restrict__ out, size_t plane,
                                 size_t total) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const size_t b = i / plane, r = i - b * plane;
    out[i] = make_ulonglong2(in[(2 * b) * plane + r], in[(2 * b + 1) * plane + r]);
}

void launch_interleave_key(const u64* in, u64* out, size_t plane, u32 beta_max, cudaStream_t st) {
    const size_t total = plane * beta_max;
    k_interleave_key<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in, (ulonglong2*)out, plane, total);
    count_launch();
}

void launch_lift(const ModC* mods, const u64* lift_c, const u64* lift_sh, const u64* const* in, u64* const* out,
                 u32 count, u32 level, u32 log_n, cudaStream_t st) {
    const u32 N = 1u << log_n;
    for (u32 c0 = 0; c0 < count; c0 += DM_MAX_B) {
        LiftArgs p{};
        const u32 n = std::min<u32>(DM_MAX_B, count - c0);
        for (u32 i = 0; i < n; i++) p.in[i] = in[c0 + i], p.out[i] = out[c0 + i];
        k_lift<<<dim3((N + 255) / 256, level, n), 256, 0, st>>>(mods, lift_c, lift_sh, p, log_n);
        count_launch();
    }
}

void launch_wait_selftest(u32* err, u64 limit_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
    count_launch();
}

void launch_ks_batch(const KsBatchArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    ProfScope ps(K_KS_INNER, st, 2.0 * a.beta * a.count * a.ext * N);
    k_ks_batch<<<dim3(((N + THREADS - 1) / THREADS) * a.count, a.ext), THREADS, 0, st>>>(a);
    count_launch();
}

void launch_ks_multi(const KsMultiArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    ProfScope ps(K_KS_INNER, st, 2.0 * a.beta * a.count * a.ext * N);
    k_ks_multi<<<dim3((N + THREADS - 1) / THREADS, a.ext), THREADS, 0, st>>>(a);
    count_launch();
}

void launch_ks_inner(const KsArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    ProfScope ps(K_KS_INNER, st, 2.0 * a.beta * a.ext * N);
    k_ks_inner<<<dim3((N + THREADS - 1) / THREADS, a.ext), THREADS, 0, st>>>(a);
    count_launch();
}

void launch_diag_mac(const DiagMacArgs& a, cudaStream_t st) {
    const u32 N = 1u << a.log_n;
    u32 k3 = 1;
    while (k3 < a.n3 && k3 < (u32)DM_MAX_K3) k3 *= 2;
    // a tile with fewer outer indices per CTA (more CTAs along z, each redoing the middle layer)
    if (a.tile_k3 && a.tile_k3 < k3 && !(a.tile_k3 & (a.tile_k3 - 1))) k3 = a.tile_k3;
    const dim3 grid(((N + THREADS - 1) / THREADS) * a.batch, a.ext, (a.n3 + k3 - 1) / k3);
    // multiply-accumulates: two per diagonal product (c0, c1), and the middle
    // layer's 2 beta per step with j > 0, once per block of k3 outer indices
    const double n1n2 = (double)a.n1 * a.n2, beta_mid = a.n2 > 1 ? a.beta : 0;
    const double macs = (double)N * a.batch * a.ext *
                        (2.0 * n1n2 * a.n3 + 2.0 * beta_mid * grid.z * (n1n2 - a.n1));
    ProfScope ps(K_DIAG_MAC, st, macs);
    bool done = false;
    switch (k3) {
        case 1: done = launch_staged<1>(a, st); break;
        case 2: done = launch_staged<2>(a, st); break;
        case 4: done = launch_staged<4>(a, st); break;
        default: done = launch_staged<8>(a, st); break;
    }
    if (done) {
        count_launch();
        return;
    }
    switch (k3) {
        case 1: k_diag_mac<1><<<grid, THREADS, 0, st>>>(a); break;
        case 2: k_diag_mac<2><<<grid, THREADS, 0, st>>>(a); break;
        case 4: k_diag_mac<4><<<grid, THREADS, 0, st>>>(a); break;
        default: k_diag_mac<8><<<grid, THREADS, 0, st>>>(a); break;
    }
    count_launch();
}

}  // namespace ckks
