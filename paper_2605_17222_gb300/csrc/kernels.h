// Kernel launch interface shared by the .cu files of the library (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "modarith.cuh"

namespace ckks {

// Per-context device tables every NTT kernel reads.
struct NttTables {
    const ModC* mods;          // [n_mod] {q, mu}
    const ulonglong2* psi;     // [n_mod][N] (psi^brv(i), Shoup companion)
    const ulonglong2* ipsi;    // [n_mod][N] (psi^-brv(i), Shoup companion)
    u32 log_n;
};

// One limb of a forward NTT.
//   pass 1 load : nsrc == 0 -> src[x];
//                 nsrc  > 0 -> sum_j src[j*N + x] * bcst[j] mod q   (basis conversion, Eq. 3)
//                 (bits 0-15: the source count; bit 16: every source word is
//                 below 2^41, which with a target 2^32 < q < 2^41 allows 96-bit sums)
//   pass 2 store: subout == nullptr -> dst[x] = X;
//                 otherwise subout[x] = (subx[x] - X) * c mod q        (ModDown tail, Eq. 4)
// Pass 1 writes dst; pass 2 runs in place on dst.
// FwdJob::nsrc bit 17: a copy job, dst[x] = src[x -> x^gal] with gal in c
// (0: plain copy) and no transform, for the limbs a Decompose passes through
// unchanged; it rides in the same launch as the transforms.
// Bit 18 (with bit 17): a scaling job instead, dst[x] = src[x] * c mod q
// (c_sh its Shoup companion), e.g. the lift P c0 of Alg. 2 line 2.
constexpr u32 FWD_COPY = 1u << 17;
constexpr u32 FWD_SCALE = 1u << 18;
struct FwdJob {
    const u64* src;
    u64* dst;
    const u64* bcst;
    const u64* subx;
    u64* subout;
    u64 c, c_sh;
    u32 mod;
    u32 nsrc;
};

// One limb of an inverse NTT: pass A reads src (gathered through x -> x^gal
// when gal != 0) and writes tmp; pass B reads tmp and writes dst scaled by c
// (c includes N^-1).  tmp may alias dst; src may alias tmp only when gal == 0.
struct InvJob {
    const u64* src;
    u64* tmp;
    u64* dst;
    u64 c, c_sh;
    u32 mod;
    u32 gal;
};

void launch_fwd_ntt(const NttTables& T, const FwdJob* jobs, int njobs, cudaStream_t st);
void launch_inv_ntt(const NttTables& T, const InvJob* jobs, int njobs, cudaStream_t st);

// out[l][s] = in[l][src_g(s)] for n_limbs limbs (NTT-domain automorphism, Eq. 7).
void launch_automorphism(const u64* in, u64* out, u32 n_limbs, u32 gal, u32 log_n, cudaStream_t st);

// out[s] = (acc ? out[s] : 0) + a[src_g(s)] + b[s] mod q_l, per limb (b may be null).
struct AddJob {
    const u64* a;
    const u64* b;
    u64* out;
    u32 mod;
    u32 pad;
};
void launch_add_gather(const ModC* mods, const AddJob* jobs, int njobs, u32 gal, int accumulate, u32 log_n,
                       cudaStream_t st);

// Switching-key inner product with hoisted automorphism (K4).
struct KsArgs {
    const u64* digits;      // [beta][ext][N]
    const u64* key;         // [beta_max][L+k][N] word pairs (interleaved layout below)
    const u64* x0;          // null, ext poly, or Q poly to lift
    u64* out0;
    u64* out1;
    const ModC* mods;       // context moduli (index = global modulus id)
    const u64* lift_c;      // [L+k] [P]_{q_j} (0 for P moduli) and Shoup companions
    const u64* lift_sh;
    u32 level, ext, L, beta, beta_max, gal, x0_mode, accumulate, log_n;
};
void launch_ks_inner(const KsArgs& a, cudaStream_t st);

// out_c += sum_k phi_{r_k}(x0_k (c = 0 only) + <D_k, swk~_{r_k, c}>), k < count:
// the outer key-switch layer of Algorithm 2 (lines 17-18) for every giant
// index at once.
constexpr int KS_MAX_MULTI = 64;
struct KsMultiArgs {
    const u64* digits[KS_MAX_MULTI];  // [beta][ext][N] each
    const u64* keys[KS_MAX_MULTI];    // [beta_max][L+k][N] word pairs each (interleaved)
    const u64* x0[KS_MAX_MULTI];      // [ext][N] each
    u32 gal[KS_MAX_MULTI];
    u64* out0;
    u64* out1;
    const ModC* mods;
    u32 count, level, ext, L, beta, log_n;
};
void launch_ks_multi(const KsMultiArgs& a, cudaStream_t st);

// Rotation keys in the library's layout: the user's [beta_max][2][L+k][N]
// with the two components interleaved per word, [beta_max][L+k][N] x 2.
// Every kernel that reads a key reads one 16-byte word per (digit, limb,
// position).  plane = (L+k) N.
void launch_interleave_key(const u64* in, u64* out, size_t plane, u32 beta_max, cudaStream_t st);

// Many independent K4 products (overwrite form, x0 lifted from a Q
// polynomial) in one launch: entry e reads digits, key and x0 and writes
// out0/out1.  Entries that share a key are adjacent in the grid.
constexpr int KS_MAX_BATCH = 128;
struct KsBatchEntry {
    const u64* digits;
    const u64* key;
    const u64* x0;
    u64* out0;
    u64* out1;
    u32 gal;
    u32 pad;
};
struct KsBatchArgs {
    KsBatchEntry e[KS_MAX_BATCH];
    const ModC* mods;
    const u64* lift_c;
    const u64* lift_sh;
    u32 count, level, ext, L, beta, log_n;
};
void launch_ks_batch(const KsBatchArgs& a, cudaStream_t st);

// Multi-output plaintext-diagonal multiply-accumulate with the middle
// (hoisted) key-switch layer fused in (K6).  See ks.cu.
constexpr int DM_MAX_N1 = 64;
constexpr int DM_MAX_N2 = 1024;
constexpr int DM_MAX_K3 = 8;   // giant indices per thread (grid.z covers the rest)
constexpr int DM_MAX_N3 = 64;
constexpr int DM_MAX_B = 16;   // ciphertexts per batched launch
struct DiagMacArgs {
    const ModC* mods;
    const u64* lift_c;
    const u64* lift_sh;
    const u64* diags;       // [n_diag][diag_level + k][N]
    const u64* A[DM_MAX_N1];
    const u64* B[DM_MAX_N1];
    const u64* Dg[DM_MAX_N1];        // digits per baby index (middle layer), [beta][ext][N]
    const u64* keys[DM_MAX_N2];      // middle-layer keys, index j (j >= 1)
    u32 gal_mid[DM_MAX_N2];          // x -> x^gal for rotation n1*j*stride
    u64* U0[DM_MAX_N3];
    u64* U1[DM_MAX_N3];
    u32 gal_diag[DM_MAX_N3];         // rotation -(n1*n2*k*stride), 0 = none
    u32 level, ext, L, k_p, beta, log_n;
    u32 n1, n2, n3, lift0, diag_level;
    u32* err;                        // set to nonzero when a bounded device wait gives up
    // Failure-detection test hook of the staged kernel: the step loop's
    // waits give up after wait_ns (0: the default of one second), and step
    // starve_step (~0u: none) is never issued, so that its wait runs out.
    // The drain of copies in flight always keeps the default limit.
    u64 wait_ns;
    u32 starve_step;
    // Tile (0 = default): outer indices per CTA (a power of two below the
    // default, which is the next power of two >= n3, at most 8) and positions
    // per CTA (128, 256 or 512; see launch_ws).  Results do not depend on it.
    u32 tile_k3, tile_run;
    // Batch of ciphertexts sharing the diagonals and keys: ciphertext b uses
    // c0[b], c1[b] as its lifted inputs and A[i] + b*bs_ab, B[i] + b*bs_ab,
    // Dg[i] + b*bs_dg, U0/U1[k] + b*bs_u for the rest.  CTAs of the same
    // (limb, run) for different b are adjacent in the grid, so the diagonal
    // and key words they share are read from HBM once.
    u32 batch;
    u64 bs_ab, bs_dg, bs_u;
    const u64* c0[DM_MAX_B];
    const u64* c1[DM_MAX_B];
    // P c0 per ciphertext (Q limbs [level][N], from launch_lift), or null:
    // the lifted input of Alg. 2 line 2 computed once instead of at every step
    const u64* c0l[DM_MAX_B];
};
void launch_diag_mac(const DiagMacArgs& a, cudaStream_t st);
// out_i[t][s] = in_i[t][s] * [P]_{q_t} mod q_t for t < level (Alg. 2 line 2,
// the Q limbs of P c0; the P limbs are zero and not stored), i < count.
void launch_lift(const ModC* mods, const u64* lift_c, const u64* lift_sh, const u64* const* in, u64* const* out,
                 u32 count, u32 level, u32 log_n, cudaStream_t st);
void launch_wait_selftest(u32* err, u64 limit_ns, cudaStream_t st);

uint64_t launches();
void count_launch(int n = 1);

// Kernel classes for live timing (ckks_profile_*).
enum KClass { K_DIAG_MAC = 0, K_KS_INNER, K_FWD_COLS, K_FWD_ROWS, K_INV_ROWS, K_INV_COLS, K_AUTO, K_ADD, K_NCLASS };
extern const char* const kclass_names[K_NCLASS];
bool prof_on(int cls);
// Brackets one launch with events when its class is enabled, and adds the
// launch's algorithmic integer work (128-bit multiply-accumulates, NTT
// butterflies) to the class's totals.
struct ProfScope {
    int cls;
    cudaStream_t st;
    void* ev;
    ProfScope(int c, cudaStream_t s, double macs = 0, double butterflies = 0);
    ~ProfScope();
};
int prof_class(const char* name);
void prof_enable(int cls, bool on);
bool prof_read(int cls, double* ms, uint64_t* n);
bool prof_work(int cls, double* macs, double* butterflies);
void prof_reset();

// Register-only rate probes of the library's own 128-bit multiply-accumulate
// and forward NTT butterfly over `blocks` CTAs (best of two timed runs after a
// warm-up); synchronous, on a stream of its own.
cudaError_t probe_int_rates(u32 blocks, double* macs_per_s, double* butterflies_per_s);

}  // namespace ckks
