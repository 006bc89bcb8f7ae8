// Host side of the library: context constants, device memory, the key
// switching steps (Fig. 1), the four LT schedules and the C ABI of
// include/ckks_lt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <functional>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ckks_lt.h"
#include "kernels.h"

using namespace ckks;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

namespace {

struct Fail {
    ckks_status st;
};

[[noreturn]] void fail(ckks_status st, const std::string& msg) {
    g_err = msg;
    throw Fail{st};
}

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(e == cudaErrorMemoryAllocation ? CKKS_ENOMEM : CKKS_ECUDA,
                               std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(x) cuda_check((x), #x)

template <typename F>
ckks_status guarded(F&& f) {
    try {
        f();
        return CKKS_OK;
    } catch (const Fail& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return CKKS_ENOMEM;
    } catch (...) {
        g_err = "unexpected exception";
        return CKKS_EINVAL;
    }
}

// ------------------------------------------------------------------ host modular arithmetic
u64 mulmod_h(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 powmod_h(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_h(r, a, q);
        a = mulmod_h(a, a, q);
        e >>= 1;
    }
    return r;
}
u64 invmod_h(u64 a, u64 q) { return powmod_h(a % q, q - 2, q); }  // q prime
u64 shoup_h(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

bool is_prime_h(u64 n) {
    if (n < 2) return false;
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) d >>= 1, s++;
    for (u64 a : bases) {
        u64 x = powmod_h(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mulmod_h(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

ModC modc_h(u64 q) {
    u128 mu = (~(u128)0) / q;  // = floor(2^128 / q) since q does not divide 2^128
    return ModC{q, (u64)(mu >> 64), (u64)mu};
}

u32 brv_h(u32 x, u32 bits) {
    u32 r = 0;
    for (u32 i = 0; i < bits; i++) r = (r << 1) | ((x >> i) & 1);
    return r;
}

// ------------------------------------------------------------------ device buffers
struct DevBuf {
    u64* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// ------------------------------------------------------------------ context
struct LevelConsts {
    // Decompose: per Q limb j, N^-1 (Q_b/q_j)^-1 mod q_j; table [beta][ext][alpha] of [Q_b/q_j]_t
    std::vector<u64> dec_c, dec_sh;
    u64* dec_tab = nullptr;
    // ModDown: per P limb, N^-1 (P/p_i)^-1; table [level][k] of [P/p_i]_{q_j}; P^-1 mod q_j
    std::vector<u64> md_c, md_sh, md_pinv, md_pinv_sh;
    u64* md_tab = nullptr;
    // ModDown+rescale over {q_{l-1}, p_0..}: same shapes with k+1 sources, level-1 targets
    std::vector<u64> mdr_c, mdr_sh, mdr_pinv, mdr_pinv_sh;
    u64* mdr_tab = nullptr;
    // rescale: source q_{l-1}
    std::vector<u64> rs_c, rs_sh, rs_inv, rs_inv_sh;
    u64* rs_tab = nullptr;
};

struct ckks_ctx {
    int device = 0;
    u32 log_n = 0, N = 0, L = 0, K = 0, dnum = 0, alpha = 0, beta_max = 0;
    std::vector<u64> mods;  // q_0..q_{L-1}, p_0..p_{K-1}
    DevBuf d_mods, d_psi, d_ipsi, d_lift, d_lift_sh, d_err;
    std::vector<u64> lift_c, lift_sh;  // host copies: [P]_{q_t} and its Shoup companion per Q limb
    NttTables T{};
    std::map<u32, LevelConsts> levels;
    std::map<u32, u64*> keys;  // rotation (mod N/2) -> [beta_max][L+K][N] word pairs (components interleaved)
    std::map<std::tuple<int, u32, u32, int32_t, int32_t>, lt_split> tuned;  // (algo, level, D, stride, offset0 mod N/2)
    // DH-BSGS schedule per (level, D, stride, offset0 mod N/2, n1, n2) measured by lt_autotune:
    // true = the baby steps fused into the diagonal kernel's middle layer, TH(1, n1, n2)
    std::map<std::tuple<u32, u32, int32_t, int32_t, u32, u32>, bool> dh_fused;
    // the diagonal kernel's tile measured by lt_autotune for a shape's tuned split (same key as `tuned`)
    std::map<std::tuple<int, u32, u32, int32_t, int32_t>, std::pair<u32, u32>> tuned_tile;
    mutable std::mutex mu;
    size_t bytes = 0;
    // failure-detection test hook of the staged diagonal kernel (ckks_debug_diag_mac_waits)
    u64 dbg_wait_ns = 0;
    u32 dbg_starve_step = ~0u;
    u32 dbg_tile_k3 = 0, dbg_tile_run = 0;  // forced diagonal-kernel tile (ckks_debug_diag_mac_tile)
    // fork/join lanes of lt_eval_batch: independent groups run on the caller's
    // stream and up to FORK_LANES - 1 more, so that one group's NTT-bound
    // phases overlap another's HBM-bound diagonal multiply-accumulate
    // Each caller stream has its own lanes, so that a stream being recorded
    // into a graph captures only its own lanes, never another caller's work.
    static constexpr u32 FORK_LANES = 4;
    struct Lanes {
        cudaStream_t s[FORK_LANES - 1] = {};
        cudaEvent_t fork = nullptr, join[FORK_LANES - 1] = {};
    };
    std::mutex fork_mu;
    std::map<cudaStream_t, Lanes> lanes;

    u32 beta(u32 level) const { return (level + alpha - 1) / alpha; }
    u32 slots() const { return N / 2; }
    size_t key_words() const { return (size_t)beta_max * 2 * (L + K) * N; }
    u32 gmod(u32 level, u32 t) const { return t < level ? t : L + (t - level); }
    u32 galois(int64_t r) const {
        int64_t rr = r % (int64_t)slots();
        if (rr < 0) rr += slots();
        return (u32)powmod_h(5, (u64)rr, 2ull * N);
    }
    u32 rotkey(int64_t r) const {
        int64_t rr = r % (int64_t)slots();
        if (rr < 0) rr += slots();
        return (u32)rr;
    }

    u64* dalloc(size_t words) {
        void* p = nullptr;
        CK(cudaMalloc(&p, words * sizeof(u64)));
        bytes += words * sizeof(u64);
        return (u64*)p;
    }
    void dfree(u64* p, size_t words) {
        if (p) {
            cudaFree(p);
            bytes -= words * sizeof(u64);
        }
    }
    u64* upload(const std::vector<u64>& v) {
        u64* p = dalloc(v.size());
        const cudaError_t e = cudaMemcpy(p, v.data(), v.size() * sizeof(u64), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {  // the block is not stored anywhere yet: free and uncount it here
            dfree(p, v.size());
            CK(e);
        }
        return p;
    }

    const LevelConsts& lc(u32 level);
};

struct ckks_ct {
    ckks_ctx* ctx;
    u32 level;
    u64* d;
    bool owned;
};

struct ckks_diags {
    ckks_ctx* ctx;
    u32 n_diag, level;
    int32_t offset0, stride;
    u64* d;
};

// Constants that depend on the level (digit boundaries, sources of the
// merged rescale), computed on first use.
const LevelConsts& ckks_ctx::lc(u32 level) {
    std::lock_guard<std::mutex> g(mu);
    auto it = levels.find(level);
    if (it != levels.end()) return it->second;
    LevelConsts c;
    const u32 ext = level + K, beta = this->beta(level);
    // the device tables uploaded so far are freed (and uncounted) if a later upload fails
    struct Unwind {
        ckks_ctx* ctx;
        LevelConsts* c;
        size_t words[4];
        bool armed = true;
        ~Unwind() {
            if (!armed) return;
            u64* tabs[4] = {c->dec_tab, c->md_tab, c->mdr_tab, c->rs_tab};
            for (int i = 0; i < 4; i++) ctx->dfree(tabs[i], words[i]);
        }
    } unwind{this, &c, {(size_t)beta * ext * alpha, (size_t)level * K, (size_t)(level - 1) * (K + 1),
                        (size_t)(level - 1)}};
    auto modof = [&](u32 t) { return mods[gmod(level, t)]; };
    // Decompose, Eq. (3) per digit
    c.dec_c.resize(level);
    c.dec_sh.resize(level);
    std::vector<u64> dt((size_t)beta * ext * alpha, 0);
    for (u32 b = 0; b < beta; b++) {
        const u32 first = b * alpha, cnt = std::min(alpha, level - first);
        for (u32 jj = 0; jj < cnt; jj++) {
            const u32 j = first + jj;
            const u64 qj = mods[j];
            u64 qhat = 1;
            for (u32 ii = 0; ii < cnt; ii++)
                if (ii != jj) qhat = mulmod_h(qhat, mods[first + ii] % qj, qj);
            const u64 v = mulmod_h(invmod_h(N % qj, qj), invmod_h(qhat, qj), qj);
            c.dec_c[j] = v;
            c.dec_sh[j] = shoup_h(v, qj);
            for (u32 t = 0; t < ext; t++) {
                if (t >= first && t < first + cnt) continue;
                const u64 mt = modof(t);
                u64 h = 1;
                for (u32 ii = 0; ii < cnt; ii++)
                    if (ii != jj) h = mulmod_h(h, mods[first + ii] % mt, mt);
                dt[((size_t)b * ext + t) * alpha + jj] = h;
            }
        }
    }
    c.dec_tab = upload(dt);
    // generic "modulus switch down" constants for a source set S and target limbs 0..ntgt-1
    auto down = [&](const std::vector<u32>& srcg, u32 ntgt, std::vector<u64>& sc, std::vector<u64>& ssh,
                    std::vector<u64>& pinv, std::vector<u64>& pinv_sh, u64*& tab) {
        const u32 ns = (u32)srcg.size();
        sc.resize(ns);
        ssh.resize(ns);
        for (u32 i = 0; i < ns; i++) {
            const u64 pi = mods[srcg[i]];
            u64 hat = 1;
            for (u32 o = 0; o < ns; o++)
                if (o != i) hat = mulmod_h(hat, mods[srcg[o]] % pi, pi);
            const u64 v = mulmod_h(invmod_h(N % pi, pi), invmod_h(hat, pi), pi);
            sc[i] = v;
            ssh[i] = shoup_h(v, pi);
        }
        std::vector<u64> tb((size_t)ntgt * ns);
        pinv.resize(ntgt);
        pinv_sh.resize(ntgt);
        for (u32 j = 0; j < ntgt; j++) {
            const u64 qj = mods[j];
            u64 prod = 1;
            for (u32 i = 0; i < ns; i++) {
                u64 hat = 1;
                for (u32 o = 0; o < ns; o++)
                    if (o != i) hat = mulmod_h(hat, mods[srcg[o]] % qj, qj);
                tb[(size_t)j * ns + i] = hat;
                prod = mulmod_h(prod, mods[srcg[i]] % qj, qj);
            }
            pinv[j] = invmod_h(prod, qj);
            pinv_sh[j] = shoup_h(pinv[j], qj);
        }
        tab = upload(tb);
    };
    std::vector<u32> P;
    for (u32 i = 0; i < K; i++) P.push_back(L + i);
    down(P, level, c.md_c, c.md_sh, c.md_pinv, c.md_pinv_sh, c.md_tab);
    if (level >= 2) {
        std::vector<u32> S{level - 1};
        for (u32 i = 0; i < K; i++) S.push_back(L + i);
        down(S, level - 1, c.mdr_c, c.mdr_sh, c.mdr_pinv, c.mdr_pinv_sh, c.mdr_tab);
        down(std::vector<u32>{level - 1}, level - 1, c.rs_c, c.rs_sh, c.rs_inv, c.rs_inv_sh, c.rs_tab);
    }
    unwind.armed = false;
    return levels.emplace(level, std::move(c)).first->second;
}

// ------------------------------------------------------------------ stream-ordered scratch
namespace {

struct Arena {
    cudaStream_t st;
    std::vector<void*> blocks;
    size_t limb_words;
    explicit Arena(cudaStream_t s, size_t lw) : st(s), limb_words(lw) {}
    u64* limbs(size_t n) {
        void* p = nullptr;
        CK(cudaMallocAsync(&p, std::max<size_t>(1, n) * limb_words * sizeof(u64), st));
        blocks.push_back(p);
        return (u64*)p;
    }
    ~Arena() {
        for (void* p : blocks) cudaFreeAsync(p, st);
    }
};

// The fork lanes of one caller stream (lt_eval_batch).
void destroy_lanes(ckks_ctx::Lanes& ln) {
    for (u32 i = 0; i + 1 < ckks_ctx::FORK_LANES; i++) {
        if (ln.s[i]) cudaStreamDestroy(ln.s[i]);
        if (ln.join[i]) cudaEventDestroy(ln.join[i]);
    }
    if (ln.fork) cudaEventDestroy(ln.fork);
    ln = ckks_ctx::Lanes{};
}
// Drops the lanes of a private stream the library is about to destroy (its
// work must be complete).
void release_lanes(ckks_ctx* C, cudaStream_t st) {
    std::lock_guard<std::mutex> g(C->fork_mu);
    auto it = C->lanes.find(st);
    if (it == C->lanes.end()) return;
    destroy_lanes(it->second);
    C->lanes.erase(it);
}

// ------------------------------------------------------------------ key switching steps
// Decompose (Fig. 1, Eq. 3) of `count` polynomials at once: c_i [level][N]
// (gathered through x -> x^gal if gal) -> digits_i [beta][level+K][N].
// Y: scratch [count][level][N].  One launch pair per transform direction
// covers every polynomial, so small steps still fill the GPU.
// extra: further elementwise jobs (FWD_COPY) to run in the forward launch.
void op_decompose_batch(ckks_ctx* C, u32 level, const std::vector<const u64*>& cs, u32 gal,
                        const std::vector<u64*>& digits, u64* Y, cudaStream_t st,
                        const std::vector<FwdJob>* extra = nullptr) {
    const LevelConsts& LC = C->lc(level);
    const u32 N = C->N, ext = level + C->K, beta = C->beta(level);
    const u32 cnt = (u32)cs.size();
    std::vector<InvJob> ij;
    ij.reserve((size_t)cnt * level);
    for (u32 p = 0; p < cnt; p++) {
        u64* Yp = Y + (size_t)p * level * N;
        for (u32 j = 0; j < level; j++)
            ij.push_back(InvJob{cs[p] + (size_t)j * N, Yp + (size_t)j * N, Yp + (size_t)j * N, LC.dec_c[j], LC.dec_sh[j],
                                j, gal});
    }
    launch_inv_ntt(C->T, ij.data(), (int)ij.size(), st);
    std::vector<FwdJob> fj;
    for (u32 p = 0; p < cnt; p++) {
        u64* Yp = Y + (size_t)p * level * N;
        for (u32 b = 0; b < beta; b++) {
            const u32 first = b * C->alpha, n = std::min(C->alpha, level - first);
            // the digit's words are canonical residues of its moduli: below 2^41 if every one is
            bool small = true;
            for (u32 j = first; j < first + n; j++) small = small && C->mods[j] < (1ull << 41);
            for (u32 t = 0; t < ext; t++) {
                if (t >= first && t < first + n) continue;
                fj.push_back(FwdJob{Yp + (size_t)first * N, digits[p] + ((size_t)b * ext + t) * N,
                                    LC.dec_tab + ((size_t)b * ext + t) * C->alpha, nullptr, nullptr, 0, 0,
                                    C->gmod(level, t), n | (small ? 1u << 16 : 0u)});
            }
        }
        // each digit's own limbs are the (gathered) input limbs: copy jobs in the same launch, after
        // the polynomial's transforms, so that they fill the transforms' last wave
        for (u32 b = 0; b < beta; b++) {
            const u32 first = b * C->alpha, n = std::min(C->alpha, level - first);
            for (u32 j = first; j < first + n; j++)
                fj.push_back(FwdJob{cs[p] + (size_t)j * N, digits[p] + ((size_t)b * ext + j) * N, nullptr, nullptr,
                                    nullptr, gal, 0, j, FWD_COPY});
        }
    }
    if (extra) fj.insert(fj.end(), extra->begin(), extra->end());
    launch_fwd_ntt(C->T, fj.data(), (int)fj.size(), st);
}

void op_decompose(ckks_ctx* C, u32 level, const u64* c, u32 gal, u64* digits, u64* Y, cudaStream_t st,
                  const std::vector<FwdJob>* extra = nullptr) {
    op_decompose_batch(C, level, std::vector<const u64*>{c}, gal, std::vector<u64*>{digits}, Y, st, extra);
}

// Modulus switch down of `count` polynomials over a contiguous source run:
// INTT the sources (scaled), basis-convert to the targets 0..ntgt-1 fused into
// the forward NTT, and finish with out = (x_j - conv_j) * inv_j (Eq. 4 / Eq. 1).
// Y: scratch [count][ns][N].
void op_down_batch(ckks_ctx* C, const std::vector<const u64*>& xs, u32 src_first, const std::vector<u32>& src_g,
                   const std::vector<u64>& sc, const std::vector<u64>& ssh, const u64* tab, u32 ntgt,
                   const std::vector<u64>& inv, const std::vector<u64>& inv_sh, const std::vector<u64*>& outs, u64* Y,
                   cudaStream_t st) {
    const u32 N = C->N, ns = (u32)src_g.size(), cnt = (u32)xs.size();
    std::vector<InvJob> ij;
    for (u32 p = 0; p < cnt; p++)
        for (u32 i = 0; i < ns; i++) {
            u64* y = Y + ((size_t)p * ns + i) * N;
            ij.push_back(InvJob{xs[p] + (size_t)(src_first + i) * N, y, y, sc[i], ssh[i], src_g[i], 0});
        }
    launch_inv_ntt(C->T, ij.data(), (int)ij.size(), st);
    std::vector<FwdJob> fj;
    for (u32 p = 0; p < cnt; p++)
        for (u32 j = 0; j < ntgt; j++)
            fj.push_back(FwdJob{Y + (size_t)p * ns * N, outs[p] + (size_t)j * N, tab + (size_t)j * ns,
                                xs[p] + (size_t)j * N, outs[p] + (size_t)j * N, inv[j], inv_sh[j], j, ns});
    launch_fwd_ntt(C->T, fj.data(), (int)fj.size(), st);
}

void op_moddown_batch(ckks_ctx* C, u32 level, const std::vector<const u64*>& xs, const std::vector<u64*>& outs,
                      u64* Y, cudaStream_t st) {
    const LevelConsts& LC = C->lc(level);
    std::vector<u32> g;
    for (u32 i = 0; i < C->K; i++) g.push_back(C->L + i);
    op_down_batch(C, xs, level, g, LC.md_c, LC.md_sh, LC.md_tab, level, LC.md_pinv, LC.md_pinv_sh, outs, Y, st);
}

void op_moddown(ckks_ctx* C, u32 level, const u64* x, u64* out, u64* Y, cudaStream_t st) {
    op_moddown_batch(C, level, std::vector<const u64*>{x}, std::vector<u64*>{out}, Y, st);
}

void op_moddown_rescale_batch(ckks_ctx* C, u32 level, const std::vector<const u64*>& xs,
                              const std::vector<u64*>& outs, u64* Y, cudaStream_t st) {
    const LevelConsts& LC = C->lc(level);
    std::vector<u32> g{level - 1};
    for (u32 i = 0; i < C->K; i++) g.push_back(C->L + i);
    op_down_batch(C, xs, level - 1, g, LC.mdr_c, LC.mdr_sh, LC.mdr_tab, level - 1, LC.mdr_pinv, LC.mdr_pinv_sh, outs,
                  Y, st);
}

void op_moddown_rescale(ckks_ctx* C, u32 level, const u64* x, u64* out, u64* Y, cudaStream_t st) {
    op_moddown_rescale_batch(C, level, std::vector<const u64*>{x}, std::vector<u64*>{out}, Y, st);
}

void op_rescale_batch(ckks_ctx* C, u32 level, const std::vector<const u64*>& xs, const std::vector<u64*>& outs,
                      u64* Y, cudaStream_t st) {
    const LevelConsts& LC = C->lc(level);
    op_down_batch(C, xs, level - 1, std::vector<u32>{level - 1}, LC.rs_c, LC.rs_sh, LC.rs_tab, level - 1, LC.rs_inv,
                  LC.rs_inv_sh, outs, Y, st);
}

void op_rescale(ckks_ctx* C, u32 level, const u64* x, u64* out, u64* Y, cudaStream_t st) {
    op_rescale_batch(C, level, std::vector<const u64*>{x}, std::vector<u64*>{out}, Y, st);
}

const u64* key_of(ckks_ctx* C, int64_t r) {
    auto it = C->keys.find(C->rotkey(r));
    if (it == C->keys.end()) fail(CKKS_ENOKEY, "missing rotation key for r = " + std::to_string(C->rotkey(r)));
    return it->second;
}

void op_ks_inner(ckks_ctx* C, u32 level, const u64* digits, const u64* key, u32 gal, const u64* x0, int x0_mode,
                 u64* out0, u64* out1, int acc, cudaStream_t st) {
    KsArgs a{};
    a.digits = digits;
    a.key = key;
    a.x0 = x0;
    a.out0 = out0;
    a.out1 = out1;
    a.mods = (const ModC*)C->d_mods.p;
    a.lift_c = C->d_lift.p;
    a.lift_sh = C->d_lift_sh.p;
    a.level = level;
    a.ext = level + C->K;
    a.L = C->L;
    a.beta = C->beta(level);
    a.beta_max = C->beta_max;
    a.gal = gal;
    a.x0_mode = x0 ? x0_mode : 0;
    a.accumulate = acc;
    a.log_n = C->log_n;
    launch_ks_inner(a, st);
}

void op_add_gather(ckks_ctx* C, u32 nlimbs, u32 level, const u64* a, const u64* b, u64* out, u32 gal, int acc,
                   cudaStream_t st) {
    std::vector<AddJob> j(nlimbs);
    for (u32 t = 0; t < nlimbs; t++)
        j[t] = AddJob{a + (size_t)t * C->N, b ? b + (size_t)t * C->N : nullptr, out + (size_t)t * C->N,
                      C->gmod(level, t), 0};
    launch_add_gather((const ModC*)C->d_mods.p, j.data(), (int)nlimbs, gal, acc, C->log_n, st);
}

// Tile of the diagonal kernel (0 = default; see DiagMacArgs).
struct K6Tile {
    u32 k3 = 0, run = 0;
};

DiagMacArgs dm_base(ckks_ctx* C, u32 level, bool with_p, const ckks_diags* f, K6Tile tile = K6Tile{}) {
    DiagMacArgs a;
    memset(&a, 0, sizeof(a));
    a.tile_k3 = tile.k3;
    a.tile_run = tile.run;
    a.mods = (const ModC*)C->d_mods.p;
    a.lift_c = C->d_lift.p;
    a.lift_sh = C->d_lift_sh.p;
    a.diags = f->d;
    a.level = level;
    a.ext = level + (with_p ? C->K : 0);
    a.L = C->L;
    a.k_p = C->K;
    a.beta = C->beta(level);
    a.log_n = C->log_n;
    a.diag_level = f->level;
    a.err = (u32*)C->d_err.p;
    a.wait_ns = C->dbg_wait_ns;
    a.starve_step = C->dbg_starve_step;
    a.batch = 1;
    return a;
}

// ------------------------------------------------------------------ the four schedules
struct LtIO {
    const u64* c0;
    const u64* c1;
    u64* o0;
    u64* o1;
};

// The outermost rotation layer of a schedule: amounts offset0 + stride * step * k
// (mod N/2) for k < count.  Offsets o_t = offset0 + stride t give
//   sum_t f_t . Rot(z, o_t) = sum_k Rot( sum_t' f^_t' . Rot(z, stride t'), amount_k )
// with f^ = Rot(f, -amount_k), so the base offset0 joins this layer (every k,
// the first included).  An amount of 0 needs no key; at most one k has it,
// since the amounts differ by nonzero multiples of stride * step below N/2.
struct OuterLayer {
    std::vector<int64_t> amount;  // in [0, N/2)
    std::vector<u32> rotated;     // the k with a nonzero amount, ascending
    int identity = -1;            // the k with amount 0, or -1
};

OuterLayer outer_layer(const ckks_ctx* C, const ckks_diags* f, int64_t step, u32 count) {
    OuterLayer o;
    for (u32 k = 0; k < count; k++) {
        const int64_t r = C->rotkey((int64_t)f->offset0 + (int64_t)f->stride * step * k);
        o.amount.push_back(r);
        if (r) o.rotated.push_back(k);
        else if (o.identity < 0) o.identity = (int)k;
    }
    return o;
}

// TH-BSGS, Algorithm 2 (n1, n2, n3 = n'1, n'2, n'3).  DH-BSGS (Algorithm 1)
// is the case n1 = 1 with (n2, n3) = (n1, n2) of Algorithm 1, and the hoisted
// diagonal method the case (1, D, 1): the three share this schedule and give
// identical residues for those splits.
void sched_th(ckks_ctx* C, u32 level, LtIO io, const ckks_diags* f, u32 n1, u32 n2, u32 n3, cudaStream_t st,
              K6Tile tile = K6Tile{}) {
    const u32 N = C->N, ext = level + C->K, beta = C->beta(level);
    const int64_t s = f->stride;
    Arena ar(st, N);
    const u32 nb = std::max<u32>(1, std::max(n1 - 1, n3));  // widest batch of the key-switch phases
    u64* Y = ar.limbs(std::max<size_t>((size_t)nb * level, 2 * (C->K + 1)));
    std::vector<u64*> A(n1, nullptr), B(n1, nullptr), Dg(n1, nullptr);
    Dg[0] = ar.limbs((size_t)beta * ext);
    // P c0 once (line 2), read by every middle-layer step of the first baby index: scaling jobs
    // of the line-1 Decompose's forward launch
    u64* c0l = ar.limbs(level);
    std::vector<FwdJob> lift_jobs;
    for (u32 t = 0; t < level; t++)
        lift_jobs.push_back(FwdJob{io.c0 + (size_t)t * N, c0l + (size_t)t * N, nullptr, nullptr, nullptr,
                                   C->lift_c[t], C->lift_sh[t], t, FWD_COPY | FWD_SCALE});
    op_decompose(C, level, io.c1, 0, Dg[0], Y, st, &lift_jobs);  // line 1
    for (u32 i = 1; i < n1; i++) {                     // lines 2-5 (the lift is fused)
        const int64_t r = s * i;
        A[i] = ar.limbs(ext);
        B[i] = ar.limbs(ext);
        op_ks_inner(C, level, Dg[0], key_of(C, r), C->galois(r), io.c0, 2, A[i], B[i], 0, st);
    }
    if (n2 > 1 && n1 > 1) {  // lines 6-7 for every i at once
        std::vector<const u64*> bs, tqc;
        std::vector<u64*> tq, dg;
        for (u32 i = 1; i < n1; i++) {
            bs.push_back(B[i]);
            tq.push_back(ar.limbs(level));
            tqc.push_back(tq.back());
            Dg[i] = ar.limbs((size_t)beta * ext);
            dg.push_back(Dg[i]);
        }
        op_moddown_batch(C, level, bs, tq, Y, st);
        op_decompose_batch(C, level, tqc, 0, dg, Y, st);
    }
    DiagMacArgs a = dm_base(C, level, true, f, tile);
    a.n1 = n1;
    a.n2 = n2;
    a.n3 = n3;
    a.lift0 = 1;
    a.A[0] = io.c0;
    a.B[0] = io.c1;
    a.c0[0] = io.c0;
    a.c1[0] = io.c1;
    a.c0l[0] = c0l;
    for (u32 i = 1; i < n1; i++) a.A[i] = A[i], a.B[i] = B[i];
    for (u32 i = 0; i < n1; i++) a.Dg[i] = Dg[i];
    for (u32 j = 1; j < n2; j++) {
        a.keys[j] = key_of(C, s * n1 * j);
        a.gal_mid[j] = C->galois(s * n1 * j);
    }
    const OuterLayer ol = outer_layer(C, f, (int64_t)n1 * n2, n3);
    std::vector<u64*> U0(n3), U1(n3);
    for (u32 k = 0; k < n3; k++) {
        U0[k] = ar.limbs(ext);
        U1[k] = ar.limbs(ext);
        a.U0[k] = U0[k];
        a.U1[k] = U1[k];
        a.gal_diag[k] = ol.amount[k] ? C->galois(-ol.amount[k]) : 0;
    }
    launch_diag_mac(a, st);  // lines 8-14
    // the accumulator: the partial sum whose outer amount is 0, else zeros
    u64* acc0 = ol.identity >= 0 ? U0[ol.identity] : ar.limbs(ext);
    u64* acc1 = ol.identity >= 0 ? U1[ol.identity] : ar.limbs(ext);
    if (ol.identity < 0) {
        CK(cudaMemsetAsync(acc0, 0, (size_t)ext * N * sizeof(u64), st));
        CK(cudaMemsetAsync(acc1, 0, (size_t)ext * N * sizeof(u64), st));
    }
    if (!ol.rotated.empty()) {  // lines 15-18 for every rotated k at once
        std::vector<const u64*> us, tqc;
        std::vector<u64*> tq, dk;
        for (u32 k : ol.rotated) {
            us.push_back(U1[k]);
            tq.push_back(ar.limbs(level));
            tqc.push_back(tq.back());
            dk.push_back(ar.limbs((size_t)beta * ext));
        }
        op_moddown_batch(C, level, us, tq, Y, st);
        op_decompose_batch(C, level, tqc, 0, dk, Y, st);
        for (size_t c0 = 0; c0 < ol.rotated.size(); c0 += KS_MAX_MULTI) {
            KsMultiArgs m;
            memset(&m, 0, sizeof(m));
            m.count = (u32)std::min<size_t>(KS_MAX_MULTI, ol.rotated.size() - c0);
            for (u32 c = 0; c < m.count; c++) {
                const u32 k = ol.rotated[c0 + c];
                m.digits[c] = dk[c0 + c];
                m.keys[c] = key_of(C, ol.amount[k]);
                m.x0[c] = U0[k];
                m.gal[c] = C->galois(ol.amount[k]);
            }
            m.out0 = acc0;
            m.out1 = acc1;
            m.mods = (const ModC*)C->d_mods.p;
            m.level = level;
            m.ext = ext;
            m.L = C->L;
            m.beta = beta;
            m.log_n = C->log_n;
            launch_ks_multi(m, st);
        }
    }
    op_moddown_rescale_batch(C, level, std::vector<const u64*>{acc0, acc1}, std::vector<u64*>{io.o0, io.o1}, Y,
                             st);  // line 19
}

// TH-BSGS (and its DH / diagonal special cases) for a batch of ciphertexts at
// one level that share the diagonals, the keys and the split.  Every step runs
// once for the whole batch: the Decompose/ModDown launches take every
// ciphertext's limbs, the inner-layer key products go out as one launch with
// the ciphertexts of each key adjacent, and K6 runs with a batch dimension so
// that each diagonal and key word is fetched from HBM once for the batch.
// The results are identical to per-ciphertext sched_th.
void sched_th_batch(ckks_ctx* C, u32 level, const std::vector<LtIO>& ios, const ckks_diags* f, u32 n1, u32 n2,
                    u32 n3, cudaStream_t st, K6Tile tile = K6Tile{}) {
    const u32 N = C->N, ext = level + C->K, beta = C->beta(level);
    const u32 nbat = (u32)ios.size();
    const size_t dig = (size_t)beta * ext;  // limbs of one digit set
    const int64_t s = f->stride;
    Arena ar(st, N);
    const u32 nb = std::max<u32>(1, std::max(n1 - 1, n3)) * nbat;
    u64* Y = ar.limbs(std::max<size_t>((size_t)std::max(nb, nbat) * level, 2ull * nbat * (C->K + 1)));
    u64* Aall = ar.limbs((size_t)nbat * n1 * ext);  // [b][i][ext]; i = 0 unused (lifted input)
    u64* Ball = ar.limbs((size_t)nbat * n1 * ext);
    u64* Dall = ar.limbs((size_t)nbat * n1 * dig);  // [b][i][beta][ext]
    u64* Uall = ar.limbs((size_t)nbat * n3 * 2 * ext);  // [b][k][c][ext]
    auto Ap = [&](u32 b, u32 i) { return Aall + ((size_t)b * n1 + i) * ext * N; };
    auto Bp = [&](u32 b, u32 i) { return Ball + ((size_t)b * n1 + i) * ext * N; };
    auto Dp = [&](u32 b, u32 i) { return Dall + ((size_t)b * n1 + i) * dig * N; };
    auto Up = [&](u32 b, u32 k, u32 c) { return Uall + (((size_t)b * n3 + k) * 2 + c) * ext * N; };
    {  // line 1
        std::vector<const u64*> cs;
        std::vector<u64*> ds;
        for (u32 b = 0; b < nbat; b++) cs.push_back(ios[b].c1), ds.push_back(Dp(b, 0));
        op_decompose_batch(C, level, cs, 0, ds, Y, st);
    }
    if (n1 > 1) {  // lines 2-5, every (i, b) in launches of KS_MAX_BATCH products
        std::vector<KsBatchEntry> es;
        for (u32 i = 1; i < n1; i++)
            for (u32 b = 0; b < nbat; b++) {
                const int64_t r = s * i;
                es.push_back(KsBatchEntry{Dp(b, 0), key_of(C, r), ios[b].c0, Ap(b, i), Bp(b, i), C->galois(r), 0});
            }
        for (size_t e0 = 0; e0 < es.size(); e0 += KS_MAX_BATCH) {
            KsBatchArgs k;
            memset(&k, 0, sizeof(k));
            k.count = (u32)std::min<size_t>(KS_MAX_BATCH, es.size() - e0);
            for (u32 c = 0; c < k.count; c++) k.e[c] = es[e0 + c];
            k.mods = (const ModC*)C->d_mods.p;
            k.lift_c = C->d_lift.p;
            k.lift_sh = C->d_lift_sh.p;
            k.level = level;
            k.ext = ext;
            k.L = C->L;
            k.beta = beta;
            k.log_n = C->log_n;
            launch_ks_batch(k, st);
        }
    }
    if (n2 > 1 && n1 > 1) {  // lines 6-7
        std::vector<const u64*> bs, tqc;
        std::vector<u64*> tq, dg;
        for (u32 b = 0; b < nbat; b++)
            for (u32 i = 1; i < n1; i++) {
                bs.push_back(Bp(b, i));
                tq.push_back(ar.limbs(level));
                tqc.push_back(tq.back());
                dg.push_back(Dp(b, i));
            }
        op_moddown_batch(C, level, bs, tq, Y, st);
        op_decompose_batch(C, level, tqc, 0, dg, Y, st);
    }
    DiagMacArgs a = dm_base(C, level, true, f, tile);
    a.n1 = n1;
    a.n2 = n2;
    a.n3 = n3;
    a.lift0 = 1;
    a.batch = nbat;
    for (u32 b = 0; b < nbat; b++) a.c0[b] = ios[b].c0, a.c1[b] = ios[b].c1;
    {  // P c0 once per ciphertext (line 2)
        std::vector<const u64*> cin;
        std::vector<u64*> cout;
        u64* c0l = ar.limbs((size_t)nbat * level);
        for (u32 b = 0; b < nbat; b++) {
            cin.push_back(ios[b].c0);
            cout.push_back(c0l + (size_t)b * level * N);
            a.c0l[b] = cout.back();
        }
        launch_lift((const ModC*)C->d_mods.p, C->d_lift.p, C->d_lift_sh.p, cin.data(), cout.data(), nbat, level,
                    C->log_n, st);
    }
    for (u32 i = 0; i < n1; i++) a.A[i] = Ap(0, i), a.B[i] = Bp(0, i), a.Dg[i] = Dp(0, i);
    a.bs_ab = (u64)n1 * ext * N;
    a.bs_dg = (u64)n1 * dig * N;
    a.bs_u = (u64)n3 * 2 * ext * N;
    for (u32 j = 1; j < n2; j++) {
        a.keys[j] = key_of(C, s * n1 * j);
        a.gal_mid[j] = C->galois(s * n1 * j);
    }
    const OuterLayer ol = outer_layer(C, f, (int64_t)n1 * n2, n3);
    for (u32 k = 0; k < n3; k++) {
        a.U0[k] = Up(0, k, 0);
        a.U1[k] = Up(0, k, 1);
        a.gal_diag[k] = ol.amount[k] ? C->galois(-ol.amount[k]) : 0;
    }
    launch_diag_mac(a, st);  // lines 8-14
    // per ciphertext: the accumulator is its partial sum with outer amount 0, else zeros
    u64* Zall = nullptr;
    if (ol.identity < 0) {
        Zall = ar.limbs((size_t)nbat * 2 * ext);
        CK(cudaMemsetAsync(Zall, 0, (size_t)nbat * 2 * ext * N * sizeof(u64), st));
    }
    auto Acc = [&](u32 b, u32 c) {
        return ol.identity >= 0 ? Up(b, (u32)ol.identity, c) : Zall + ((size_t)b * 2 + c) * ext * N;
    };
    const size_t nrot = ol.rotated.size();
    if (nrot) {  // lines 15-18
        std::vector<const u64*> us, tqc;
        std::vector<u64*> tq, dk;
        for (u32 b = 0; b < nbat; b++)
            for (u32 k : ol.rotated) {
                us.push_back(Up(b, k, 1));
                tq.push_back(ar.limbs(level));
                tqc.push_back(tq.back());
                dk.push_back(ar.limbs(dig));
            }
        op_moddown_batch(C, level, us, tq, Y, st);
        op_decompose_batch(C, level, tqc, 0, dk, Y, st);
        for (u32 b = 0; b < nbat; b++)
            for (size_t c0 = 0; c0 < nrot; c0 += KS_MAX_MULTI) {
                KsMultiArgs m;
                memset(&m, 0, sizeof(m));
                m.count = (u32)std::min<size_t>(KS_MAX_MULTI, nrot - c0);
                for (u32 c = 0; c < m.count; c++) {
                    const u32 k = ol.rotated[c0 + c];
                    m.digits[c] = dk[(size_t)b * nrot + c0 + c];
                    m.keys[c] = key_of(C, ol.amount[k]);
                    m.x0[c] = Up(b, k, 0);
                    m.gal[c] = C->galois(ol.amount[k]);
                }
                m.out0 = Acc(b, 0);
                m.out1 = Acc(b, 1);
                m.mods = (const ModC*)C->d_mods.p;
                m.level = level;
                m.ext = ext;
                m.L = C->L;
                m.beta = beta;
                m.log_n = C->log_n;
                launch_ks_multi(m, st);
            }
    }
    std::vector<const u64*> xs;
    std::vector<u64*> outs;
    for (u32 b = 0; b < nbat; b++) {
        xs.push_back(Acc(b, 0));
        outs.push_back(ios[b].o0);
        xs.push_back(Acc(b, 1));
        outs.push_back(ios[b].o1);
    }
    op_moddown_rescale_batch(C, level, xs, outs, Y, st);  // line 19
}

// BSGS, Eq. (5): un-hoisted rotations (each with its own Decompose of the
// rotated c1 and two ModDowns), products over Q, plain rescale at the end.
void sched_bsgs(ckks_ctx* C, u32 level, LtIO io, const ckks_diags* f, u32 n1, u32 n2, cudaStream_t st,
                K6Tile tile = K6Tile{}) {
    const u32 N = C->N, ext = level + C->K, beta = C->beta(level);
    const int64_t s = f->stride;
    Arena ar(st, N);
    u64* Y = ar.limbs(std::max(level, C->K + 1));
    u64* D = ar.limbs((size_t)beta * ext);
    u64* X0 = ar.limbs(ext);
    u64* X1 = ar.limbs(ext);
    u64* T0 = ar.limbs(level);
    auto rotate_into = [&](const u64* c0, const u64* c1, int64_t r, u64* o0, u64* o1, int acc) {
        const u32 g = C->galois(r);
        op_decompose(C, level, c1, g, D, Y, st);
        op_ks_inner(C, level, D, key_of(C, r), 0, nullptr, 0, X0, X1, 0, st);
        op_moddown(C, level, X0, T0, Y, st);
        if (acc) {
            op_add_gather(C, level, level, c0, T0, o0, g, 1, st);
            op_moddown(C, level, X1, X0, Y, st);  // reuse X0 as [level] scratch
            op_add_gather(C, level, level, X0, nullptr, o1, 0, 1, st);
        } else {
            op_add_gather(C, level, level, c0, T0, o0, g, 0, st);
            op_moddown(C, level, X1, o1, Y, st);
        }
    };
    DiagMacArgs a = dm_base(C, level, false, f, tile);
    a.n1 = n1;
    a.n2 = 1;
    a.n3 = n2;
    a.A[0] = io.c0;
    a.B[0] = io.c1;
    for (u32 i = 1; i < n1; i++) {
        u64* c0 = ar.limbs(level);
        u64* c1 = ar.limbs(level);
        rotate_into(io.c0, io.c1, s * i, c0, c1, 0);
        a.A[i] = c0;
        a.B[i] = c1;
    }
    const OuterLayer ol = outer_layer(C, f, n1, n2);
    std::vector<u64*> V0(n2), V1(n2);
    for (u32 j = 0; j < n2; j++) {
        V0[j] = ar.limbs(level);
        V1[j] = ar.limbs(level);
        a.U0[j] = V0[j];
        a.U1[j] = V1[j];
        a.gal_diag[j] = ol.amount[j] ? C->galois(-ol.amount[j]) : 0;
    }
    launch_diag_mac(a, st);
    u64* acc0 = ol.identity >= 0 ? V0[ol.identity] : ar.limbs(level);
    u64* acc1 = ol.identity >= 0 ? V1[ol.identity] : ar.limbs(level);
    if (ol.identity < 0) {
        CK(cudaMemsetAsync(acc0, 0, (size_t)level * N * sizeof(u64), st));
        CK(cudaMemsetAsync(acc1, 0, (size_t)level * N * sizeof(u64), st));
    }
    for (u32 j : ol.rotated) rotate_into(V0[j], V1[j], ol.amount[j], acc0, acc1, 1);
    op_rescale(C, level, acc0, io.o0, Y, st);
    op_rescale(C, level, acc1, io.o1, Y, st);
}

void validate_split(lt_algo algo, u32 D, const lt_split& sp) {
    switch (algo) {
        case LT_DIAG: break;
        case LT_BSGS:
        case LT_DH_BSGS:
            if (sp.n1 < 1 || sp.n2 < 1 || (sp.n3 != 1 && sp.n3 != 0) || sp.n1 * sp.n2 != D)
                fail(CKKS_EINVAL, "BSGS/DH split needs n1*n2 = n_diag and n3 = 1");
            if (sp.n1 > (u32)DM_MAX_N1 || sp.n2 > (u32)DM_MAX_N3) fail(CKKS_EINVAL, "split exceeds kernel limits");
            break;
        case LT_TH_BSGS:
            if (sp.n1 < 1 || sp.n2 < 1 || sp.n3 < 1 || sp.n1 * sp.n2 * sp.n3 != D)
                fail(CKKS_EINVAL, "TH split needs n1*n2*n3 = n_diag");
            if (sp.n1 > (u32)DM_MAX_N1 || sp.n2 > (u32)DM_MAX_N2 || sp.n3 > (u32)DM_MAX_N3)
                fail(CKKS_EINVAL, "split exceeds kernel limits");
            break;
        default: fail(CKKS_EINVAL, "unknown algorithm");
    }
    if (algo == LT_DIAG && D > (u32)DM_MAX_N2) fail(CKKS_EINVAL, "too many diagonals for the diagonal method");
}

// Rotation amounts (in [1, N/2)) whose keys an LT over offsets
// offset0 + stride t needs with this split; the outermost layer carries offset0.
std::vector<int64_t> rotations(const ckks_ctx* C, lt_algo algo, const lt_split& sp, u32 D, int64_t stride,
                               int64_t offset0) {
    std::vector<int64_t> r;
    auto add = [&](int64_t x) {
        x = C->rotkey(x);
        if (x) r.push_back(x);
    };
    if (algo == LT_DIAG) {
        for (u32 t = 1; t < D; t++) add(stride * t);
        add(offset0);
    } else if (algo == LT_BSGS || algo == LT_DH_BSGS) {
        for (u32 i = 1; i < sp.n1; i++) add(stride * i);
        for (u32 j = 0; j < sp.n2; j++) add(offset0 + stride * sp.n1 * j);
    } else {
        for (u32 i = 1; i < sp.n1; i++) add(stride * i);
        for (u32 j = 1; j < sp.n2; j++) add(stride * sp.n1 * j);
        for (u32 k = 0; k < sp.n3; k++) add(offset0 + stride * sp.n1 * sp.n2 * k);
    }
    return r;
}

std::vector<int64_t> rotations(const ckks_ctx* C, lt_algo algo, const lt_split& sp, const ckks_diags* f) {
    return rotations(C, algo, sp, f->n_diag, f->stride, f->offset0);
}

}  // namespace

// ------------------------------------------------------------------ split choice (autotuner model)
// Time model of one LT on this GPU, phase by phase: the diagonal kernel K6 at
// the slower of its DRAM bytes and its multiply-accumulates, the key-switch
// inner products at their DRAM bytes, and the Decompose / ModDown transforms
// at their NTT butterflies.  The split with the smallest estimate wins.
namespace {
// The model over a TH-shaped schedule (n1, n2, n3) = (n'1, n'2, n'3): with
// n2 = 1 there is no middle layer, so neither the baby steps' ModDown and
// Decompose nor the middle keys (Algorithm 1's counts); with n2 > 1 the
// counts of Algorithm 2.
struct ModelEst {
    double bytes, ntt_s, mac_s, seconds;
};
// Rates of this library's kernels on GB300, fitted to LTs measured at N = 2^16,
// level 24, D = 256 over the splits (1,64,4), (2,32,4), (4,16,4), (2,16,8),
// (1,32,8) (time within 3% of each; DRAM bytes within 2% of ncu's per-LT sum
// for (1,64,4), (2,32,4) and (4,8,8)):
//   effective HBM bandwidth of the streaming kernels                6.2e12 B/s
//   K6 multiply-accumulates, 4 or fewer outer indices per CTA       9.5e11 /s
//                            8 outer indices per CTA                7.0e11 /s
//   NTT butterflies (about 1.35 us per 2^16-point limb transform)   3.9e11 /s
//   DRAM traffic of a limb transform: 2.75 limbs (input, the two passes'
//   intermediate mostly through DRAM, output)
constexpr double M_BW = 6.2e12, M_MAC4 = 9.5e11, M_MAC8 = 7.0e11, M_NTT = 5.8e11, M_FIXED = 1e-4;
constexpr double M_NTT_LIMBS = 2.75;

ModelEst model_th_est(const ckks_ctx* C, u32 level, u32 D, u32 n1, u32 n2, u32 n3) {
    const double limb = 8.0 * C->N, ext = level + C->K, beta = (double)((level + C->alpha - 1) / C->alpha);
    const double L = level, K = C->K, N = C->N;
    const bool mid = n2 > 1;
    // K6: diagonals, middle keys, the baby indices' digits (re-read from L2), baby pairs, input, outputs
    u32 k3 = 1;
    while (k3 < n3 && k3 < (u32)DM_MAX_K3) k3 *= 2;
    const double blocks = (n3 + k3 - 1) / k3;
    const double k6_bytes = limb * (D * ext + (mid ? (n2 - 1.0) * 2 * beta * ext + n1 * beta * ext : 0.0) +
                                    2.0 * (n1 - 1) * ext + 2 * L + 2.0 * n3 * ext);
    const double k6_macs = N * ext * (2.0 * D + (mid ? 2.0 * beta * ((double)n1 * n2 - n1) * blocks : 0.0));
    const double t_k6 = std::max(k6_bytes / M_BW, k6_macs / (k3 >= 8 ? M_MAC8 : M_MAC4));
    // K4: inner layer (n1 - 1 products: digits, key, lifted x0, two outputs) and outer layer
    // (n3 - 1 giant indices: digits, key, x0; the two accumulators once)
    const double k4_bytes =
        limb * ((n1 - 1.0) * (3 * beta * ext + L + 2 * ext) + (n3 - 1.0) * (3 * beta * ext + ext) + 4 * ext);
    // Decompose (inverse of the level limbs, forward of each digit's other limbs) and ModDown
    // (inverse of the k P limbs, forward of the level Q limbs), the last one merged with rescale
    const double dec = 1.0 + (mid ? n1 - 1.0 : 0.0) + (n3 - 1.0);
    const double mdp = (mid ? n1 - 1.0 : 0.0) + (n3 - 1.0);
    const double ntt_limbs = dec * (L + beta * (ext - C->alpha)) + mdp * (K + L) + 2 * (K + L);
    const double ntt_bytes = limb * M_NTT_LIMBS * ntt_limbs;
    ModelEst e{k6_bytes + k4_bytes + ntt_bytes, ntt_limbs * (N / 2) * C->log_n / M_NTT, t_k6, 0};
    e.seconds = t_k6 + k4_bytes / M_BW + e.ntt_s + M_FIXED * N / 65536.0;
    return e;
}
double model_th(const ckks_ctx* C, u32 level, u32 D, u32 n1, u32 n2, u32 n3) {
    return model_th_est(C, level, D, n1, n2, n3).seconds;
}

bool fused_ok(u32 n1, u32 n2) { return n1 <= (u32)DM_MAX_N2 && n2 <= (u32)DM_MAX_N3; }

// DH-BSGS(n1, n2) has two schedules with identical residues: Algorithm 1's
// materialised baby steps, TH(n1, 1, n2), and the baby steps computed on the
// fly in the diagonal kernel's middle layer, TH(1, n1, n2).  The model's pick.
bool dh_fused_model(const ckks_ctx* C, u32 level, u32 D, u32 n1, u32 n2) {
    return fused_ok(n1, n2) && model_th(C, level, D, 1, n1, n2) < model_th(C, level, D, n1, 1, n2);
}

double model_time(const ckks_ctx* C, lt_algo algo, u32 level, u32 D, const lt_split& sp) {
    if (algo == LT_TH_BSGS) return model_th(C, level, D, sp.n1, sp.n2, sp.n3);
    if (algo == LT_DH_BSGS) {
        const double a = model_th(C, level, D, sp.n1, 1, sp.n2);
        return fused_ok(sp.n1, sp.n2) ? std::min(a, model_th(C, level, D, 1, sp.n1, sp.n2)) : a;
    }
    if (algo == LT_DIAG) return model_th(C, level, D, 1, D, 1);
    // BSGS: every rotation un-hoisted (its own Decompose and two ModDowns), products over Q
    const double limb = 8.0 * C->N, ext = level + C->K, beta = (double)((level + C->alpha - 1) / C->alpha);
    const double ntt = (C->N / 2.0) * C->log_n;
    const double keys = sp.n1 + sp.n2 - 2.0;
    const double bytes = limb * (D * level + keys * 2 * beta * ext + 4 * level + keys * beta * ext * 2.0);
    const double flops = keys * (level + beta * (ext - C->alpha)) * ntt + 2 * keys * (C->K + level) * ntt;
    const double mac = (keys * 2 * beta * ext + 2.0 * D * level) * C->N;
    return bytes / M_BW + flops / M_NTT + mac / M_MAC4;
}
}  // namespace

// Every admissible split of D for `algo`, fastest first by the model.
static std::vector<lt_split> ranked_splits(const ckks_ctx* C, lt_algo algo, u32 level, u32 D) {
    std::vector<std::pair<double, lt_split>> all;
    if (algo == LT_DIAG) return {lt_split{1, D, 1}};
    std::vector<u32> divs;
    for (u32 d = 1; d <= D; d++)
        if (D % d == 0) divs.push_back(d);
    for (u32 a : divs)
        for (u32 b : divs) {
            if ((u64)a * b > D || D % ((u64)a * b)) continue;
            lt_split sp;
            if (algo == LT_TH_BSGS) {
                sp = lt_split{a, b, D / (a * b)};
                if (sp.n1 > (u32)DM_MAX_N1 || sp.n3 > (u32)DM_MAX_N3 || sp.n2 > (u32)DM_MAX_N2) continue;
            } else {
                if (a * b != D) continue;
                sp = lt_split{a, b, 1};
                if (sp.n1 > (u32)DM_MAX_N1 || sp.n2 > (u32)DM_MAX_N3) continue;
            }
            all.push_back({model_time(C, algo, level, D, sp), sp});
        }
    std::stable_sort(all.begin(), all.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    std::vector<lt_split> out;
    for (auto& e : all) out.push_back(e.second);
    return out;
}

static lt_split choose_split(const ckks_ctx* C, lt_algo algo, u32 level, u32 D, int32_t stride = 1,
                             int32_t offset0 = 0) {
    if (algo == LT_DIAG) return lt_split{1, D, 1};
    {
        std::lock_guard<std::mutex> g(C->mu);
        auto it = C->tuned.find(std::make_tuple((int)algo, level, D, stride, (int32_t)C->rotkey(offset0)));
        if (it != C->tuned.end()) return it->second;
    }
    std::vector<lt_split> r = ranked_splits(C, algo, level, D);
    return r.empty() ? lt_split{0, 0, 0} : r[0];
}

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* ckks_last_error(void) { return g_err.c_str(); }

// Reads (and clears) the context's device error word: nonzero means a bounded
// device-side wait gave up, so results computed since the last check are void.
static void check_device_flag(ckks_ctx* ctx) {
    uint32_t flag = 0;
    CK(cudaMemcpy(&flag, ctx->d_err.p, 4, cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(ctx->d_err.p, 0, 4));
        fail(CKKS_ETIMEOUT, "a bounded device-side wait gave up; results since the last check are void");
    }
}

ckks_status ckks_device_status(ckks_ctx* ctx) {
    return guarded([&] {
        if (!ctx) fail(CKKS_EINVAL, "null argument");
        CK(cudaSetDevice(ctx->device));
        CK(cudaDeviceSynchronize());
        check_device_flag(ctx);
    });
}

ckks_status ckks_selftest_bounded_wait(ckks_ctx* ctx, uint32_t limit_ms, void* stream) {
    return guarded([&] {
        if (!ctx) fail(CKKS_EINVAL, "null argument");
        if (limit_ms < 1 || limit_ms > 5000) fail(CKKS_EINVAL, "limit must be 1..5000 ms");
        CK(cudaSetDevice(ctx->device));
        launch_wait_selftest((u32*)ctx->d_err.p, (u64)limit_ms * 1000000ull, (cudaStream_t)stream);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_debug_diag_mac_waits(ckks_ctx* ctx, uint64_t wait_limit_ns, uint32_t starve_step) {
    return guarded([&] {
        if (!ctx) fail(CKKS_EINVAL, "null argument");
        if (wait_limit_ns > 5000000000ull) fail(CKKS_EINVAL, "wait limit above 5 s");
        ctx->dbg_wait_ns = wait_limit_ns;
        ctx->dbg_starve_step = starve_step;
    });
}

ckks_status ckks_debug_diag_mac_tile(ckks_ctx* ctx, uint32_t outer_per_cta, uint32_t positions_per_cta) {
    return guarded([&] {
        if (!ctx) fail(CKKS_EINVAL, "null argument");
        if (outer_per_cta & (outer_per_cta - 1) || outer_per_cta > (u32)DM_MAX_K3)
            fail(CKKS_EINVAL, "outer indices per CTA: 0 or a power of two up to 8");
        if (positions_per_cta != 0 && positions_per_cta != 128 && positions_per_cta != 256 && positions_per_cta != 512)
            fail(CKKS_EINVAL, "positions per CTA: 0, 128, 256 or 512");
        ctx->dbg_tile_k3 = outer_per_cta;
        ctx->dbg_tile_run = positions_per_cta;
    });
}

ckks_status ckks_profile_enable(const char* kernel_class, int on) {
    return guarded([&] {
        const int c = prof_class(kernel_class);
        if (c < 0) fail(CKKS_EINVAL, "unknown kernel class");
        prof_enable(c, on != 0);
    });
}

ckks_status ckks_profile_read(const char* kernel_class, double* total_ms, uint64_t* launches) {
    return guarded([&] {
        const int c = prof_class(kernel_class);
        if (c < 0 || !total_ms || !launches) fail(CKKS_EINVAL, "unknown kernel class or null output");
        prof_read(c, total_ms, launches);
    });
}

ckks_status ckks_profile_work(const char* kernel_class, double* macs, double* butterflies) {
    return guarded([&] {
        const int c = prof_class(kernel_class);
        if (c < 0 || !macs || !butterflies) fail(CKKS_EINVAL, "unknown kernel class or null output");
        prof_work(c, macs, butterflies);
    });
}

ckks_status ckks_probe_int_rates(int device, double* macs_per_s, double* butterflies_per_s) {
    return guarded([&] {
        if (!macs_per_s || !butterflies_per_s) fail(CKKS_EINVAL, "null output");
        CK(cudaSetDevice(device));
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        CK(probe_int_rates((u32)sms * 8, macs_per_s, butterflies_per_s));
    });
}

void ckks_profile_reset(void) { prof_reset(); }
uint64_t ckks_kernel_launch_count(void) { return ckks::launches(); }
size_t ckks_device_bytes_in_use(const ckks_ctx* ctx) { return ctx ? ctx->bytes : 0; }

ckks_status ckks_ctx_create(ckks_ctx** out, uint32_t log_n, const uint64_t* q, uint32_t n_q, const uint64_t* p,
                            uint32_t n_p, uint32_t dnum, int device) {
    return guarded([&] {
        if (!out || !q || !p) fail(CKKS_EINVAL, "null argument");
        *out = nullptr;
        if (log_n < 12 || log_n > 16) fail(CKKS_EINVAL, "log_n must be in [12, 16]");
        if (n_q < 2 || n_p < 1 || dnum < 1 || dnum > n_q) fail(CKKS_EINVAL, "need n_q >= 2, n_p >= 1, 1 <= dnum <= n_q");
        auto C = std::make_unique<ckks_ctx>();
        C->device = device;
        C->log_n = log_n;
        C->N = 1u << log_n;
        C->L = n_q;
        C->K = n_p;
        C->dnum = dnum;
        C->alpha = (n_q + dnum - 1) / dnum;
        C->beta_max = (n_q + C->alpha - 1) / C->alpha;
        if (C->alpha > 64 || C->K > 63) fail(CKKS_EINVAL, "alpha and k must be at most 64 and 63");
        for (u32 i = 0; i < n_q; i++) C->mods.push_back(q[i]);
        for (u32 i = 0; i < n_p; i++) C->mods.push_back(p[i]);
        const u64 two_n = 2ull * C->N;
        for (size_t i = 0; i < C->mods.size(); i++) {
            const u64 m = C->mods[i];
            if (m >= (1ull << 60) || m % two_n != 1 || !is_prime_h(m))
                fail(CKKS_EINVAL, "modulus " + std::to_string(i) + " is not a prime = 1 mod 2N below 2^60");
            for (size_t j = 0; j < i; j++)
                if (C->mods[j] == m) fail(CKKS_EINVAL, "moduli must be distinct");
        }
        CK(cudaSetDevice(device));
        cudaMemPool_t pool;
        CK(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        const u32 nm = (u32)C->mods.size(), N = C->N;
        std::vector<ModC> mc(nm);
        std::vector<u64> psi((size_t)nm * N * 2), ipsi((size_t)nm * N * 2);  // (w, Shoup(w)) pairs
        std::vector<u64> lift(nm, 0), lsh(nm, 0);
        for (u32 i = 0; i < nm; i++) {
            const u64 m = C->mods[i];
            mc[i] = modc_h(m);
            // psi = x^((m-1)/2N) for the smallest x >= 2 with psi^N = -1
            u64 w = 0;
            for (u64 x = 2;; x++) {
                w = powmod_h(x, (m - 1) / two_n, m);
                if (powmod_h(w, N, m) == m - 1) break;
            }
            const u64 wi = invmod_h(w, m);
            std::vector<u64> pw(N), ipw(N);
            pw[0] = ipw[0] = 1;
            for (u32 k = 1; k < N; k++) pw[k] = mulmod_h(pw[k - 1], w, m), ipw[k] = mulmod_h(ipw[k - 1], wi, m);
            for (u32 k = 0; k < N; k++) {
                const u32 e = brv_h(k, log_n);
                psi[2 * ((size_t)i * N + k)] = pw[e];
                psi[2 * ((size_t)i * N + k) + 1] = shoup_h(pw[e], m);
                ipsi[2 * ((size_t)i * N + k)] = ipw[e];
                ipsi[2 * ((size_t)i * N + k) + 1] = shoup_h(ipw[e], m);
            }
            if (i < n_q) {
                u64 P = 1;
                for (u32 k = 0; k < n_p; k++) P = mulmod_h(P, p[k] % m, m);
                lift[i] = P;
                lsh[i] = shoup_h(P, m);
            }
        }
        C->d_mods.p = C->dalloc((nm * sizeof(ModC) + 7) / 8);
        CK(cudaMemcpy(C->d_mods.p, mc.data(), nm * sizeof(ModC), cudaMemcpyHostToDevice));
        C->d_psi.p = C->upload(psi);
        C->d_ipsi.p = C->upload(ipsi);
        C->d_err.p = C->dalloc(1);
        CK(cudaMemset(C->d_err.p, 0, 8));
        C->d_lift.p = C->upload(lift);
        C->d_lift_sh.p = C->upload(lsh);
        C->lift_c = lift;
        C->lift_sh = lsh;
        C->T = NttTables{(const ModC*)C->d_mods.p, (const ulonglong2*)C->d_psi.p, (const ulonglong2*)C->d_ipsi.p,
                         log_n};
        *out = C.release();
    });
}

ckks_status ckks_ctx_destroy(ckks_ctx* ctx) {
    return guarded([&] {
        if (!ctx) return;
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto& kv : ctx->keys) cudaFree(kv.second);
        for (auto& kv : ctx->levels) {
            cudaFree(kv.second.dec_tab);
            cudaFree(kv.second.md_tab);
            cudaFree(kv.second.mdr_tab);
            cudaFree(kv.second.rs_tab);
        }
        for (DevBuf* b : {&ctx->d_mods, &ctx->d_psi, &ctx->d_ipsi, &ctx->d_lift, &ctx->d_lift_sh, &ctx->d_err})
            cudaFree(b->p);
        for (auto& kv : ctx->lanes) destroy_lanes(kv.second);
        delete ctx;
    });
}

static void put_key(ckks_ctx* ctx, int32_t r, const uint64_t* src, size_t n_words, cudaMemcpyKind kind,
                    cudaStream_t st) {
    if (!ctx || !src) fail(CKKS_EINVAL, "null argument");
    if (n_words != ctx->key_words()) fail(CKKS_EINVAL, "key size must be beta_max*2*(L+k)*N words");
    CK(cudaSetDevice(ctx->device));
    const u32 rk = ctx->rotkey(r);
    u64* d;
    auto it = ctx->keys.find(rk);
    if (it != ctx->keys.end()) d = it->second;
    else d = ctx->dalloc(n_words);
    ctx->keys[rk] = d;
    // stored with the two components interleaved per word (one 16-byte load per digit word)
    const size_t plane = (size_t)(ctx->L + ctx->K) * ctx->N;
    if (kind == cudaMemcpyHostToDevice) {
        u64* tmp = ctx->dalloc(n_words);
        CK(cudaMemcpy(tmp, src, n_words * 8, kind));
        launch_interleave_key(tmp, d, plane, ctx->beta_max, 0);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        ctx->dfree(tmp, n_words);
    } else {
        launch_interleave_key(src, d, plane, ctx->beta_max, st);
        CK(cudaGetLastError());
    }
}

ckks_status ckks_upload_rotation_key(ckks_ctx* ctx, int32_t r, const uint64_t* host, size_t n_words) {
    return guarded([&] { put_key(ctx, r, host, n_words, cudaMemcpyHostToDevice, 0); });
}

ckks_status ckks_upload_rotation_key_device(ckks_ctx* ctx, int32_t r, const uint64_t* dev, size_t n_words,
                                            void* stream) {
    return guarded([&] { put_key(ctx, r, dev, n_words, cudaMemcpyDeviceToDevice, (cudaStream_t)stream); });
}

int ckks_has_rotation_key(const ckks_ctx* ctx, int32_t r) {
    return ctx && ctx->keys.count(ctx->rotkey(r)) ? 1 : 0;
}

static void put_diags(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0, int32_t stride,
                      uint32_t level, const uint64_t* host, size_t n_words, cudaMemcpyKind kind, cudaStream_t st) {
        if (!ctx || !out || !host) fail(CKKS_EINVAL, "null argument");
        *out = nullptr;
        if (offset0 <= -(int64_t)ctx->slots() || offset0 >= (int64_t)ctx->slots())
            fail(CKKS_EINVAL, "offset0 must lie in (-N/2, N/2)");
        if (stride < 1 || n_diag < 1) fail(CKKS_EINVAL, "need n_diag >= 1 and stride >= 1");
        if ((u64)stride * (n_diag - 1) >= ctx->slots()) fail(CKKS_EINVAL, "offsets exceed N/2");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        if (n_words != (size_t)n_diag * (level + ctx->K) * ctx->N) fail(CKKS_EINVAL, "size mismatch");
        CK(cudaSetDevice(ctx->device));
        auto f = std::make_unique<ckks_diags>();
        f->ctx = ctx;
        f->n_diag = n_diag;
        f->level = level;
        f->offset0 = offset0;
        f->stride = stride;
        f->d = ctx->dalloc(n_words);
        if (kind == cudaMemcpyHostToDevice) CK(cudaMemcpy(f->d, host, n_words * 8, kind));
        else CK(cudaMemcpyAsync(f->d, host, n_words * 8, kind, st));
        *out = f.release();
}

ckks_status ckks_upload_diagonals(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0, int32_t stride,
                                  uint32_t level, const uint64_t* host, size_t n_words) {
    return guarded([&] {
        put_diags(ctx, out, n_diag, offset0, stride, level, host, n_words, cudaMemcpyHostToDevice, 0);
    });
}

ckks_status ckks_upload_diagonals_device(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0,
                                         int32_t stride, uint32_t level, const uint64_t* dev, size_t n_words,
                                         void* stream) {
    return guarded([&] {
        put_diags(ctx, out, n_diag, offset0, stride, level, dev, n_words, cudaMemcpyDeviceToDevice,
                  (cudaStream_t)stream);
    });
}

ckks_status ckks_diags_create(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0, int32_t stride,
                              uint32_t level) {
    return guarded([&] {
        if (!ctx || !out) fail(CKKS_EINVAL, "null argument");
        *out = nullptr;
        if (offset0 <= -(int64_t)ctx->slots() || offset0 >= (int64_t)ctx->slots())
            fail(CKKS_EINVAL, "offset0 must lie in (-N/2, N/2)");
        if (stride < 1 || n_diag < 1) fail(CKKS_EINVAL, "need n_diag >= 1 and stride >= 1");
        if ((u64)stride * (n_diag - 1) >= ctx->slots()) fail(CKKS_EINVAL, "offsets exceed N/2");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        auto f = std::make_unique<ckks_diags>();
        f->ctx = ctx;
        f->n_diag = n_diag;
        f->level = level;
        f->offset0 = offset0;
        f->stride = stride;
        f->d = ctx->dalloc((size_t)n_diag * (level + ctx->K) * ctx->N);
        *out = f.release();
    });
}

ckks_status ckks_diags_write_device(ckks_diags* f, uint32_t first, uint32_t count, const uint64_t* dev,
                                   size_t n_words, void* stream) {
    return guarded([&] {
        if (!f || !dev) fail(CKKS_EINVAL, "null argument");
        const size_t per = (size_t)(f->level + f->ctx->K) * f->ctx->N;
        if ((u64)first + count > f->n_diag) fail(CKKS_EINVAL, "range exceeds n_diag");
        if (n_words != per * count) fail(CKKS_EINVAL, "size mismatch");
        CK(cudaSetDevice(f->ctx->device));
        CK(cudaMemcpyAsync(f->d + per * first, dev, n_words * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    });
}

ckks_status ckks_free_diags(ckks_diags* f) {
    return guarded([&] {
        if (!f) return;
        cudaSetDevice(f->ctx->device);
        f->ctx->dfree(f->d, (size_t)f->n_diag * (f->level + f->ctx->K) * f->ctx->N);
        delete f;
    });
}

ckks_status ckks_ct_create(ckks_ctx* ctx, ckks_ct** out, uint32_t level) {
    return guarded([&] {
        if (!ctx || !out) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        *out = new ckks_ct{ctx, level, ctx->dalloc(2ull * level * ctx->N), true};
    });
}

ckks_status ckks_ct_upload(ckks_ctx* ctx, ckks_ct** out, uint32_t level, const uint64_t* host) {
    ckks_status st = ckks_ct_create(ctx, out, level);
    if (st != CKKS_OK) return st;
    return guarded([&] {
        if (!host) fail(CKKS_EINVAL, "null host buffer");
        CK(cudaMemcpy((*out)->d, host, 2ull * level * ctx->N * 8, cudaMemcpyHostToDevice));
    });
}

ckks_status ckks_ct_wrap_device(ckks_ctx* ctx, ckks_ct** out, uint32_t level, uint64_t* dev_ptr) {
    return guarded([&] {
        if (!ctx || !out || !dev_ptr) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        *out = new ckks_ct{ctx, level, dev_ptr, false};
    });
}

ckks_status ckks_ct_h2d_async(ckks_ct* ct, const uint64_t* host, size_t n_words, void* stream) {
    return guarded([&] {
        if (!ct || !host) fail(CKKS_EINVAL, "null argument");
        if (n_words != 2ull * ct->level * ct->ctx->N) fail(CKKS_EINVAL, "size mismatch");
        CK(cudaMemcpyAsync(ct->d, host, n_words * 8, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    });
}

ckks_status ckks_ct_d2h_async(const ckks_ct* ct, uint64_t* host, size_t n_words, void* stream) {
    return guarded([&] {
        if (!ct || !host) fail(CKKS_EINVAL, "null argument");
        if (n_words != 2ull * ct->level * ct->ctx->N) fail(CKKS_EINVAL, "size mismatch");
        CK(cudaMemcpyAsync(host, ct->d, n_words * 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    });
}

ckks_status ckks_ct_download(const ckks_ct* ct, uint64_t* host, size_t n_words) {
    return guarded([&] {
        if (!ct || !host) fail(CKKS_EINVAL, "null argument");
        if (n_words != 2ull * ct->level * ct->ctx->N) fail(CKKS_EINVAL, "size mismatch");
        CK(cudaSetDevice(ct->ctx->device));
        CK(cudaDeviceSynchronize());
        check_device_flag(ct->ctx);
        CK(cudaMemcpy(host, ct->d, n_words * 8, cudaMemcpyDeviceToHost));
    });
}

uint32_t ckks_ct_level(const ckks_ct* ct) { return ct ? ct->level : 0; }
uint64_t* ckks_ct_device_ptr(const ckks_ct* ct) { return ct ? ct->d : nullptr; }

ckks_status ckks_free_ct(ckks_ct* ct) {
    return guarded([&] {
        if (!ct) return;
        if (ct->owned) {
            cudaSetDevice(ct->ctx->device);
            ct->ctx->dfree(ct->d, 2ull * ct->level * ct->ctx->N);
        }
        delete ct;
    });
}

int32_t lt_required_rotations(const ckks_ctx* ctx, lt_algo algo, const lt_split* split, uint32_t n_diag,
                              int32_t offset0, int32_t stride, int32_t* rot_out, uint32_t cap) {
    if (!ctx) return -1;
    lt_split sp = split ? *split : lt_split{0, 0, 0};
    if (algo == LT_DIAG) sp = lt_split{1, n_diag, 1};
    if (sp.n3 == 0 && algo != LT_TH_BSGS) sp.n3 = 1;
    try {
        validate_split(algo, n_diag, sp);
    } catch (const Fail&) {
        return -1;
    }
    std::vector<u32> rs;
    for (int64_t r : rotations(ctx, algo, sp, n_diag, stride, offset0)) rs.push_back((u32)r);
    std::sort(rs.begin(), rs.end());
    rs.erase(std::unique(rs.begin(), rs.end()), rs.end());
    u32 n = 0;
    for (u32 r : rs)
        if (n < cap && rot_out) rot_out[n++] = (int32_t)r;
        else n++;
    return (int32_t)std::min<u32>(n, cap);
}

static void lt_eval_impl(ckks_ctx* ctx, const ckks_ct* in, const ckks_diags* f, lt_algo algo, const lt_split* split,
                         ckks_ct* out, cudaStream_t st, lt_split* chosen);

ckks_status lt_model_estimate(const ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag,
                              const lt_split* split, double* hbm_bytes, double* seconds) {
    return guarded([&] {
        if (!ctx || !split || !hbm_bytes || !seconds) fail(CKKS_EINVAL, "null argument");
        if (level < 2 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        lt_split sp = *split;
        if (algo == LT_DIAG) sp = lt_split{1, n_diag, 1};
        if (algo != LT_TH_BSGS && sp.n3 == 0) sp.n3 = 1;
        validate_split(algo, n_diag, sp);
        if (algo == LT_TH_BSGS || algo == LT_DIAG) {
            const ModelEst e = model_th_est(ctx, level, n_diag, sp.n1, sp.n2, sp.n3);
            *hbm_bytes = e.bytes;
            *seconds = e.seconds;
        } else if (algo == LT_DH_BSGS) {
            const bool fz = dh_fused_model(ctx, level, n_diag, sp.n1, sp.n2);
            const ModelEst e = fz ? model_th_est(ctx, level, n_diag, 1, sp.n1, sp.n2)
                                  : model_th_est(ctx, level, n_diag, sp.n1, 1, sp.n2);
            *hbm_bytes = e.bytes;
            *seconds = e.seconds;
        } else {
            *hbm_bytes = -1;
            *seconds = model_time(ctx, algo, level, n_diag, sp);
        }
    });
}

int32_t lt_candidate_splits(const ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag, lt_split* out,
                            uint32_t cap) {
    if (!ctx) return -1;
    const std::vector<lt_split> r = ranked_splits(ctx, algo, level, n_diag);
    uint32_t n = 0;
    for (const lt_split& sp : r) {
        if (n >= cap) break;
        if (out) out[n] = sp;
        n++;
    }
    return (int32_t)n;
}

static lt_split th_form(const ckks_ctx* ctx, u32 level, const ckks_diags* f, lt_algo algo, const lt_split& sp);

ckks_status lt_autotune(ckks_ctx* ctx, lt_algo algo, const ckks_ct* sample, const ckks_diags* f,
                        uint32_t max_candidates, lt_split* chosen, double* best_ms) {
    cudaStream_t st = nullptr;
    ckks_ct* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ckks_status rc = guarded([&] {
        if (!ctx || !sample || !f) fail(CKKS_EINVAL, "null argument");
        const u32 level = sample->level, D = f->n_diag;
        if (level < 2 || level > f->level) fail(CKKS_EINVAL, "bad sample level");
        CK(cudaSetDevice(ctx->device));
        // candidates: the model's ranking, keeping the splits whose keys are all present
        std::vector<lt_split> cand;
        for (const lt_split& sp : ranked_splits(ctx, algo, level, D)) {
            bool ok = true;
            for (int64_t r : rotations(ctx, algo, sp, f))
                if (!ctx->keys.count(ctx->rotkey(r))) ok = false;
            if (ok) cand.push_back(sp);
            if (cand.size() >= std::max<u32>(1, max_candidates)) break;
        }
        if (cand.empty()) fail(CKKS_ENOKEY, "no candidate split has all of its rotation keys");
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        out = new ckks_ct{ctx, level - 1, ctx->dalloc(2ull * (level - 1) * ctx->N), true};
        double best = 1e300;
        lt_split bsp = cand[0];
        auto dh_key = [&](const lt_split& sp) {
            return std::make_tuple(level, D, f->stride, (int32_t)ctx->rotkey(f->offset0), sp.n1, sp.n2);
        };
        for (const lt_split& sp : cand) {
            // DH: both schedules of the split (identical residues), the faster one kept for it
            const int forms = (algo == LT_DH_BSGS && fused_ok(sp.n1, sp.n2)) ? 2 : 1;
            double best_form = 1e300;
            bool fused_best = false;
            for (int fm = 0; fm < forms; fm++) {
                if (algo == LT_DH_BSGS) {
                    std::lock_guard<std::mutex> g(ctx->mu);
                    ctx->dh_fused[dh_key(sp)] = forms == 2 && fm == 1;
                }
                lt_eval_impl(ctx, sample, f, algo, &sp, out, st, nullptr);  // warm-up (tables, attributes)
                CK(cudaEventRecord(e0, st));
                const int reps = 5;  // candidates are often within a few percent of each other
                for (int r = 0; r < reps; r++) lt_eval_impl(ctx, sample, f, algo, &sp, out, st, nullptr);
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms / reps < best_form) best_form = ms / reps, fused_best = forms == 2 && fm == 1;
            }
            if (algo == LT_DH_BSGS) {
                std::lock_guard<std::mutex> g(ctx->mu);
                ctx->dh_fused[dh_key(sp)] = fused_best;
            }
            if (best_form < best) best = best_form, bsp = sp;
        }
        const auto key = std::make_tuple((int)algo, level, D, f->stride, (int32_t)ctx->rotkey(f->offset0));
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            ctx->tuned[key] = bsp;
            ctx->tuned_tile[key] = {0u, 0u};
        }
        // the diagonal kernel's tile for the chosen split: fewer outer indices per CTA
        // (half the default), and the other number of positions per CTA (see launch_ws)
        if (algo != LT_BSGS) {
            const lt_split t = th_form(ctx, level, f, algo, bsp);
            u32 k3 = 1;
            while (k3 < t.n3 && k3 < (u32)DM_MAX_K3) k3 *= 2;
            std::vector<std::pair<u32, u32>> tiles;
            if (k3 >= 2) tiles.push_back({k3 / 2, 0u});
            tiles.push_back({0u, 256u});
            std::pair<u32, u32> btile{0u, 0u};
            for (const auto& tl : tiles) {
                {
                    std::lock_guard<std::mutex> g(ctx->mu);
                    ctx->tuned_tile[key] = tl;
                }
                lt_eval_impl(ctx, sample, f, algo, &bsp, out, st, nullptr);
                CK(cudaEventRecord(e0, st));
                const int reps = 5;
                for (int r = 0; r < reps; r++) lt_eval_impl(ctx, sample, f, algo, &bsp, out, st, nullptr);
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms / reps < best) best = ms / reps, btile = tl;
            }
            std::lock_guard<std::mutex> g(ctx->mu);
            ctx->tuned_tile[key] = btile;
        }
        if (chosen) *chosen = bsp;
        if (best_ms) *best_ms = best;
    });
    if (out) {
        ctx->dfree(out->d, 2ull * out->level * ctx->N);
        delete out;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) {
        release_lanes(ctx, st);
        cudaStreamDestroy(st);
    }
    return rc;
}

ckks_status lt_autotune_batch(ckks_ctx* ctx, lt_algo algo, uint32_t count, const ckks_ct* const* samples,
                              const ckks_diags* f, uint32_t max_candidates, lt_split* chosen, double* best_ms) {
    cudaStream_t st = nullptr;
    std::vector<ckks_ct*> outs;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ckks_status rc = guarded([&] {
        if (!ctx || !samples || !f || !count) fail(CKKS_EINVAL, "null argument or empty batch");
        const u32 level = samples[0] ? samples[0]->level : 0, D = f->n_diag;
        for (u32 i = 0; i < count; i++)
            if (!samples[i] || samples[i]->ctx != ctx || samples[i]->level != level)
                fail(CKKS_EINVAL, "samples must be ciphertexts of this context at one level");
        if (level < 2 || level > f->level) fail(CKKS_EINVAL, "bad sample level");
        CK(cudaSetDevice(ctx->device));
        std::vector<lt_split> cand;
        for (const lt_split& sp : ranked_splits(ctx, algo, level, D)) {
            bool ok = true;
            for (int64_t r : rotations(ctx, algo, sp, f))
                if (!ctx->keys.count(ctx->rotkey(r))) ok = false;
            if (ok) cand.push_back(sp);
            if (cand.size() >= std::max<u32>(1, max_candidates)) break;
        }
        if (cand.empty()) fail(CKKS_ENOKEY, "no candidate split has all of its rotation keys");
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (u32 i = 0; i < count; i++)
            outs.push_back(new ckks_ct{ctx, level - 1, ctx->dalloc(2ull * (level - 1) * ctx->N), true});
        std::vector<const ckks_diags*> fs(count, f);
        std::vector<lt_algo> al(count, algo);
        double best = 1e300;
        lt_split bsp = cand[0];
        for (const lt_split& sp : cand) {
            std::vector<lt_split> sps(count, sp);
            auto run = [&] {
                const ckks_status r = lt_eval_batch(ctx, count, samples, fs.data(), al.data(), sps.data(),
                                                    outs.data(), st);
                if (r != CKKS_OK) fail(r, "batch evaluation failed while tuning");
            };
            run();  // warm-up (tables, attributes)
            CK(cudaEventRecord(e0, st));
            const int reps = 2;
            for (int r = 0; r < reps; r++) run();
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms / reps < best) best = ms / reps, bsp = sp;
        }
        if (chosen) *chosen = bsp;
        if (best_ms) *best_ms = best;
    });
    for (ckks_ct* o : outs) {
        ctx->dfree(o->d, 2ull * o->level * ctx->N);
        delete o;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) {
        release_lanes(ctx, st);
        cudaStreamDestroy(st);
    }
    return rc;
}

static bool dh_fused(const ckks_ctx* ctx, u32 level, const ckks_diags* f, const lt_split& sp);

int32_t lt_tuned_tile(const ckks_ctx* ctx, lt_algo algo, const ckks_diags* f, uint32_t level, uint32_t* outer_per_cta,
                      uint32_t* positions_per_cta) {
    if (!ctx || !f || !outer_per_cta || !positions_per_cta) return -1;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto tt = ctx->tuned_tile.find(
        std::make_tuple((int)algo, level, f->n_diag, f->stride, (int32_t)ctx->rotkey(f->offset0)));
    if (tt == ctx->tuned_tile.end()) return 0;
    *outer_per_cta = tt->second.first;
    *positions_per_cta = tt->second.second;
    return 1;
}

int32_t lt_dh_schedule(const ckks_ctx* ctx, const ckks_diags* f, uint32_t level, const lt_split* split) {
    if (!ctx || !f || !split || f->ctx != ctx || level < 2 || level > f->level) return -1;
    if (split->n1 < 1 || split->n2 < 1 || (uint64_t)split->n1 * split->n2 != f->n_diag) return -1;
    return dh_fused(ctx, level, f, *split) ? 1 : 0;
}

ckks_status lt_choose_split(ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag, lt_split* out) {
    return guarded([&] {
        if (!ctx || !out) fail(CKKS_EINVAL, "null argument");
        *out = choose_split(ctx, algo, level, n_diag);
        if (out->n1 == 0) fail(CKKS_EINVAL, "no admissible split");
    });
}

// The split an LT of f at `level` runs with (the given one, else the tuned or
// modelled choice), validated, with every rotation key it needs present.
static lt_split resolve_split(ckks_ctx* ctx, u32 level, const ckks_diags* f, lt_algo algo, const lt_split* split) {
    const u32 D = f->n_diag;
    lt_split sp = (split && (split->n1 || split->n2 || split->n3))
                      ? *split
                      : choose_split(ctx, algo, level, D, f->stride, f->offset0);
    if (algo == LT_DIAG) sp = lt_split{1, D, 1};
    if (algo != LT_TH_BSGS && sp.n3 == 0) sp.n3 = 1;
    validate_split(algo, D, sp);
    for (int64_t r : rotations(ctx, algo, sp, f)) key_of(ctx, r);
    return sp;
}

// Whether DH-BSGS(n1, n2) on f at `level` runs with its baby steps fused into
// the diagonal kernel (TH(1, n1, n2)): the measured choice of lt_autotune for
// that shape and split if there is one, else the model's.
static bool dh_fused(const ckks_ctx* ctx, u32 level, const ckks_diags* f, const lt_split& sp) {
    if (!fused_ok(sp.n1, sp.n2)) return false;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->dh_fused.find(
            std::make_tuple(level, f->n_diag, f->stride, (int32_t)ctx->rotkey(f->offset0), sp.n1, sp.n2));
        if (it != ctx->dh_fused.end()) return it->second;
    }
    return dh_fused_model(ctx, level, f->n_diag, sp.n1, sp.n2);
}

// The TH-shaped schedule (n'1, n'2, n'3) a hoisted algorithm runs as: TH as
// given; DH-BSGS(n1, n2) as TH(n1, 1, n2) (Algorithm 1) or TH(1, n1, n2) (baby
// steps fused, identical residues); the hoisted diagonal method as TH(1, D, 1).
static lt_split th_form(const ckks_ctx* ctx, u32 level, const ckks_diags* f, lt_algo algo, const lt_split& sp) {
    switch (algo) {
        case LT_DH_BSGS:
            return dh_fused(ctx, level, f, sp) ? lt_split{1, sp.n1, sp.n2} : lt_split{sp.n1, 1, sp.n2};
        case LT_DIAG: return lt_split{1, f->n_diag, 1};
        default: return sp;
    }
}

// The diagonal kernel's tile for an LT: the one lt_autotune measured for the
// shape when `sp` is the shape's tuned split, else the default.
static K6Tile tile_for(const ckks_ctx* ctx, u32 level, const ckks_diags* f, lt_algo algo, const lt_split& sp) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->dbg_tile_k3 || ctx->dbg_tile_run) return K6Tile{ctx->dbg_tile_k3, ctx->dbg_tile_run};
    const auto key = std::make_tuple((int)algo, level, f->n_diag, f->stride, (int32_t)ctx->rotkey(f->offset0));
    auto it = ctx->tuned.find(key);
    auto tt = ctx->tuned_tile.find(key);
    if (it == ctx->tuned.end() || tt == ctx->tuned_tile.end()) return K6Tile{};
    const lt_split& t = it->second;
    if (t.n1 != sp.n1 || t.n2 != sp.n2 || (algo == LT_TH_BSGS && t.n3 != sp.n3)) return K6Tile{};
    return K6Tile{tt->second.first, tt->second.second};
}

static void dispatch(ckks_ctx* ctx, u32 level, const LtIO& io, const ckks_diags* f, lt_algo algo, const lt_split& sp,
                     cudaStream_t st) {
    const K6Tile tile = tile_for(ctx, level, f, algo, sp);
    if (algo == LT_BSGS) {
        sched_bsgs(ctx, level, io, f, sp.n1, sp.n2, st, tile);
        return;
    }
    const lt_split t = th_form(ctx, level, f, algo, sp);
    sched_th(ctx, level, io, f, t.n1, t.n2, t.n3, st, tile);
}

static void lt_eval_impl(ckks_ctx* ctx, const ckks_ct* in, const ckks_diags* f, lt_algo algo, const lt_split* split,
                         ckks_ct* out, cudaStream_t st, lt_split* chosen) {
    if (!ctx || !in || !f || !out) fail(CKKS_EINVAL, "null argument");
    if (in->ctx != ctx || f->ctx != ctx || out->ctx != ctx) fail(CKKS_EINVAL, "objects of another context");
    const u32 level = in->level;
    if (level < 2) fail(CKKS_EINVAL, "input level must be >= 2");
    if (level > f->level) fail(CKKS_EINVAL, "diagonals encoded below the ciphertext level");
    if (out->level != level - 1) fail(CKKS_EINVAL, "output level must be input level - 1");
    if (out->d == in->d) fail(CKKS_EINVAL, "output must not alias input");
    const lt_split sp = resolve_split(ctx, level, f, algo, split);
    if (chosen) *chosen = sp;
    CK(cudaSetDevice(ctx->device));
    const size_t lw = (size_t)level * ctx->N;
    dispatch(ctx, level, LtIO{in->d, in->d + lw, out->d, out->d + (size_t)(level - 1) * ctx->N}, f, algo, sp, st);
    CK(cudaGetLastError());
}

ckks_status lt_eval(ckks_ctx* ctx, const ckks_ct* in, const ckks_diags* f, lt_algo algo, const lt_split* split,
                    ckks_ct* out, void* stream, lt_split* chosen) {
    return guarded([&] { lt_eval_impl(ctx, in, f, algo, split, out, (cudaStream_t)stream, chosen); });
}

// Validates one LT of a batch and returns its split (as lt_eval would choose it).
static lt_split batch_item_split(ckks_ctx* ctx, const ckks_ct* in, const ckks_diags* f, lt_algo algo,
                                 const lt_split* split, const ckks_ct* out) {
    if (!in || !f || !out) fail(CKKS_EINVAL, "null argument");
    if (in->ctx != ctx || f->ctx != ctx || out->ctx != ctx) fail(CKKS_EINVAL, "objects of another context");
    const u32 level = in->level;
    if (level < 2 || level > f->level || out->level != level - 1) fail(CKKS_EINVAL, "bad levels in the batch");
    if (out->d == in->d) fail(CKKS_EINVAL, "output must not alias input");
    return resolve_split(ctx, level, f, algo, split);
}

ckks_status lt_eval_batch(ckks_ctx* ctx, uint32_t count, const ckks_ct* const* in, const ckks_diags* const* f,
                          const lt_algo* algos, const lt_split* splits, ckks_ct* const* out, void* stream) {
    return guarded([&] {
        if (!ctx || (count && (!in || !f || !out))) fail(CKKS_EINVAL, "null argument");
        cudaStream_t st = (cudaStream_t)stream;
        // validate everything before queuing anything
        struct Item {
            u32 idx;
            lt_algo algo;
            lt_split sp;
        };
        std::vector<Item> items;
        for (u32 i = 0; i < count; i++) {
            const lt_algo algo = algos ? algos[i] : LT_TH_BSGS;
            items.push_back(Item{i, algo, batch_item_split(ctx, in[i], f[i], algo, splits ? &splits[i] : nullptr,
                                                           out[i])});
        }
        CK(cudaSetDevice(ctx->device));
        // group the hoisted LTs by (diagonals, level, split); BSGS runs one by one
        struct Unit {
            double cost;  // model time of the unit's LTs
            std::function<void(cudaStream_t)> run;
        };
        std::vector<Unit> units;
        std::vector<bool> done(count, false);
        for (u32 a = 0; a < count; a++) {
            if (done[a]) continue;
            const Item& ia = items[a];
            const u32 lva = in[ia.idx]->level;
            const double one = model_time(ctx, ia.algo, lva, f[ia.idx]->n_diag, ia.sp);
            if (ia.algo == LT_BSGS) {
                const ckks_ct* ci = in[ia.idx];
                const ckks_diags* fi = f[ia.idx];
                ckks_ct* oi = out[ia.idx];
                const lt_split spi = ia.sp;
                units.push_back(Unit{one, [=](cudaStream_t s) { lt_eval_impl(ctx, ci, fi, LT_BSGS, &spi, oi, s, nullptr); }});
                done[a] = true;
                continue;
            }
            const lt_split ta = th_form(ctx, lva, f[ia.idx], ia.algo, ia.sp);
            const u32 n1 = ta.n1, n2 = ta.n2, n3 = ta.n3;
            std::vector<LtIO> group;
            for (u32 b = a; b < count && group.size() < (size_t)DM_MAX_B; b++) {
                if (done[b]) continue;
                const Item& ib = items[b];
                if (ib.algo == LT_BSGS || f[ib.idx] != f[ia.idx] || in[ib.idx]->level != in[ia.idx]->level) continue;
                const lt_split tb = th_form(ctx, in[ib.idx]->level, f[ib.idx], ib.algo, ib.sp);
                if (tb.n1 != n1 || tb.n2 != n2 || tb.n3 != n3) continue;
                const u32 level = in[ib.idx]->level;
                const size_t lw = (size_t)level * ctx->N;
                group.push_back(LtIO{in[ib.idx]->d, in[ib.idx]->d + lw, out[ib.idx]->d,
                                     out[ib.idx]->d + (size_t)(level - 1) * ctx->N});
                done[b] = true;
            }
            const ckks_diags* fa = f[ia.idx];
            const K6Tile tile = tile_for(ctx, lva, fa, ia.algo, ia.sp);
            units.push_back(Unit{one * group.size(), [=](cudaStream_t s) {
                                     sched_th_batch(ctx, lva, group, fa, n1, n2, n3, s, tile);
                                 }});
        }
        if (units.size() <= 1) {
            for (Unit& u : units) u.run(st);
        } else {
            // fork: the biggest units first, each onto the least-loaded lane; join on the caller's stream
            std::lock_guard<std::mutex> g(ctx->fork_mu);
            const u32 nl = (u32)std::min<size_t>(units.size(), ckks_ctx::FORK_LANES);
            ckks_ctx::Lanes& ln = ctx->lanes[st];
            if (!ln.fork) CK(cudaEventCreateWithFlags(&ln.fork, cudaEventDisableTiming));
            for (u32 i = 0; i + 1 < nl; i++) {
                if (!ln.s[i]) CK(cudaStreamCreateWithFlags(&ln.s[i], cudaStreamNonBlocking));
                if (!ln.join[i]) CK(cudaEventCreateWithFlags(&ln.join[i], cudaEventDisableTiming));
            }
            CK(cudaEventRecord(ln.fork, st));
            for (u32 i = 0; i + 1 < nl; i++) CK(cudaStreamWaitEvent(ln.s[i], ln.fork, 0));
            std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.cost > y.cost; });
            std::vector<double> load(nl, 0.0);
            for (Unit& u : units) {
                const u32 w = (u32)(std::min_element(load.begin(), load.end()) - load.begin());
                load[w] += u.cost;
                u.run(w == 0 ? st : ln.s[w - 1]);
            }
            for (u32 i = 0; i + 1 < nl; i++) {
                CK(cudaEventRecord(ln.join[i], ln.s[i]));
                CK(cudaStreamWaitEvent(st, ln.join[i], 0));
            }
        }
        CK(cudaGetLastError());
    });
}

ckks_status lt_eval_chain(ckks_ctx* ctx, const ckks_ct* in, uint32_t n_stages, const ckks_diags* const* f,
                          const lt_algo* algos, const lt_split* splits, ckks_ct* out, void* stream, lt_split* chosen) {
    return guarded([&] {
        if (!ctx || !in || !out || !f) fail(CKKS_EINVAL, "null argument");
        if (n_stages < 1) fail(CKKS_EINVAL, "need at least one stage");
        if (in->ctx != ctx || out->ctx != ctx) fail(CKKS_EINVAL, "objects of another context");
        if (in->level < n_stages + 1) fail(CKKS_EINVAL, "input level too low for the chain (one level per stage)");
        if (out->level != in->level - n_stages) fail(CKKS_EINVAL, "output level must be input level - n_stages");
        if (out->d == in->d) fail(CKKS_EINVAL, "output must not alias input");
        // validate every stage before queuing anything
        std::vector<lt_split> sp(n_stages);
        std::vector<lt_algo> al(n_stages);
        for (u32 i = 0; i < n_stages; i++) {
            if (!f[i] || f[i]->ctx != ctx) fail(CKKS_EINVAL, "stage diagonals missing or of another context");
            const u32 level = in->level - i;
            if (level > f[i]->level) fail(CKKS_EINVAL, "stage diagonals encoded below the stage's level");
            al[i] = algos ? algos[i] : LT_TH_BSGS;
            sp[i] = resolve_split(ctx, level, f[i], al[i], splits ? &splits[i] : nullptr);
        }
        CK(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Arena ar(st, ctx->N);  // the intermediate ciphertexts, freed in stream order after the chain
        const u64* c = in->d;
        for (u32 i = 0; i < n_stages; i++) {
            const u32 level = in->level - i;
            u64* o = (i + 1 == n_stages) ? out->d : ar.limbs(2ull * (level - 1));
            dispatch(ctx, level, LtIO{c, c + (size_t)level * ctx->N, o, o + (size_t)(level - 1) * ctx->N}, f[i],
                     al[i], sp[i], st);
            c = o;
        }
        CK(cudaGetLastError());
        if (chosen)
            for (u32 i = 0; i < n_stages; i++) chosen[i] = sp[i];
    });
}

// ------------------------------------------------------------------ recorded batches
}  // extern "C"

struct lt_graph {
    ckks_ctx* ctx;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

ckks_status lt_graph_create(ckks_ctx* ctx, uint32_t count, const ckks_ct* const* in, const ckks_diags* const* f,
                            const lt_algo* algos, const lt_split* splits, ckks_ct* const* out, lt_graph** graph) {
    cudaStream_t st = nullptr;
    lt_graph* gr = nullptr;
    ckks_status rc = guarded([&] {
        if (!ctx || !graph) fail(CKKS_EINVAL, "null argument");
        *graph = nullptr;
        CK(cudaSetDevice(ctx->device));
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    });
    if (rc != CKKS_OK) return rc;
    // one plain run: validates the batch and sets up every table and kernel attribute it needs
    rc = lt_eval_batch(ctx, count, in, f, algos, splits, out, st);
    if (rc == CKKS_OK)
        rc = guarded([&] {
            CK(cudaStreamSynchronize(st));
            gr = new lt_graph{ctx};
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        });
    if (rc == CKKS_OK) {
        const ckks_status run = lt_eval_batch(ctx, count, in, f, algos, splits, out, st);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        rc = run != CKKS_OK ? run : guarded([&] {
            CK(e);
            gr->graph = g;
            CK(cudaGraphInstantiate(&gr->exec, g, 0));
            *graph = gr;
            gr = nullptr;
        });
        if (rc != CKKS_OK && g && gr && !gr->graph) cudaGraphDestroy(g);
    }
    if (gr) {
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        if (gr->graph) cudaGraphDestroy(gr->graph);
        delete gr;
    }
    if (st) {
        release_lanes(ctx, st);
        cudaStreamDestroy(st);
    }
    return rc;
}

ckks_status lt_graph_begin(ckks_ctx* ctx, void* stream) {
    return guarded([&] {
        if (!ctx) fail(CKKS_EINVAL, "null argument");
        if (!stream) fail(CKKS_EINVAL, "the legacy default stream cannot be recorded; pass a created stream");
        CK(cudaSetDevice(ctx->device));
        CK(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal));
    });
}

ckks_status lt_graph_end(ckks_ctx* ctx, void* stream, lt_graph** graph) {
    cudaGraph_t g = nullptr;
    lt_graph* gr = nullptr;
    ckks_status rc = guarded([&] {
        if (!ctx || !stream || !graph) fail(CKKS_EINVAL, "null argument");
        *graph = nullptr;
        CK(cudaSetDevice(ctx->device));
        // ends the capture even when a recorded call failed (the graph is then invalid)
        CK(cudaStreamEndCapture((cudaStream_t)stream, &g));
        gr = new lt_graph{ctx};
        gr->graph = g;
        g = nullptr;
        CK(cudaGraphInstantiate(&gr->exec, gr->graph, 0));
        *graph = gr;
        gr = nullptr;
    });
    if (g) cudaGraphDestroy(g);
    if (gr) {
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        if (gr->graph) cudaGraphDestroy(gr->graph);
        delete gr;
    }
    return rc;
}

ckks_status lt_graph_launch(lt_graph* graph, void* stream) {
    return guarded([&] {
        if (!graph) fail(CKKS_EINVAL, "null argument");
        CK(cudaSetDevice(graph->ctx->device));
        CK(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
        count_launch();
    });
}

ckks_status lt_graph_destroy(lt_graph* graph) {
    return guarded([&] {
        if (!graph) return;
        cudaSetDevice(graph->ctx->device);
        if (graph->exec) cudaGraphExecDestroy(graph->exec);
        if (graph->graph) cudaGraphDestroy(graph->graph);
        delete graph;
    });
}

// ------------------------------------------------------------------ steps
ckks_status ckks_poly_ntt(ckks_ctx* ctx, uint64_t* poly, uint32_t level, int ext, int inverse, void* stream) {
    return guarded([&] {
        if (!ctx || !poly) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        const u32 nl = level + (ext ? ctx->K : 0), N = ctx->N;
        if (inverse) {
            std::vector<InvJob> j(nl);
            for (u32 t = 0; t < nl; t++) {
                const u32 g = ctx->gmod(level, t);
                const u64 m = ctx->mods[g], ninv = invmod_h(N % m, m);
                j[t] = InvJob{poly + (size_t)t * N, poly + (size_t)t * N, poly + (size_t)t * N, ninv, shoup_h(ninv, m), g,
                              0};
            }
            launch_inv_ntt(ctx->T, j.data(), (int)nl, (cudaStream_t)stream);
        } else {
            std::vector<FwdJob> j(nl);
            for (u32 t = 0; t < nl; t++)
                j[t] = FwdJob{poly + (size_t)t * N, poly + (size_t)t * N, nullptr, nullptr, nullptr, 0, 0,
                              ctx->gmod(level, t), 0};
            launch_fwd_ntt(ctx->T, j.data(), (int)nl, (cudaStream_t)stream);
        }
        CK(cudaGetLastError());
    });
}

ckks_status ckks_decompose(ckks_ctx* ctx, uint32_t level, const uint64_t* c, int32_t rot, uint64_t* digits,
                           void* stream) {
    return guarded([&] {
        if (!ctx || !c || !digits) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Arena ar(st, ctx->N);
        u64* Y = ar.limbs(level);
        op_decompose(ctx, level, c, ctx->rotkey(rot) ? ctx->galois(rot) : 0, digits, Y, st);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_ks_inner(ckks_ctx* ctx, uint32_t level, const uint64_t* digits, int32_t key_rot, int32_t rot,
                          const uint64_t* x0, int lift_x0, uint64_t* out0, uint64_t* out1, int accumulate,
                          void* stream) {
    return guarded([&] {
        if (!ctx || !digits || !out0 || !out1) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        op_ks_inner(ctx, level, digits, key_of(ctx, key_rot), ctx->rotkey(rot) ? ctx->galois(rot) : 0, x0,
                    lift_x0 ? 2 : 1, out0, out1, accumulate, (cudaStream_t)stream);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_moddown(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream) {
    return guarded([&] {
        if (!ctx || !x || !out) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        if (x == out) fail(CKKS_EINVAL, "ModDown cannot run in place");
        CK(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Arena ar(st, ctx->N);
        op_moddown(ctx, level, x, out, ar.limbs(ctx->K), st);
        CK(cudaGetLastError());
    });
}

}  // extern "C"

// ------------------------------------------------------------------ ModDown without allocation
// For host programs that cannot let the library allocate device memory while
// it runs: an application that manages all GPU memory through its own
// allocator or budget, or a latency-bound path where a cudaMalloc (and the
// device synchronisation it may imply) is not acceptable.
// ModDown's only scratch (the inverse-transformed special-prime limbs) lives
// in this fixed file-scope array instead of the stream-ordered pool: at most
// NOALLOC_SCRATCH_WORDS words (8 limbs of N = 2^16, 4 MiB), held by every
// GPU that loads the library until the process exits.
constexpr size_t NOALLOC_SCRATCH_WORDS = 8ull << 16;
static __device__ __align__(256) uint64_t g_moddown_scratch[NOALLOC_SCRATCH_WORDS];

namespace {
std::mutex g_scratch_mu;
u64* g_scratch_dev[128] = {};

// Device address of g_moddown_scratch on `dev` (the current device).  The
// array's name in host code is only a host-side stand-in, so the address is
// looked up once per device and cached.
u64* noalloc_scratch(int dev) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= 128) fail(CKKS_EINVAL, "device index out of range");
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_moddown_scratch));
        g_scratch_dev[dev] = (u64*)p;
    }
    return g_scratch_dev[dev];
}
}  // namespace

extern "C" {

ckks_status ckks_moddown_noalloc(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream) {
    return guarded([&] {
        if (!ctx || !x || !out) fail(CKKS_EINVAL, "null argument");
        if (level < 1 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        if (x == out) fail(CKKS_EINVAL, "ModDown cannot run in place");
        if ((size_t)ctx->K * ctx->N > NOALLOC_SCRATCH_WORDS)
            fail(CKKS_EINVAL, "k * N = " + std::to_string((size_t)ctx->K * ctx->N) +
                                  " words exceeds the fixed scratch of " + std::to_string(NOALLOC_SCRATCH_WORDS) +
                                  " words (8 limbs at N = 2^16)");
        if (level > 64 || ctx->K > 8) fail(CKKS_EINVAL, "level must be <= 64 and k <= 8");
        const LevelConsts* LC = nullptr;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            auto it = ctx->levels.find(level);
            if (it != ctx->levels.end()) LC = &it->second;
        }
        if (!LC)
            fail(CKKS_EINVAL, "the constants of this level are not set up yet; any earlier call at this level "
                              "(ckks_moddown, lt_eval, ...) sets them up");
        CK(cudaSetDevice(ctx->device));
        u64* Y = noalloc_scratch(ctx->device);
        const u32 N = ctx->N, k = ctx->K;
        cudaStream_t st = (cudaStream_t)stream;
        InvJob ij[8];
        for (u32 i = 0; i < k; i++)
            ij[i] = InvJob{x + (size_t)(level + i) * N, Y + (size_t)i * N, Y + (size_t)i * N, LC->md_c[i], LC->md_sh[i],
                           ctx->L + i, 0};
        launch_inv_ntt(ctx->T, ij, (int)k, st);
        FwdJob fj[64];
        for (u32 j = 0; j < level; j++)
            fj[j] = FwdJob{Y, out + (size_t)j * N, LC->md_tab + (size_t)j * k, x + (size_t)j * N, out + (size_t)j * N,
                           LC->md_pinv[j], LC->md_pinv_sh[j], j, k};
        launch_fwd_ntt(ctx->T, fj, (int)level, st);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_moddown_rescale(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream) {
    return guarded([&] {
        if (!ctx || !x || !out) fail(CKKS_EINVAL, "null argument");
        if (level < 2 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Arena ar(st, ctx->N);
        op_moddown_rescale(ctx, level, x, out, ar.limbs(ctx->K + 1), st);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_rescale(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream) {
    return guarded([&] {
        if (!ctx || !x || !out) fail(CKKS_EINVAL, "null argument");
        if (level < 2 || level > ctx->L) fail(CKKS_EINVAL, "bad level");
        CK(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Arena ar(st, ctx->N);
        op_rescale(ctx, level, x, out, ar.limbs(1), st);
        CK(cudaGetLastError());
    });
}

ckks_status ckks_automorphism(ckks_ctx* ctx, uint32_t n_limbs, const uint64_t* in, int32_t rot, uint64_t* out,
                              void* stream) {
    return guarded([&] {
        if (!ctx || !in || !out) fail(CKKS_EINVAL, "null argument");
        if (in == out) fail(CKKS_EINVAL, "automorphism cannot run in place");
        CK(cudaSetDevice(ctx->device));
        if (ctx->rotkey(rot) == 0)
            CK(cudaMemcpyAsync(out, in, (size_t)n_limbs * ctx->N * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
        else launch_automorphism(in, out, n_limbs, ctx->galois(rot), ctx->log_n, (cudaStream_t)stream);
        CK(cudaGetLastError());
    });
}

}  // extern "C"
