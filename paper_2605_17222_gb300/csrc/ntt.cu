// Negacyclic NTT / INTT kernels on uint64 limbs (sm_103a), plus the
// automorphism gather.
//
// Transform (Sec. II-A; bit-reversed storage as in Sec. V): the forward NTT is
// the merged Cooley-Tukey form whose stage m (m = 1, 2, .., N/2, half-width
// t = N/2m) pairs words j and j+t of group i = j / 2t with twiddle
// psi^brv(m+i); its output word s holds a(psi^(2 brv(s) + 1)).  The inverse
// is the Gentleman-Sande mirror with psi^-brv(m+i), followed by N^-1.
//
// A limb of N = R*C words (R = 2^ceil(logN/2) rows, C columns) is done in two
// passes so that each pass fits shared memory:
//   column pass: the stages with t >= C pair rows r and r + t/C of the same
//                column (a strided R-point transform per column);
//   row pass   : the stages with t < C stay inside one row of C contiguous words.
// The forward NTT runs column pass then row pass; the inverse runs row pass
// then column pass.  Both passes take a list of limb jobs so that one launch
// covers every limb of a step, and both carry the fused loads/epilogues of the
// key-switching path (basis conversion on load, ModDown tail on store, scaling,
// automorphism gather) so that those steps cost no extra HBM round trip.
#include "kernels.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

namespace ckks {

static std::atomic<uint64_t> g_launches{0};
uint64_t launches() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }

// ------------------------------------------------------------------ live per-kernel timing
const char* const kclass_names[K_NCLASS] = {"diag_mac", "ks_inner", "ntt_fwd_cols", "ntt_fwd_rows",
                                            "ntt_inv_rows", "ntt_inv_cols", "automorphism", "add_gather"};
namespace {
struct EvPair {
    cudaEvent_t a, b;
};
struct Profiler {
    std::mutex mu;
    std::atomic<bool> on[K_NCLASS];
    std::vector<EvPair> pending[K_NCLASS];
    std::vector<EvPair> pool;
    double ms[K_NCLASS] = {};
    uint64_t n[K_NCLASS] = {};
    Profiler() {
        for (auto& o : on) o = false;
    }
    EvPair get() {
        std::lock_guard<std::mutex> g(mu);
        if (!pool.empty()) {
            EvPair e = pool.back();
            pool.pop_back();
            return e;
        }
        EvPair e;
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        return e;
    }
    void drain(int c) {  // mu held
        for (EvPair& e : pending[c]) {
            float t = 0;
            cudaEventSynchronize(e.b);
            cudaEventElapsedTime(&t, e.a, e.b);
            ms[c] += t;
            n[c]++;
            pool.push_back(e);
        }
        pending[c].clear();
    }
};
Profiler& prof() {
    static Profiler p;
    return p;
}
}  // namespace

bool prof_on(int cls) { return prof().on[cls].load(std::memory_order_relaxed); }
int prof_class(const char* name) {
    for (int i = 0; i < K_NCLASS; i++)
        if (name && !strcmp(name, kclass_names[i])) return i;
    return -1;
}
void prof_enable(int cls, bool on) { prof().on[cls] = on; }
bool prof_read(int cls, double* ms, uint64_t* n) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    P.drain(cls);
    *ms = P.ms[cls];
    *n = P.n[cls];
    return true;
}
void prof_reset() {
    Profiler& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    for (int c = 0; c < K_NCLASS; c++) {
        P.drain(c);
        P.ms[c] = 0;
        P.n[c] = 0;
    }
}
ProfScope::ProfScope(int c, cudaStream_t s) : cls(c), st(s), ev(nullptr) {
    if (!prof_on(c)) return;
    EvPair* e = new EvPair(prof().get());
    cudaEventRecord(e->a, s);
    ev = e;
}
ProfScope::~ProfScope() {
    if (!ev) return;
    EvPair* e = (EvPair*)ev;
    cudaEventRecord(e->b, st);
    Profiler& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    P.pending[cls].push_back(*e);
    delete e;
}

namespace {

constexpr int MAXJ = 96;
constexpr int THREADS = 256;
constexpr u32 TILE = 4096;  // words per CTA in the row pass

template <typename J>
struct Jobs {
    J j[MAXJ];
};

struct Geo {
    u32 log_n, log_r, log_c, w, b;  // R = 2^log_r rows, C = 2^log_c columns, w cols/CTA, b rows/CTA
};

Geo geometry(u32 log_n) {
    Geo g;
    g.log_n = log_n;
    g.log_r = (log_n + 1) / 2;
    g.log_c = log_n - g.log_r;
    g.w = std::min<u32>(16u, 1u << g.log_c);
    g.b = std::max<u32>(1u, std::min<u32>(1u << g.log_r, TILE >> g.log_c));
    return g;
}

// ------------------------------------------------------------------ forward, column pass
template <bool BCONV>
__global__ void __launch_bounds__(THREADS) k_fwd_cols(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<FwdJob> jobs, Geo g) {
    extern __shared__ u64 sm[];
    const FwdJob& J = jobs.j[blockIdx.y];
    const u32 N = 1u << g.log_n, R = 1u << g.log_r, C = 1u << g.log_c, W = g.w;
    const u32 c0 = blockIdx.x * W;
    const ModC m = T.mods[J.mod];
    const u64* psi = T.psi + (size_t)J.mod * N;
    const u64* psh = T.psi_sh + (size_t)J.mod * N;
    for (u32 e = threadIdx.x; e < R * W; e += THREADS) {
        const u32 r = e / W, c = e % W;
        const size_t x = (size_t)r * C + c0 + c;
        u64 v;
        if constexpr (BCONV) {
            U128 acc{0, 0};
            for (u32 j = 0; j < J.nsrc; j++) mac128(acc, J.src[(size_t)j * N + x], J.bcst[j]);
            v = reduce128(acc, m);
        } else {
            v = J.src[x];
        }
        sm[e] = v;
    }
    __syncthreads();
    for (u32 s = 0; s < g.log_r; s++) {
        const u32 tr = R >> (s + 1);
        const u32 mm = 1u << s;
        for (u32 b = threadIdx.x; b < (R / 2) * W; b += THREADS) {
            const u32 c = b % W, k = b / W;
            const u32 grp = k / tr, pos = k % tr;
            const u32 r = grp * 2 * tr + pos;
            const u64 S = psi[mm + grp], Ssh = psh[mm + grp];
            const u64 U = sm[r * W + c];
            const u64 V = mul_shoup(sm[(r + tr) * W + c], S, Ssh, m.q);
            sm[r * W + c] = add_mod(U, V, m.q);
            sm[(r + tr) * W + c] = sub_mod(U, V, m.q);
        }
        __syncthreads();
    }
    for (u32 e = threadIdx.x; e < R * W; e += THREADS) {
        const u32 r = e / W, c = e % W;
        J.dst[(size_t)r * C + c0 + c] = sm[e];
    }
}

// ------------------------------------------------------------------ forward, row pass
template <bool SUBMUL>
__global__ void __launch_bounds__(THREADS) k_fwd_rows(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<FwdJob> jobs, Geo g) {
    extern __shared__ u64 sm[];
    const FwdJob& J = jobs.j[blockIdx.y];
    const u32 N = 1u << g.log_n, C = 1u << g.log_c, B = g.b;
    const u32 r0 = blockIdx.x * B;
    const size_t base = (size_t)r0 * C;
    const ModC m = T.mods[J.mod];
    const u64* psi = T.psi + (size_t)J.mod * N;
    const u64* psh = T.psi_sh + (size_t)J.mod * N;
    for (u32 e = threadIdx.x; e < B * C; e += THREADS) sm[e] = J.dst[base + e];
    __syncthreads();
    const u32 half = C / 2;
    for (u32 sp = 0; sp < g.log_c; sp++) {
        const u32 mm = 1u << (g.log_r + sp);
        const u32 t = C >> (sp + 1);
        const u32 gpr = C / (2 * t);  // groups per row
        for (u32 b = threadIdx.x; b < B * half; b += THREADS) {
            const u32 blk = b / half, k = b % half;
            const u32 grp = k / t, pos = k % t;
            const u32 x = blk * C + grp * 2 * t + pos;
            const u32 idx = mm + (r0 + blk) * gpr + grp;
            const u64 U = sm[x];
            const u64 V = mul_shoup(sm[x + t], psi[idx], psh[idx], m.q);
            sm[x] = add_mod(U, V, m.q);
            sm[x + t] = sub_mod(U, V, m.q);
        }
        __syncthreads();
    }
    for (u32 e = threadIdx.x; e < B * C; e += THREADS) {
        const u64 v = sm[e];
        if constexpr (SUBMUL) {
            J.subout[base + e] = mul_shoup(sub_mod(J.subx[base + e], v, m.q), J.c, J.c_sh, m.q);
        } else {
            J.dst[base + e] = v;
        }
    }
}

// ------------------------------------------------------------------ inverse, row pass
template <bool GATHER>
__global__ void __launch_bounds__(THREADS) k_inv_rows(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<InvJob> jobs, Geo g) {
    extern __shared__ u64 sm[];
    const InvJob& J = jobs.j[blockIdx.y];
    const u32 N = 1u << g.log_n, C = 1u << g.log_c, B = g.b;
    const u32 r0 = blockIdx.x * B;
    const size_t base = (size_t)r0 * C;
    const ModC m = T.mods[J.mod];
    const u64* ipsi = T.ipsi + (size_t)J.mod * N;
    const u64* ish = T.ipsi_sh + (size_t)J.mod * N;
    for (u32 e = threadIdx.x; e < B * C; e += THREADS) {
        if constexpr (GATHER) {
            sm[e] = J.src[auto_src((u32)(base + e), J.gal, g.log_n)];
        } else {
            sm[e] = J.src[base + e];
        }
    }
    __syncthreads();
    const u32 half = C / 2;
    for (u32 u = 0; u < g.log_c; u++) {
        const u32 t = 1u << u;
        const u32 mm = N >> (u + 1);
        const u32 gpr = C / (2 * t);
        for (u32 b = threadIdx.x; b < B * half; b += THREADS) {
            const u32 blk = b / half, k = b % half;
            const u32 grp = k / t, pos = k % t;
            const u32 x = blk * C + grp * 2 * t + pos;
            const u32 idx = mm + (r0 + blk) * gpr + grp;
            const u64 U = sm[x], V = sm[x + t];
            sm[x] = add_mod(U, V, m.q);
            sm[x + t] = mul_shoup(sub_mod(U, V, m.q), ipsi[idx], ish[idx], m.q);
        }
        __syncthreads();
    }
    for (u32 e = threadIdx.x; e < B * C; e += THREADS) J.tmp[base + e] = sm[e];
}

// ------------------------------------------------------------------ inverse, column pass
__global__ void __launch_bounds__(THREADS) k_inv_cols(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<InvJob> jobs, Geo g) {
    extern __shared__ u64 sm[];
    const InvJob& J = jobs.j[blockIdx.y];
    const u32 N = 1u << g.log_n, R = 1u << g.log_r, C = 1u << g.log_c, W = g.w;
    const u32 c0 = blockIdx.x * W;
    const ModC m = T.mods[J.mod];
    const u64* ipsi = T.ipsi + (size_t)J.mod * N;
    const u64* ish = T.ipsi_sh + (size_t)J.mod * N;
    for (u32 e = threadIdx.x; e < R * W; e += THREADS) {
        const u32 r = e / W, c = e % W;
        sm[e] = J.tmp[(size_t)r * C + c0 + c];
    }
    __syncthreads();
    for (u32 u = g.log_c; u < g.log_n; u++) {
        const u32 tr = 1u << (u - g.log_c);
        const u32 mm = N >> (u + 1);
        for (u32 b = threadIdx.x; b < (R / 2) * W; b += THREADS) {
            const u32 c = b % W, k = b / W;
            const u32 grp = k / tr, pos = k % tr;
            const u32 r = grp * 2 * tr + pos;
            const u64 U = sm[r * W + c], V = sm[(r + tr) * W + c];
            sm[r * W + c] = add_mod(U, V, m.q);
            sm[(r + tr) * W + c] = mul_shoup(sub_mod(U, V, m.q), ipsi[mm + grp], ish[mm + grp], m.q);
        }
        __syncthreads();
    }
    for (u32 e = threadIdx.x; e < R * W; e += THREADS) {
        const u32 r = e / W, c = e % W;
        J.dst[(size_t)r * C + c0 + c] = mul_shoup(sm[e], J.c, J.c_sh, m.q);
    }
}

__global__ void k_automorphism(const u64* __restrict__ in, u64* __restrict__ out, u32 gal, u32 log_n) {
    const u32 N = 1u << log_n;
    const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t l = blockIdx.y;
    if (s < N) out[l * N + s] = in[l * N + auto_src(s, gal, log_n)];
}

__global__ void k_add_gather(const ModC* __restrict__ mods, const __grid_constant__ Jobs<AddJob> jobs, u32 gal,
                             int acc, u32 log_n) {
    const u32 N = 1u << log_n;
    const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const AddJob& J = jobs.j[blockIdx.y];
    const u64 q = mods[J.mod].q;
    u64 v = J.a[gal ? auto_src(s, gal, log_n) : s];
    if (J.b) v = add_mod(v, J.b[s], q);
    if (acc) v = add_mod(v, J.out[s], q);
    J.out[s] = v;
}

// Shared memory above 48 KB (log N = 17) needs an explicit opt-in per kernel.
void set_smem_limits() {
    static bool done = false;
    if (done) return;
    done = true;
    const int lim = 96 * 1024;
    cudaFuncSetAttribute(k_fwd_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fwd_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fwd_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_fwd_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_inv_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_inv_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_inv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <typename J, typename F>
void for_chunks(const J* jobs, int njobs, F&& f) {
    for (int s = 0; s < njobs; s += MAXJ) {
        Jobs<J> pack;
        const int n = std::min(MAXJ, njobs - s);
        for (int i = 0; i < n; i++) pack.j[i] = jobs[s + i];
        f(pack, n);
    }
}

}  // namespace

void launch_fwd_ntt(const NttTables& T, const FwdJob* jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return;
    const Geo g = geometry(T.log_n);
    const u32 R = 1u << g.log_r, C = 1u << g.log_c;
    const size_t sm1 = (size_t)R * g.w * sizeof(u64), sm2 = (size_t)g.b * C * sizeof(u64);
    const bool bconv = jobs[0].nsrc > 0, submul = jobs[0].subout != nullptr;
    set_smem_limits();
    for_chunks(jobs, njobs, [&](const Jobs<FwdJob>& p, int n) {
        dim3 g1(C / g.w, n), g2(R / g.b, n);
        {
            ProfScope ps(K_FWD_COLS, st);
            if (bconv) k_fwd_cols<true><<<g1, THREADS, sm1, st>>>(T, p, g);
            else k_fwd_cols<false><<<g1, THREADS, sm1, st>>>(T, p, g);
        }
        {
            ProfScope ps(K_FWD_ROWS, st);
            if (submul) k_fwd_rows<true><<<g2, THREADS, sm2, st>>>(T, p, g);
            else k_fwd_rows<false><<<g2, THREADS, sm2, st>>>(T, p, g);
        }
        count_launch(2);
    });
}

void launch_inv_ntt(const NttTables& T, const InvJob* jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return;
    const Geo g = geometry(T.log_n);
    const u32 R = 1u << g.log_r, C = 1u << g.log_c;
    const size_t sm1 = (size_t)R * g.w * sizeof(u64), sm2 = (size_t)g.b * C * sizeof(u64);
    const bool gather = jobs[0].gal != 0;
    set_smem_limits();
    for_chunks(jobs, njobs, [&](const Jobs<InvJob>& p, int n) {
        dim3 g1(C / g.w, n), g2(R / g.b, n);
        {
            ProfScope ps(K_INV_ROWS, st);
            if (gather) k_inv_rows<true><<<g2, THREADS, sm2, st>>>(T, p, g);
            else k_inv_rows<false><<<g2, THREADS, sm2, st>>>(T, p, g);
        }
        {
            ProfScope ps(K_INV_COLS, st);
            k_inv_cols<<<g1, THREADS, sm1, st>>>(T, p, g);
        }
        count_launch(2);
    });
}

void launch_automorphism(const u64* in, u64* out, u32 n_limbs, u32 gal, u32 log_n, cudaStream_t st) {
    if (!n_limbs) return;
    const u32 N = 1u << log_n;
    ProfScope ps(K_AUTO, st);
    k_automorphism<<<dim3((N + 255) / 256, n_limbs), 256, 0, st>>>(in, out, gal, log_n);
    count_launch();
}

void launch_add_gather(const ModC* mods, const AddJob* jobs, int njobs, u32 gal, int accumulate, u32 log_n,
                       cudaStream_t st) {
    const u32 N = 1u << log_n;
    for_chunks(jobs, njobs, [&](const Jobs<AddJob>& p, int n) {
        ProfScope ps(K_ADD, st);
        k_add_gather<<<dim3((N + 255) / 256, n), 256, 0, st>>>(mods, p, gal, accumulate, log_n);
        count_launch();
    });
}

}  // namespace ckks
