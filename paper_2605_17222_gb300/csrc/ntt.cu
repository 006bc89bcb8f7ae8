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
    double mac[K_NCLASS] = {};   // algorithmic 128-bit multiply-accumulates of the timed launches
    double bfly[K_NCLASS] = {};  // algorithmic NTT butterflies of the timed launches
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
bool prof_work(int cls, double* macs, double* butterflies) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    *macs = P.mac[cls];
    *butterflies = P.bfly[cls];
    return true;
}
void prof_reset() {
    Profiler& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    for (int c = 0; c < K_NCLASS; c++) {
        P.drain(c);
        P.ms[c] = 0;
        P.n[c] = 0;
        P.mac[c] = 0;
        P.bfly[c] = 0;
    }
}
ProfScope::ProfScope(int c, cudaStream_t s, double macs, double butterflies) : cls(c), st(s), ev(nullptr) {
    if (!prof_on(c)) return;
    {
        Profiler& P = prof();
        std::lock_guard<std::mutex> g(P.mu);
        P.mac[c] += macs;
        P.bfly[c] += butterflies;
    }
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

// Jobs per launch, passed by value: 510 forward jobs (64 bytes each) and the tables fill the
// 32,764 bytes of kernel parameters; a level-24 Decompose of three polynomials (504 jobs) is one launch.
constexpr int MAXJ = 510;
static_assert(sizeof(FwdJob) * MAXJ + sizeof(NttTables) <= 32764, "forward jobs exceed the kernel parameter space");
static_assert(sizeof(InvJob) * MAXJ + sizeof(NttTables) <= 32764, "inverse jobs exceed the kernel parameter space");
static_assert(sizeof(AddJob) * MAXJ + 64 <= 32764, "add jobs exceed the kernel parameter space");
constexpr int THREADS = 256;

template <typename J>
struct Jobs {
    J j[MAXJ];
};

// Twiddle w and its Shoup companion, one 16-byte load.
__device__ __forceinline__ void tw_at(const ulonglong2* tab, u32 idx, u64& w, u64& ws) {
    const ulonglong2 v = __ldg(tab + idx);
    w = v.x;
    ws = v.y;
}

// Shoup product without the final correction: a w mod q in [0, 2q) for any a < 2^64.
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 ws, u64 q) {
    return a * w - __umul64hi(a, ws) * q;
}

// Cooley-Tukey butterfly (forward), lazy (Harvey): inputs and outputs in
// [0, 4q) (every modulus is below 2^60, so 4q < 2^64);
// (a, b) -> (a + w b, a - w b) mod q up to multiples of q.
__device__ __forceinline__ void ct_bfly_w(u64& a, u64& b, u64 w, u64 ws, u64 q) {
    const u64 q2 = 2 * q;
    const u64 x = a >= q2 ? a - q2 : a;
    const u64 v = mul_shoup_lazy(b, w, ws, q);
    a = x + v;
    b = x - v + q2;
}
__device__ __forceinline__ void ct_bfly(u64& a, u64& b, const ulonglong2* tab, u32 idx, u64 q) {
    u64 w, ws;
    tw_at(tab, idx, w, ws);
    ct_bfly_w(a, b, w, ws, q);
}

// [0, 4q) -> [0, q)
__device__ __forceinline__ u64 canon4(u64 x, u64 q) {
    x = x >= 2 * q ? x - 2 * q : x;
    return x >= q ? x - q : x;
}

// Any 64-bit word -> [0, 2q): the Shoup product by 1 (floor(2^64 / q) = mu_hi).
__device__ __forceinline__ u64 red2(u64 x, u64 q, u64 mu_hi) { return x - __umul64hi(x, mu_hi) * q; }

// x < 2^50 -> [0, 3q) for 2^32 < q < 2^41, with mu32 = floor(2^64 / q) (below
// 2^32).  The estimate qe = floor(floor(x / 2^32) mu32 / 2^32) never exceeds
// floor(x / q) and falls short of it by at most 2: the dropped low word of x
// is worth below 2^32 / q < 1, mu32's truncation below floor(x / 2^32) / 2^32
// < 2^-14, and the floor below 1.  One 32 x 32 product and one small product
// by q, instead of the 64 x 64 high product of red2.
__device__ __forceinline__ u64 red3_small(u64 x, u64 q, u32 mu32) {
    const u64 qe = ((u64)(u32)(x >> 32) * mu32) >> 32;
    return x - qe * q;
}
__device__ __forceinline__ bool small_q(u64 q) { return q > (1ull << 32) && q < (1ull << 41); }

// ------------------------------------------------------------------ growing butterflies
// For moduli well below 2^64 the per-butterfly conditional subtraction that
// keeps a lazy word bounded can be dropped inside a pass:
//   CT: if both inputs are below B, (a + v, a - v + 4q) with v = b w mod q in
//       [0, 4q) (a quotient estimate that may be 2 short, mul_shoup_approx)
//       are both below B + 4q.  The log N <= 16 stages of a forward transform
//       from [0, 4q) (a lazily reduced basis conversion) stay below 68q, below
//       2^64 for q < 2^57.
// Wider moduli (the 60-bit special primes) take the reducing butterflies.
// The inverse transform keeps one lazy form for every modulus (gs_w).
constexpr u64 FWD_GROW_MAX = 1ull << 57;

// b w mod q up to 4q, for any b < 2^64 (w < q, ws = floor(w 2^64 / q)).  Of
// the four 32 x 32 partial products of b ws the quotient estimate keeps the
// high one and the high halves of the two middle ones; what it drops carries
// at most 2 into bit 64, so the estimate is below floor(b ws / 2^64) by at
// most 2 and the remainder lies in [0, 2q) + [0, 2q).
__device__ __forceinline__ u64 mul_shoup_approx(u64 b, u64 w, u64 ws, u64 q) {
    const u32 b0 = (u32)b, b1 = (u32)(b >> 32), s0 = (u32)ws, s1 = (u32)(ws >> 32);
    const u64 qe = (u64)b1 * s1 + __umulhi(b0, s1) + __umulhi(b1, s0);
    return b * w - qe * q;
}

template <bool GROW>
__device__ __forceinline__ void ct_w(u64& a, u64& b, u64 w, u64 ws, u64 q) {
    if constexpr (GROW) {
        const u64 v = mul_shoup_approx(b, w, ws, q);  // [0, 4q)
        b = a - v + 4 * q;
        a = a + v;
    } else {
        ct_bfly_w(a, b, w, ws, q);
    }
}
template <bool GROW>
__device__ __forceinline__ void ct(u64& a, u64& b, const ulonglong2* tab, u32 idx, u64 q) {
    u64 w, ws;
    tw_at(tab, idx, w, ws);
    ct_w<GROW>(a, b, w, ws, q);
}
// A staged twiddle pair in shared memory.
template <bool GROW>
__device__ __forceinline__ void ct_s(u64& a, u64& b, const ulonglong2& t, u64 q) {
    const ulonglong2 v = t;
    ct_w<GROW>(a, b, v.x, v.y, q);
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), L2 only.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const u32 d = (u32)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Gentleman-Sande butterfly (inverse), lazy (Harvey), for every modulus below
// 2^62: inputs and outputs in [0, 2q); (a, b) -> (a + b, (a - b) w) mod q up
// to multiples of q (the lazy Shoup product of a word below 4q is in [0, 2q)).
// One form for all moduli keeps the passes to a single body: a launch of one
// or two CTAs per SM fetches a body's fully unrolled code from L2 line by
// line, and the special primes' small launches (ModDown sources) would
// otherwise run a body that the big launches never warm.
__device__ __forceinline__ void gs_w(u64& a, u64& b, u64 w, u64 ws, u64 q) {
    const u64 q2 = 2 * q;
    const u64 s = a + b;
    b = mul_shoup_lazy(a - b + q2, w, ws, q);
    a = s >= q2 ? s - q2 : s;
}
__device__ __forceinline__ void gs(u64& a, u64& b, const ulonglong2* tab, u32 idx, u64 q) {
    u64 w, ws;
    tw_at(tab, idx, w, ws);
    gs_w(a, b, w, ws, q);
}
// With a staged twiddle pair in shared memory.
__device__ __forceinline__ void gs_s(u64& a, u64& b, const ulonglong2& t, u64 q) {
    const ulonglong2 v = t;
    gs_w(a, b, v.x, v.y, q);
}

// Every pass works on "lines" of S = 2^LOGS words (a column of the R x C
// view in the column pass, a row in the row pass) with 16 words per thread
// and TPL = S/16 threads per line, in two layouts:
//   strided    : thread u holds line words u + TPL*v   (v = 0..15)
//   contiguous : thread u holds line words 16*u + v
// The four stages whose half-width is >= TPL pair words inside the strided
// layout (v and v + half/TPL); the other LOGS - 4 stages pair words inside
// the contiguous layout.  One shared-memory exchange sits between the two
// rounds.  Row passes keep each line inside one warp, so their exchanges
// need only __syncwarp; rows are padded by one word per 16 against bank
// conflicts.
__device__ __forceinline__ u32 pad16(u32 i) { return i + (i >> 4); }

// ------------------------------------------------------------------ forward, column pass
// Global stages 0..LOGS-1 (m = 2^ss, twiddle psi^brv(m + r / 2t_r)).
template <int LOGS, bool GROW>
// ts: the pass's twiddle pairs 0 .. S - 1, staged in shared memory (every
// column of a limb uses the same S - 1 pairs).
__device__ __forceinline__ void fwd_cols_stages(u64 (&x)[16], u64* sm, u32 u, u32 c, const ulonglong2* ts, u64 q) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, W = THREADS / TPL;
#pragma unroll
    for (int ss = 0; ss < 4; ss++) {
        const int tv = 8 >> ss;
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & tv)) ct_s<GROW>(x[v], x[v + tv], ts[(1u << ss) + (v >> (4 - ss))], q);
    }
#pragma unroll
    for (int v = 0; v < 16; v++) sm[(u + TPL * v) * W + c] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = sm[(16 * u + v) * W + c];
#pragma unroll
    for (int ss = 4; ss < LOGS; ss++) {
        const int t = S >> (ss + 1);
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & t)) ct_s<GROW>(x[v], x[v + t], ts[(1u << ss) + ((16 * u + v) >> (LOGS - ss))], q);
    }
}

// Basis conversion (Eq. 3) of a column-pass thread's 16 words, NS source
// limbs known at compile time (the constants held in registers), staged
// through the thread's own slots of the exchange buffer.  SMALL: sources and
// target below 2^41 (and the target above 2^32), so the four-term sums stay
// in 96 bits (mac96) and are reduced to [0, 3q) by a fold below 2^64 and a
// 32-bit quotient estimate (mu = floor(2^64 / q)); otherwise 128-bit sums
// reduced lazily to [0, 4q).  Either range feeds the butterflies.
template <int LOGS, int NS, bool SMALL>
__device__ __forceinline__ void bconv_words(u64* sm, const FwdJob& J, u32 u, u32 c, u32 col, u32 N, u32 C,
                                            const ModC& m) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, W = THREADS / TPL;
    u64 cst[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) cst[j] = J.bcst[j];
    const u64 q = m.q;
    const u64 c64 = 0 - q * m.mu_hi;                     // 2^64 mod q (mu_hi = floor(2^64 / q))
    const u64 c63 = (c64 + ((c64 & 1) ? q : 0)) >> 1;   // 2^63 mod q
    const u32 mu32 = (u32)m.mu_hi;
    const u64* src = J.src + (size_t)u * C + col;
#pragma unroll 4
    for (int v = 0; v < 16; v++) {
        const u64* p = src + (size_t)(TPL * v) * C;
        u64 y[NS];
#pragma unroll
        for (int j = 0; j < NS; j++) y[j] = p[(size_t)j * N];
        u64 r;
        if constexpr (SMALL) {
            U96 acc{0, 0};
#pragma unroll
            for (int j = 0; j < NS; j++) mac96(acc, y[j], cst[j]);
            const u64 f = (acc.lo & ~(1ull << 63)) + ((acc.lo >> 63) ? c63 : 0) + (u64)acc.hi * c64;
            const u64 qe = ((u64)(u32)(f >> 32) * mu32 + __umulhi((u32)f, mu32)) >> 32;
            r = f - qe * q;
        } else {
            U128 acc{0, 0};
#pragma unroll
            for (int j = 0; j < NS; j++) mac128(acc, y[j], cst[j]);
            r = reduce128_lazy(acc, m);
        }
        sm[(u + TPL * v) * W + c] = r;
    }
}

template <int LOGN, int LOGS, bool BCONV>
__global__ void __launch_bounds__(THREADS, 4) k_fwd_cols(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<FwdJob> jobs) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, W = THREADS / TPL;
    __shared__ u64 sm[S * W];
    __shared__ __align__(16) ulonglong2 ts[S];
    constexpr u32 N = 1u << LOGN, C = N >> LOGS;
    const u32 c = threadIdx.x % W, u = threadIdx.x / W;
    const u32 col = blockIdx.x * W + c;
    const FwdJob& J = jobs.j[blockIdx.y];
    const ModC m = T.mods[J.mod];
    const u64 q = m.q;
    const ulonglong2* tw = T.psi + (size_t)J.mod * N;
    if (J.nsrc & FWD_COPY) {  // a pass-through limb: the block copies its columns (every word loaded first)
        u64 y[16];
        if (J.nsrc & FWD_SCALE) {
#pragma unroll
            for (int v = 0; v < 16; v++) y[v] = mul_shoup(J.src[(u + TPL * v) * C + col], J.c, J.c_sh, q);
        } else {
            const u32 gal = (u32)J.c;
#pragma unroll
            for (int v = 0; v < 16; v++) {
                const u32 idx = (u + TPL * v) * C + col;
                y[v] = J.src[gal ? auto_src(idx, gal, LOGN) : idx];
            }
        }
#pragma unroll
        for (int v = 0; v < 16; v++) J.dst[(size_t)(u + TPL * v) * C + col] = y[v];
        return;
    }
    // the S - 1 twiddle pairs of the column stages (indices 1 .. S - 1), copied while the words load
    if (threadIdx.x < S) cp_async16(&ts[threadIdx.x], tw + threadIdx.x);
    cp_async_commit();
    u64 x[16];
    if constexpr (BCONV) {
        // basis conversion (Eq. 3) of the thread's 16 words, staged through its
        // own slots of the exchange buffer so that this part stays a compact loop
        const u32 ns = J.nsrc & 0xFFFFu;
        const bool small = ((J.nsrc >> 16) & 1u) && q > (1ull << 32) && q < (1ull << 41);
        if (ns == 4 && small) bconv_words<LOGS, 4, true>(sm, J, u, c, col, N, C, m);
        else if (ns == 4) bconv_words<LOGS, 4, false>(sm, J, u, c, col, N, C, m);
        else if (ns == 5) bconv_words<LOGS, 5, false>(sm, J, u, c, col, N, C, m);
        else {
            const u64* bc = J.bcst;
#pragma unroll 4
            for (int v = 0; v < 16; v++) {
                const u64* src = J.src + (size_t)(u + TPL * v) * C + col;
                U128 acc{0, 0};
                for (u32 j = 0; j < ns; j++) mac128(acc, src[(size_t)j * N], bc[j]);
                sm[(u + TPL * v) * W + c] = reduce128_lazy(acc, m);  // [0, 4q): both butterfly forms take it
            }
        }
#pragma unroll
        for (int v = 0; v < 16; v++) x[v] = sm[(u + TPL * v) * W + c];
    } else {
#pragma unroll
        for (int v = 0; v < 16; v++) x[v] = J.src[(size_t)(u + TPL * v) * C + col];
    }
    cp_async_wait_all();
    __syncthreads();
    // words enter below 4q; they leave below 4q (reducing) or 36q (growing: +4q per stage),
    // and the row pass ends below 68q < 2^64 (q < 2^57)
    if (q < FWD_GROW_MAX) fwd_cols_stages<LOGS, true>(x, sm, u, c, ts, q);
    else fwd_cols_stages<LOGS, false>(x, sm, u, c, ts, q);
#pragma unroll
    for (int v = 0; v < 16; v++) J.dst[(size_t)(16 * u + v) * C + col] = x[v];
}

// ------------------------------------------------------------------ forward, row pass
// Global stages log_r..log_n-1 (m = 2^(log_r+ss), twiddle psi^brv(m + row 2^ss + x / 2t)).
// The row pass's first round (stages 0-3) uses 15 twiddle pairs per row,
// shared by the row's threads.  The kernel stages them in shared memory (t1,
// slot 2^ss - 1 + j), copied asynchronously while the row's words load, so
// that the round's butterflies do not wait on L2 stage by stage.  Rows are 15
// pairs (240 bytes) apart: an odd number of 16-byte slots, so the rows of one
// warp (2, 4 or 8) read different banks.  The second round's pairs (240 per
// row, each used by one thread) are read from L2 as needed: staging those
// too cost more (copies and 32 KB per CTA) than their latency.
constexpr u32 T1_STRIDE = 15;
template <int LOGS, bool GROW>
__device__ __forceinline__ void fwd_rows_stages(u64 (&x)[16], u64* sr, u32 u, u32 row, u32 log_r,
                                                const ulonglong2* tw, u64 q, const ulonglong2* t1) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16;
#pragma unroll
    for (int ss = 0; ss < 4; ss++) {
        const int tv = 8 >> ss;
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & tv)) ct_s<GROW>(x[v], x[v + tv], t1[(1 << ss) - 1 + (v >> (4 - ss))], q);
    }
#pragma unroll
    for (int v = 0; v < 16; v++) sr[pad16(u + TPL * v)] = x[v];
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = sr[pad16(16 * u + v)];
#pragma unroll
    for (int ss = 4; ss < LOGS; ss++) {
        const int t = S >> (ss + 1);
        const u32 b0 = (1u << (log_r + ss)) + (row << ss);
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & t)) ct<GROW>(x[v], x[v + t], tw, b0 + ((16 * u + v) >> (LOGS - ss)), q);
    }
}

// Issues the copies of a row's first-round twiddles into t1 (the caller commits and waits).
template <int LOGS>
__device__ __forceinline__ void fwd_rows_stage_twiddles(const ulonglong2* tw, u32 u, u32 row, u32 log_r,
                                                        ulonglong2* t1) {
    constexpr u32 TPL = (1u << LOGS) / 16;
    for (u32 k = u; k < 15; k += TPL) {
        const u32 ss = 31 - __clz(k + 1), j = k + 1 - (1u << ss);
        cp_async16(&t1[k], tw + (1u << (log_r + ss)) + (row << ss) + j);
    }
}

// The row pass of one limb in one arithmetic class (chosen once per block, so
// that each class is compiled and register-allocated on its own):
// AR = 0: reducing butterflies, words below 4q;
// AR = 1: growing butterflies, words below 68q, reduced by red2;
// AR = 2: growing butterflies with 2^32 < q < 2^41, reduced by red3_small.
// Every class occurs in the big Decompose launches (special-prime, first-prime
// and 40-bit targets), so none runs cold in a small launch.
template <int LOGN, int LOGS, bool SUBMUL, int AR>
__device__ __forceinline__ void fwd_rows_limb(const FwdJob& J, const ModC& m, const ulonglong2* tw, u64* sr,
                                              const ulonglong2* t1, u32 u, u32 row) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, log_r = LOGN - LOGS;
    const u64 q = m.q;
    const size_t base = (size_t)row * S;
    u64 x[16];
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = J.dst[base + u + TPL * v];
    cp_async_wait_all();
    __syncwarp();  // a row's threads are lanes of one warp
    fwd_rows_stages<LOGS, (AR > 0)>(x, sr, u, row, log_r, tw, q, t1);
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) sr[pad16(16 * u + v)] = x[v];
    // The ModDown tail's x words, every one loaded before this thread's first
    // store.  The compiler cannot tell that the output limbs never overlap
    // them, so loads interleaved with the stores could not move ahead of them
    // and would each wait a full round trip.
    u64 sx[SUBMUL ? 16 : 1];
    if constexpr (SUBMUL) {
#pragma unroll
        for (int v = 0; v < 16; v++) sx[v] = J.subx[base + u + TPL * v];
    }
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) {
        const u32 xi = u + TPL * v;
        const u64 y = sr[pad16(xi)];
        u64 val;
        if constexpr (AR == 2) {  // below 68q < 2^48 -> [0, 3q)
            val = red3_small(y, q, (u32)m.mu_hi);
            val = val >= 2 * q ? val - 2 * q : val;
            val = val >= q ? val - q : val;
        } else if constexpr (AR == 1) {  // below 68q
            val = red2(y, q, m.mu_hi);
            val = val >= q ? val - q : val;
        } else {  // below 4q
            val = canon4(y, q);
        }
        if constexpr (SUBMUL) {
            J.subout[base + xi] = mul_shoup(sub_mod(sx[v], val, q), J.c, J.c_sh, q);
        } else {
            J.dst[base + xi] = val;
        }
    }
}

// Shared memory of k_fwd_rows: the exchange rows, then t1 (38 KB at N = 2^16, 49 KB at 2^12).
template <int LOGS>
constexpr size_t fwd_rows_smem() {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, B = THREADS / TPL, SP = S + S / 16;
    return (size_t)B * SP * 8 + (size_t)B * T1_STRIDE * 16;
}

// Three CTAs per SM (80 registers; measured faster than four at 64).
template <int LOGN, int LOGS, bool SUBMUL>
__global__ void __launch_bounds__(THREADS, 3) k_fwd_rows(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<FwdJob> jobs) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, B = THREADS / TPL, SP = S + S / 16;
    constexpr u32 N = 1u << LOGN, log_r = LOGN - LOGS;
    extern __shared__ __align__(16) u64 dsm[];
    u64* sm = dsm;
    ulonglong2* t1s = (ulonglong2*)(dsm + B * SP);
    const u32 u = threadIdx.x % TPL, rl = threadIdx.x / TPL;
    const u32 row = blockIdx.x * B + rl;
    const FwdJob& J = jobs.j[blockIdx.y];
    if (J.nsrc & FWD_COPY) return;  // copied by the column pass
    const ModC m = T.mods[J.mod];
    const ulonglong2* tw = T.psi + (size_t)J.mod * N;
    u64* sr = sm + rl * SP;
    ulonglong2* t1 = t1s + rl * T1_STRIDE;
    fwd_rows_stage_twiddles<LOGS>(tw, u, row, log_r, t1);
    cp_async_commit();
    if (small_q(m.q)) fwd_rows_limb<LOGN, LOGS, SUBMUL, 2>(J, m, tw, sr, t1, u, row);
    else if (m.q < FWD_GROW_MAX) fwd_rows_limb<LOGN, LOGS, SUBMUL, 1>(J, m, tw, sr, t1, u, row);
    else fwd_rows_limb<LOGN, LOGS, SUBMUL, 0>(J, m, tw, sr, t1, u, row);
}

// Sets a kernel's dynamic shared memory limit once per device.
template <typename K>
void smem_limit(K kernel, size_t bytes, std::atomic<uint64_t>& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;  // the launch reports it
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
        done.fetch_or(bit, std::memory_order_release);
}

// ------------------------------------------------------------------ inverse, row pass
// GS stages with half-width t = 1..S/2 (m = N/2t, twiddle psi^-brv(m + row S/2t + x/2t)).
// Words enter below q (canonical) and stay in [0, 2q).
template <int LOGS>
__device__ __forceinline__ void inv_rows_stages(u64 (&x)[16], u64* sr, u32 u, u32 row, u32 N,
                                                const ulonglong2* tw, u64 q) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16;
#pragma unroll
    for (int lt = 0; lt < LOGS - 4; lt++) {  // t = 1 .. TPL/2
        const int t = 1 << lt;
        const u32 b0 = (N >> (lt + 1)) + row * (S >> (lt + 1));
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & t)) gs(x[v], x[v + t], tw, b0 + ((16 * u + v) >> (lt + 1)), q);
    }
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) sr[pad16(16 * u + v)] = x[v];
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = sr[pad16(u + TPL * v)];
#pragma unroll
    for (int k = 0; k < 4; k++) {  // t = TPL * 2^k
        const int lt = (LOGS - 4) + k;
        const u32 b0 = (N >> (lt + 1)) + row * (S >> (lt + 1));
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & (1 << k))) gs(x[v], x[v + (1 << k)], tw, b0 + (v >> (k + 1)), q);
    }
}

template <int LOGN, int LOGS, bool GATHER>
__global__ void __launch_bounds__(THREADS, 3) k_inv_rows(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<InvJob> jobs) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, B = THREADS / TPL, SP = S + S / 16;
    __shared__ u64 sm[B * SP];
    constexpr u32 N = 1u << LOGN;
    const u32 u = threadIdx.x % TPL, rl = threadIdx.x / TPL;
    const u32 row = blockIdx.x * B + rl;
    const InvJob& J = jobs.j[blockIdx.y];
    const u64 q = T.mods[J.mod].q;
    const ulonglong2* tw = T.ipsi + (size_t)J.mod * N;
    u64* sr = sm + rl * SP;
    const size_t base = (size_t)row * S;
    u64 x[16];
#pragma unroll
    for (int v = 0; v < 16; v++) {
        const u32 xi = u + TPL * v;
        if constexpr (GATHER) x[v] = J.src[auto_src((u32)(base + xi), J.gal, LOGN)];
        else x[v] = J.src[base + xi];
    }
#pragma unroll
    for (int v = 0; v < 16; v++) sr[pad16(u + TPL * v)] = x[v];
    __syncwarp();
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = sr[pad16(16 * u + v)];
    inv_rows_stages<LOGS>(x, sr, u, row, N, tw, q);  // [0, 2q)
#pragma unroll
    for (int v = 0; v < 16; v++) J.tmp[base + u + TPL * v] = x[v];
}

// ------------------------------------------------------------------ inverse, column pass
// GS stages with half-width C*t_r, t_r = 1..S/2 (m = S/2t_r, twiddle psi^-brv(m + r/2t_r)),
// then the scaling by c (N^-1 and any per-limb constant).  Words enter and stay in [0, 2q).
// ts: the pass's twiddle pairs 0 .. S - 1, staged in shared memory.
template <int LOGS>
__device__ __forceinline__ void inv_cols_stages(u64 (&x)[16], u64* sm, u32 u, u32 c, const ulonglong2* ts, u64 q) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, W = THREADS / TPL;
#pragma unroll
    for (int lt = 0; lt < LOGS - 4; lt++) {
        const int t = 1 << lt;
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & t)) gs_s(x[v], x[v + t], ts[(S >> (lt + 1)) + ((16 * u + v) >> (lt + 1))], q);
    }
#pragma unroll
    for (int v = 0; v < 16; v++) sm[(16 * u + v) * W + c] = x[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = sm[(u + TPL * v) * W + c];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int lt = (LOGS - 4) + k;
#pragma unroll
        for (int v = 0; v < 16; v++)
            if (!(v & (1 << k))) gs_s(x[v], x[v + (1 << k)], ts[(S >> (lt + 1)) + (v >> (k + 1))], q);
    }
}

template <int LOGN, int LOGS>
__global__ void __launch_bounds__(THREADS, 3) k_inv_cols(const __grid_constant__ NttTables T,
                                                      const __grid_constant__ Jobs<InvJob> jobs) {
    constexpr u32 S = 1u << LOGS, TPL = S / 16, W = THREADS / TPL;
    __shared__ u64 sm[S * W];
    __shared__ __align__(16) ulonglong2 ts[S];
    constexpr u32 N = 1u << LOGN, C = N >> LOGS;
    const u32 c = threadIdx.x % W, u = threadIdx.x / W;
    const u32 col = blockIdx.x * W + c;
    const InvJob& J = jobs.j[blockIdx.y];
    const u64 q = T.mods[J.mod].q;
    const ulonglong2* tw = T.ipsi + (size_t)J.mod * N;
    // the S - 1 twiddle pairs of the column stages (indices 1 .. S - 1), copied while the words load
    if (threadIdx.x < S) cp_async16(&ts[threadIdx.x], tw + threadIdx.x);
    cp_async_commit();
    u64 x[16];
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = J.tmp[(size_t)(16 * u + v) * C + col];
    cp_async_wait_all();
    __syncthreads();
    inv_cols_stages<LOGS>(x, sm, u, c, ts, q);
    // the scaling: mul_shoup reduces any 64-bit word fully
#pragma unroll
    for (int v = 0; v < 16; v++) J.dst[(size_t)(u + TPL * v) * C + col] = mul_shoup(x[v], J.c, J.c_sh, q);
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

template <typename J, typename F>
void for_chunks(const J* jobs, int njobs, F&& f) {
    for (int s = 0; s < njobs; s += MAXJ) {
        Jobs<J> pack;
        const int n = std::min(MAXJ, njobs - s);
        for (int i = 0; i < n; i++) pack.j[i] = jobs[s + i];
        f(pack, n);
    }
}

template <int LR, int LC>
void fwd_impl(const NttTables& T, const Jobs<FwdJob>& p, int n, bool bconv, bool submul, cudaStream_t st) {
    const u32 N = 1u << T.log_n;
    const dim3 g1((N >> LR) / (THREADS / ((1u << LR) / 16)), n), g2((N >> LC) / (THREADS / ((1u << LC) / 16)), n);
    int nt = 0;  // transformed limbs (copy jobs aside)
    for (int i = 0; i < n; i++) nt += (p.j[i].nsrc & FWD_COPY) ? 0 : 1;
    const double half = (double)nt * (N / 2);  // butterflies per stage over the launch's limbs
    double bconv_macs = 0;
    if (bconv)
        for (int i = 0; i < n; i++)
            if (!(p.j[i].nsrc & FWD_COPY)) bconv_macs += (double)(p.j[i].nsrc & 0xFFFFu) * N;
    {
        ProfScope ps(K_FWD_COLS, st, bconv_macs, half * LR);
        if (bconv) k_fwd_cols<LR + LC, LR, true><<<g1, THREADS, 0, st>>>(T, p);
        else k_fwd_cols<LR + LC, LR, false><<<g1, THREADS, 0, st>>>(T, p);
    }
    {
        ProfScope ps(K_FWD_ROWS, st, 0, half * LC);
        constexpr size_t sm = fwd_rows_smem<LC>();
        static std::atomic<uint64_t> lim_t{0}, lim_f{0};
        if (submul) {
            smem_limit(k_fwd_rows<LR + LC, LC, true>, sm, lim_t);
            k_fwd_rows<LR + LC, LC, true><<<g2, THREADS, sm, st>>>(T, p);
        } else {
            smem_limit(k_fwd_rows<LR + LC, LC, false>, sm, lim_f);
            k_fwd_rows<LR + LC, LC, false><<<g2, THREADS, sm, st>>>(T, p);
        }
    }
}

template <int LR, int LC>
void inv_impl(const NttTables& T, const Jobs<InvJob>& p, int n, bool gather, cudaStream_t st) {
    const u32 N = 1u << T.log_n;
    const dim3 g1((N >> LR) / (THREADS / ((1u << LR) / 16)), n), g2((N >> LC) / (THREADS / ((1u << LC) / 16)), n);
    const double half = (double)n * (N / 2);
    {
        ProfScope ps(K_INV_ROWS, st, 0, half * LC);
        if (gather) k_inv_rows<LR + LC, LC, true><<<g2, THREADS, 0, st>>>(T, p);
        else k_inv_rows<LR + LC, LC, false><<<g2, THREADS, 0, st>>>(T, p);
    }
    {
        ProfScope ps(K_INV_COLS, st, 0, half * LR);
        k_inv_cols<LR + LC, LR><<<g1, THREADS, 0, st>>>(T, p);
    }
}

// N = 2^log_n is viewed as R x C with log R = ceil(log_n / 2).
#define NTT_DISPATCH(IMPL, ...)                                   \
    switch (T.log_n) {                                            \
        case 12: IMPL<6, 6>(T, p, n, __VA_ARGS__, st); break;    \
        case 13: IMPL<7, 6>(T, p, n, __VA_ARGS__, st); break;    \
        case 14: IMPL<7, 7>(T, p, n, __VA_ARGS__, st); break;    \
        case 15: IMPL<8, 7>(T, p, n, __VA_ARGS__, st); break;    \
        default: IMPL<8, 8>(T, p, n, __VA_ARGS__, st); break; /* 16: contexts take 12..16 */ \
    }

// ------------------------------------------------------------------ integer-rate probes
// Register-only loops of the library's own arithmetic, the denominators of
// the integer-ALU roofline: k_probe_mac runs mac128 into 8 independent
// accumulators per thread, k_probe_bfly runs radix-16 rounds (4 stages of 8
// growing forward butterflies, ct<true>) on 16 words per thread with the 15
// twiddles of a round held in registers.  Each thread writes one word so that
// nothing is optimised away; the values themselves are meaningless.
constexpr int PROBE_ITERS = 1024, PROBE_THREADS = 256, PROBE_MACS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_mac(const u64* __restrict__ in, u64* __restrict__ out) {
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    u64 b[PROBE_MACS];
    U128 acc[PROBE_MACS];
#pragma unroll
    for (int k = 0; k < PROBE_MACS; k++) {
        b[k] = in[(tid + k) & 1023];
        acc[k] = U128{0, 0};
    }
    u64 x = in[tid & 1023];
    for (int i = 0; i < PROBE_ITERS; i++) {
        x ^= (u64)i;
#pragma unroll
        for (int k = 0; k < PROBE_MACS; k++) mac128(acc[k], x, b[k]);
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < PROBE_MACS; k++) r ^= acc[k].lo ^ acc[k].hi;
    out[tid] = r;
}

__global__ void __launch_bounds__(PROBE_THREADS, 4) k_probe_bfly(const ulonglong2* __restrict__ tw,
                                                                 const u64* __restrict__ in, u64* __restrict__ out,
                                                                 u64 q) {
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[16];
#pragma unroll
    for (int v = 0; v < 16; v++) x[v] = in[(tid * 16 + v) & 1023];
    for (int i = 0; i < PROBE_ITERS; i++) {
#pragma unroll
        for (int ss = 0; ss < 4; ss++) {
            const int tv = 8 >> ss;
#pragma unroll
            for (int v = 0; v < 16; v++)
                if (!(v & tv)) ct<true>(x[v], x[v + tv], tw, (1u << ss) + (v >> (4 - ss)), q);
        }
    }
    u64 r = 0;
#pragma unroll
    for (int v = 0; v < 16; v++) r ^= x[v] * (u64)(v + 1);
    out[tid] = r;
}

}  // namespace

void launch_fwd_ntt(const NttTables& T, const FwdJob* jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return;
    // every transform job of a launch is of one kind (copy jobs may join any)
    bool bconv = false, submul = false;
    for (int i = 0; i < njobs; i++)
        if (!(jobs[i].nsrc & FWD_COPY)) {
            bconv = (jobs[i].nsrc & 0xFFFFu) > 0;
            submul = jobs[i].subout != nullptr;
            break;
        }
    for_chunks(jobs, njobs, [&](const Jobs<FwdJob>& p, int n) {
        NTT_DISPATCH(fwd_impl, bconv, submul);
        count_launch(2);
    });
}

void launch_inv_ntt(const NttTables& T, const InvJob* jobs, int njobs, cudaStream_t st) {
    if (njobs <= 0) return;
    const bool gather = jobs[0].gal != 0;
    for_chunks(jobs, njobs, [&](const Jobs<InvJob>& p, int n) {
        NTT_DISPATCH(inv_impl, gather);
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

cudaError_t probe_int_rates(u32 blocks, double* macs_per_s, double* butterflies_per_s) {
    // q: any odd modulus below 2^57 (the growing butterflies' range); the
    // twiddles are arbitrary residues with their Shoup companions
    const u64 q = (1ull << 56) - 5;
    u64 h_in[1024];
    ulonglong2 h_tw[16];
    for (int i = 0; i < 1024; i++) h_in[i] = (0x9E3779B97F4A7C15ull * (u64)(i + 1)) % q;
    for (int i = 0; i < 16; i++) {
        const u64 w = (0xD1B54A32D192ED03ull * (u64)(i + 3)) % q;
        h_tw[i] = make_ulonglong2(w, (u64)(((unsigned __int128)w << 64) / q));
    }
    u64 *in = nullptr, *out = nullptr;
    ulonglong2* tw = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaSuccess;
    float best[2] = {0, 0};
    auto step = [&](cudaError_t e) {
        if (err == cudaSuccess) err = e;
        return err == cudaSuccess;
    };
    if (step(cudaMalloc(&in, sizeof(h_in))) && step(cudaMalloc(&tw, sizeof(h_tw))) &&
        step(cudaMalloc(&out, (size_t)blocks * PROBE_THREADS * sizeof(u64))) &&
        step(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) && step(cudaEventCreate(&e0)) &&
        step(cudaEventCreate(&e1)) && step(cudaMemcpyAsync(in, h_in, sizeof(h_in), cudaMemcpyHostToDevice, st)) &&
        step(cudaMemcpyAsync(tw, h_tw, sizeof(h_tw), cudaMemcpyHostToDevice, st))) {
        for (int which = 0; which < 2 && err == cudaSuccess; which++)
            for (int rep = 0; rep < 3 && err == cudaSuccess; rep++) {  // the first run warms up
                step(cudaEventRecord(e0, st));
                if (which == 0) k_probe_mac<<<blocks, PROBE_THREADS, 0, st>>>(in, out);
                else k_probe_bfly<<<blocks, PROBE_THREADS, 0, st>>>(tw, in, out, q);
                count_launch();
                step(cudaGetLastError());
                step(cudaEventRecord(e1, st));
                step(cudaEventSynchronize(e1));
                float ms = 0;
                if (step(cudaEventElapsedTime(&ms, e0, e1)) && rep > 0 && (best[which] == 0 || ms < best[which]))
                    best[which] = ms;
            }
    }
    if (st) cudaStreamSynchronize(st);
    if (in) cudaFree(in);
    if (tw) cudaFree(tw);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (err != cudaSuccess) return err;
    const double threads = (double)blocks * PROBE_THREADS;
    *macs_per_s = threads * PROBE_ITERS * PROBE_MACS / (best[0] * 1e-3);
    *butterflies_per_s = threads * PROBE_ITERS * 32 / (best[1] * 1e-3);
    return cudaSuccess;
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
