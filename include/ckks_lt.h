/*
 * ckks_lt.h - C ABI of the GB300 library for the CKKS homomorphic linear
 * transformation (plaintext matrix times encrypted slot vector).
 *
 * Paper: S. Akherati, X. Zhang, "Triple-Hoisted Baby-Step Giant-Step Linear
 * Transformation over CKKS Homomorphic Encryption and Hardware Accelerator".
 * The calls follow the paper's problem statement: an RNS-CKKS context
 * (Sec. II-A; parameter sets as in Table "HE parameters": N, L+1, alpha, beta),
 * rotation (Galois) keys, a ciphertext, the encoded diagonals of the matrix
 * and their offsets, and the LT algorithm: diagonal method (Sec. II-B),
 * BSGS (Eq. 5), double-hoisted BSGS (Algorithm 1) or triple-hoisted BSGS
 * (Algorithm 2, Eq. 6).
 *
 * Data conventions (every call):
 *   - A "limb" is N uint64 words holding residues modulo one prime, canonical
 *     in [0, q).  A polynomial is consecutive limbs.
 *   - Ring elements are in the NTT domain, bit-reversed order: word s of a
 *     limb holds a(psi^(2*brv(s)+1)), psi the primitive 2N-th root of unity
 *     x^((q-1)/2N) for the smallest integer x >= 2 with psi^N = -1 (mod q).
 *   - The context's moduli are q_0..q_{L-1} (the Q chain) then p_0..p_{k-1}
 *     (special primes, P = prod p_i).  Every modulus must be prime, = 1 mod 2N,
 *     below 2^60, and all must be distinct.
 *   - A ciphertext at level l has l Q limbs: layout [2][l][N] (c0 then c1).
 *   - An "extended" polynomial at level l has l + k limbs: q_0..q_{l-1} then
 *     p_0..p_{k-1}.
 *   - alpha = ceil(L / dnum) limbs per digit; at level l there are
 *     beta_l = ceil(l / alpha) digits, digit b holding Q limbs
 *     [alpha*b, min(alpha*(b+1), l)).
 *   - Rotation by r slots is to the left: new slot j = old slot j + r, through
 *     the automorphism x -> x^(5^r mod 2N) (Eq. 2).
 *
 * Ownership: the library copies host buffers into device memory it owns;
 * handles are freed with the matching ckks_free_* call and all of them by
 * ckks_ctx_destroy.  Buffers passed as device pointers stay owned by the
 * caller and must outlive every call that uses them.
 *
 * Errors: every call returns a ckks_status; nothing is thrown across the ABI.
 * ckks_last_error() gives a message for the calling thread.  Validation
 * failures return before any device work is queued.
 *
 * Threads: evaluation calls (lt_eval*, the steps, the autotuners) on one
 * context may run concurrently from several host threads, each on its own
 * stream.  Uploading or replacing keys and diagonals, allocating
 * library-owned ciphertexts (ckks_ct_create, ckks_ct_upload) and destroying
 * objects update the context's tables and memory count: such calls must not
 * overlap each other or evaluation calls on the same context.  Wrapping
 * caller memory (ckks_ct_wrap_device) and freeing a wrapped handle may run at
 * any time.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls that take a stream are asynchronous on it unless stated.
 * Device scratch memory is taken from the stream-ordered allocator of the
 * context's device and returned on the same stream.
 */
#ifndef CKKS_LT_H
#define CKKS_LT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ckks_ctx ckks_ctx;
typedef struct ckks_ct ckks_ct;
typedef struct ckks_diags ckks_diags;

typedef enum {
    CKKS_OK = 0,
    CKKS_EINVAL = 1,   /* bad argument, shape, level or split            */
    CKKS_ENOMEM = 2,   /* device or host allocation failed               */
    CKKS_ENOKEY = 3,   /* a rotation key the algorithm needs is missing  */
    CKKS_ECUDA = 4,    /* a CUDA runtime call failed                     */
    CKKS_ETIMEOUT = 5, /* a bounded device-side wait gave up             */
    CKKS_EBUSY = 6     /* resource in use                                */
} ckks_status;

typedef enum {
    LT_DIAG = 0,     /* diagonal method, hoisted (Sec. II-B)             */
    LT_BSGS = 1,     /* baby-step giant-step (Eq. 5)                     */
    LT_DH_BSGS = 2,  /* double-hoisted BSGS (Algorithm 1)                */
    LT_TH_BSGS = 3   /* triple-hoisted BSGS (Algorithm 2)                */
} lt_algo;

/* Baby/giant split: TH uses (n'1, n'2, n'3) with n1*n2*n3 = D; BSGS and DH
 * use (n1, n2) with n3 = 1 and n1*n2 = D; the diagonal method ignores it.
 * All zero (or a NULL pointer) asks the library to choose. */
typedef struct {
    uint32_t n1, n2, n3;
} lt_split;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device` for ring degree N = 2^log_n
 * (12 <= log_n <= 16), Q chain q[0..n_q-1], special primes p[0..n_p-1]
 * (n_p >= 1) and dnum digits at the top level (Sec. II-A, Fig. 1).
 * Computes and uploads every constant (twiddles, basis-conversion tables).
 * EINVAL on a modulus that is not an NTT-friendly prime below 2^60. */
ckks_status ckks_ctx_create(ckks_ctx** out, uint32_t log_n, const uint64_t* q, uint32_t n_q,
                            const uint64_t* p, uint32_t n_p, uint32_t dnum, int device);
ckks_status ckks_ctx_destroy(ckks_ctx* ctx);

/* Upload the switching key from phi_r(s) to s for left rotation by r slots,
 * in standard (un-hoisted) form (Fig. 1).  Host layout [beta_max][2][L+k][N]
 * (beta_max = ceil(L/alpha); all L Q limbs then all k P limbs), n_words must
 * equal beta_max*2*(L+k)*N.  The same key serves every algorithm and split:
 * the hoisted form swk~_r = phi_{-r}(swk_r) of Algorithms 1-2 is applied as
 * an index gather on the digits.  r is taken mod N/2; replacing a key is
 * allowed when no queued work uses it.  The library stores the key with its
 * two components interleaved per word ([beta_max][L+k][N] pairs), so that
 * every kernel reads one 16-byte word per digit word; the upload converts. */
ckks_status ckks_upload_rotation_key(ckks_ctx* ctx, int32_t r, const uint64_t* host, size_t n_words);
/* Same, from a device buffer the library reads in stream order on `stream`
 * (the conversion is a kernel there; `dev` must stay valid until it ran). */
ckks_status ckks_upload_rotation_key_device(ckks_ctx* ctx, int32_t r, const uint64_t* dev,
                                            size_t n_words, void* stream);
int ckks_has_rotation_key(const ckks_ctx* ctx, int32_t r);

/* Upload the encoded, un-rotated diagonals f_t (t < n_diag) of the matrix,
 * with offsets o_t = offset0 + stride*t (Sec. II-B: f_t packs diagonal o_t).
 * Host layout [n_diag][level + k][N]: Q limbs q_0..q_{level-1} then the k P
 * limbs, NTT domain.  `level` is the level the diagonals were encoded at; an
 * LT at a ciphertext level l <= level uses the first l Q limbs and the P
 * limbs.  offset0 lies in (-N/2, N/2) (EINVAL otherwise), stride >= 1 and
 * stride*(n_diag-1) < N/2, so that the n_diag offsets are distinct mod N/2.
 * A nonzero offset0 joins the outermost rotation layer of each algorithm:
 * with g_t = Rot(f_t, -offset0), sum_t f_t . Rot(z, offset0 + stride t) =
 * Rot(sum_t g_t . Rot(z, stride t), offset0), so the giant (BSGS, DH-BSGS)
 * or outer (TH-BSGS) amounts become offset0 + stride*n1(*n2)*k for every k,
 * the first included, and the diagonal method ends with one rotation by
 * offset0 (one more key, Decompose and ModDown).  An amount that is 0 mod
 * N/2 needs no key.  Such windows o_t = -m*s .. m*s are the sparse stages of
 * a factored DFT (CoeffToSlot / SlotToCoeff). */
ckks_status ckks_upload_diagonals(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0,
                                  int32_t stride, uint32_t level, const uint64_t* host, size_t n_words);
/* Same, from a device buffer the library copies (stream-ordered on `stream`). */
ckks_status ckks_upload_diagonals_device(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0,
                                         int32_t stride, uint32_t level, const uint64_t* dev, size_t n_words,
                                         void* stream);
/* Allocate diagonals without contents (layout as above), to be filled with
 * ckks_diags_write_device, e.g. in pieces when the whole matrix is too large
 * to stage twice in device memory. */
ckks_status ckks_diags_create(ckks_ctx* ctx, ckks_diags** out, uint32_t n_diag, int32_t offset0, int32_t stride,
                              uint32_t level);
/* Copy diagonals [first, first + count) from a device buffer
 * [count][level + k][N] (stream-ordered). */
ckks_status ckks_diags_write_device(ckks_diags* f, uint32_t first, uint32_t count, const uint64_t* dev,
                                   size_t n_words, void* stream);
ckks_status ckks_free_diags(ckks_diags* f);

/* ------------------------------------------------------------------ ciphertexts */

/* New device ciphertext at `level` (library-owned, contents undefined). */
ckks_status ckks_ct_create(ckks_ctx* ctx, ckks_ct** out, uint32_t level);
/* New device ciphertext holding a copy of host [2][level][N] (synchronous). */
ckks_status ckks_ct_upload(ckks_ctx* ctx, ckks_ct** out, uint32_t level, const uint64_t* host);
/* Wrap caller-owned device memory [2][level][N] (e.g. a torch tensor). */
ckks_status ckks_ct_wrap_device(ckks_ctx* ctx, ckks_ct** out, uint32_t level, uint64_t* dev_ptr);
/* Stream-ordered copies between a ciphertext and host memory (pinned host
 * memory makes them asynchronous; n_words must be 2*level*N). */
ckks_status ckks_ct_h2d_async(ckks_ct* ct, const uint64_t* host, size_t n_words, void* stream);
ckks_status ckks_ct_d2h_async(const ckks_ct* ct, uint64_t* host, size_t n_words, void* stream);
/* Synchronous download (waits for the whole device). */
ckks_status ckks_ct_download(const ckks_ct* ct, uint64_t* host, size_t n_words);
uint32_t ckks_ct_level(const ckks_ct* ct);
uint64_t* ckks_ct_device_ptr(const ckks_ct* ct);
ckks_status ckks_free_ct(ckks_ct* ct);

/* ------------------------------------------------------------------ the LT */

/* out <- LT_F(in): the diagonals f applied to `in` by algorithm `algo` with
 * `split` (NULL or all-zero = the library's choice, written to `chosen` if it
 * is not NULL).  `out` must have level in->level - 1: the hoisted algorithms
 * end with ModDown merged with rescale (Algorithm 2 line 19), BSGS with the
 * rescale of Eq. (1).  Rotation amounts are multiples of f's stride; ENOKEY
 * when a needed key is missing.  in->level must be >= 2 and <= f's level.
 * Asynchronous on `stream`. */
ckks_status lt_eval(ckks_ctx* ctx, const ckks_ct* in, const ckks_diags* f, lt_algo algo,
                    const lt_split* split, ckks_ct* out, void* stream, lt_split* chosen);

/* `count` independent LTs, possibly at different levels and with different
 * diagonal sets, queued as one unit on `stream`: LTs that share a diagonal
 * set and level are evaluated together so that every key and diagonal limb is
 * read from HBM once per group.  algos may be NULL (TH-BSGS for all);
 * splits may be NULL (library choice).  Results equal count separate
 * lt_eval calls bit for bit when the same splits are used. */
ckks_status lt_eval_batch(ckks_ctx* ctx, uint32_t count, const ckks_ct* const* in,
                          const ckks_diags* const* f, const lt_algo* algos, const lt_split* splits,
                          ckks_ct* const* out, void* stream);

/* A chain of LTs, one level each: the stages of a factored transform such as
 * the CoeffToSlot / SlotToCoeff DFTs of bootstrapping, the multi-stage sparse
 * LTs the hoisted algorithms target (Sec. I).  Stage i evaluates LT_{f[i]} at
 * level in->level - i on the previous stage's output (stage 0 on `in`);
 * `out` receives the last stage's result, at level in->level - n_stages.
 * algos/splits: per stage, or NULL for TH-BSGS with the library's split (the
 * tuned one if lt_autotune ran for that shape).  Every stage is validated --
 * levels, splits, keys -- before anything is queued.  Intermediate
 * ciphertexts come from the stream-ordered allocator on `stream` and are
 * released in stream order.  chosen (may be NULL) receives each stage's
 * split.  Each stage's residues equal those of a separate lt_eval. */
ckks_status lt_eval_chain(ckks_ctx* ctx, const ckks_ct* in, uint32_t n_stages, const ckks_diags* const* f,
                          const lt_algo* algos, const lt_split* splits, ckks_ct* out, void* stream,
                          lt_split* chosen);

/* A recorded batch.  lt_graph_create runs lt_eval_batch once with these
 * arguments (which also sets up every table the batch needs), then records
 * the same work into a CUDA graph; lt_graph_launch replays it on `stream`,
 * recomputing every output from the current contents of the inputs, with no
 * host-side work.  The ciphertexts, diagonals and keys named at creation must
 * stay alive and keep their buffers while the graph exists; the graph owns
 * its scratch memory.  Replays of one graph must not overlap in time. */
typedef struct lt_graph lt_graph;
ckks_status lt_graph_create(ckks_ctx* ctx, uint32_t count, const ckks_ct* const* in, const ckks_diags* const* f,
                            const lt_algo* algos, const lt_split* splits, ckks_ct* const* out, lt_graph** graph);
ckks_status lt_graph_launch(lt_graph* graph, void* stream);
/* Recording of any sequence of LT calls (a chain, several batches, single
 * LTs).  lt_graph_begin starts capturing `stream` (a created stream, not the
 * legacy default stream; thread-local capture mode); the lt_eval,
 * lt_eval_batch and lt_eval_chain calls this thread then queues on `stream`
 * are recorded instead of run, and lt_graph_end returns them as one graph
 * for lt_graph_launch.  Every recorded call must have run once before with
 * the same shapes: first use sets up per-level tables with synchronous copies
 * that a recording cannot hold, and such a call fails (CKKS_ECUDA) and leaves
 * the recording invalid, so that lt_graph_end fails too.  lt_graph_end always
 * ends the capture.  The capture is thread-local: while a thread records, it
 * may not queue LT calls on other streams (CUDA forbids the stream-ordered
 * allocations they make); other threads may, and a batch forked over lanes
 * uses lanes of its own caller stream, never those of the recorded stream.
 * The same lifetime rules as for lt_graph_create apply. */
ckks_status lt_graph_begin(ckks_ctx* ctx, void* stream);
ckks_status lt_graph_end(ckks_ctx* ctx, void* stream, lt_graph** graph);
ckks_status lt_graph_destroy(lt_graph* graph);

/* Rotation amounts (mod N/2, ascending, multiples of stride) whose keys the
 * algorithm needs for n_diag diagonals and this split; returns how many were
 * written (at most cap), or -1 on a bad split. */
int32_t lt_required_rotations(const ckks_ctx* ctx, lt_algo algo, const lt_split* split,
                              uint32_t n_diag, int32_t offset0, int32_t stride, int32_t* rot_out,
                              uint32_t cap);

/* The cost model's ranking of the admissible splits for (algo, level,
 * n_diag), fastest first; writes at most cap and returns how many. */
int32_t lt_candidate_splits(const ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag, lt_split* out,
                            uint32_t cap);

/* The cost model that ranks the splits (the key-memory / compute trade-off
 * of Sec. III) for one LT: hbm_bytes = the DRAM bytes it counts (diagonals,
 * distinct keys, input and output, and each Decompose's digits written and
 * read once; -1 for BSGS, whose model counts them differently) and seconds =
 * its time estimate (bytes over a fitted bandwidth plus the NTT butterflies
 * and the multiply-accumulates over fitted kernel rates).  DH-BSGS is
 * modelled in the schedule the model prefers (see lt_dh_schedule).  EINVAL
 * on a bad level or split. */
ckks_status lt_model_estimate(const ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag,
                              const lt_split* split, double* hbm_bytes, double* seconds);

/* Measuring autotuner (split selection per shape): ranks every admissible
 * split of f's n_diag for `algo` with the library's cost model, keeps the
 * first max_candidates whose rotation keys are all uploaded, times each on
 * `sample` (its level and f's stride define the shape), and records the
 * fastest for that (algo, level, n_diag, stride, offset0); lt_eval and lt_eval_batch
 * then use it whenever no split is given.  Synchronous; allocates one scratch
 * ciphertext.  ENOKEY if no candidate has all of its keys. */
ckks_status lt_autotune(ckks_ctx* ctx, lt_algo algo, const ckks_ct* sample, const ckks_diags* f,
                        uint32_t max_candidates, lt_split* chosen, double* best_ms);

/* Measuring autotuner for batches: the same candidates as lt_autotune, each
 * timed as one lt_eval_batch over the `count` sample ciphertexts (one level,
 * all multiplied by f) on a private stream, so that the choice reflects what a
 * batch shares -- every key and diagonal word is read once for the group, which
 * moves the cost from HBM towards the middle layer's multiply-accumulates.
 * Returns the fastest split and its time per batch; records nothing (the
 * single-LT choice for the shape is unchanged).  Synchronous; allocates
 * `count` output ciphertexts for its own use.  EINVAL if the samples are not
 * all at one level, ENOKEY if no candidate has all of its keys. */
ckks_status lt_autotune_batch(ckks_ctx* ctx, lt_algo algo, uint32_t count, const ckks_ct* const* samples,
                              const ckks_diags* f, uint32_t max_candidates, lt_split* chosen, double* best_ms);

/* The tile lt_autotune measured for the shape (algo, f, level) besides its
 * split: outer rotation indices per CTA of the diagonal multiply-accumulate
 * kernel (Alg. 2 lines 8-14) and positions per CTA, each 0 for the default
 * (outer: the next power of two >= n'3, at most 8; positions: 128, four
 * CTAs per SM, or two with 8 outer indices).  lt_autotune times the default,
 * half the outer indices, and 256 positions for its chosen split, and
 * lt_eval uses the fastest whenever it runs that split for that shape;
 * results do not depend on the tile.  Returns 1 and writes the tile, 0 if
 * the shape was not tuned, -1 on a null argument. */
int32_t lt_tuned_tile(const ckks_ctx* ctx, lt_algo algo, const ckks_diags* f, uint32_t level, uint32_t* outer_per_cta,
                      uint32_t* positions_per_cta);

/* Which schedule DH-BSGS (Algorithm 1) with `split` = (n1, n2) runs with on
 * f at `level`: 0 = the baby steps materialised by key switching, then the
 * diagonal products and the giant steps (Algorithm 1 as printed); 1 = the
 * baby steps computed inside the diagonal multiply-accumulate kernel, the
 * schedule TH-BSGS(1, n1, n2) of Algorithm 2 runs.  Both give identical
 * residues.  The choice is lt_autotune's measurement for that shape and split
 * (lt_autotune times DH candidates in both), else the cost model's.  -1 on a
 * bad argument. */
int32_t lt_dh_schedule(const ckks_ctx* ctx, const ckks_diags* f, uint32_t level, const lt_split* split);

/* The split the library would choose for (algo, level, n_diag) with stride 1:
 * the autotuned one if lt_autotune has measured that shape, else the model's. */
ckks_status lt_choose_split(ckks_ctx* ctx, lt_algo algo, uint32_t level, uint32_t n_diag, lt_split* out);

/* ------------------------------------------------------------------ steps
 * The steps of the key-switching path (Fig. 1), each on caller-owned device
 * buffers, asynchronous on `stream`.  They are what lt_eval is built from
 * and are exported for step-by-step checking and custom schedules. */

/* Forward (inverse = 0) or inverse (inverse = 1) negacyclic NTT, in place, of
 * a polynomial at `level` with (ext = 1) or without (ext = 0) the P limbs.
 * Words must be canonical residues (limb j in [0, q_j)); so are the results. */
ckks_status ckks_poly_ntt(ckks_ctx* ctx, uint64_t* poly, uint32_t level, int ext, int inverse, void* stream);

/* Decompose (ModUp), Fig. 1 and Eq. (3): digits of phi_rot(c) (rot = 0: of c)
 * over the extended basis.  c: [level][N]; digits: [beta_level][level+k][N]. */
ckks_status ckks_decompose(ckks_ctx* ctx, uint32_t level, const uint64_t* c, int32_t rot,
                           uint64_t* digits, void* stream);

/* Switching-key inner product with hoisted automorphism (Alg. 2 lines 4-5):
 *   out0 = phi_rot(x0 + <d, swk~_0>),  out1 = phi_rot(<d, swk~_1>)
 * with swk~ = phi_{-rot}(swk_key_rot), evaluated as phi_rot(x0) + <phi_rot(d), swk>.
 * digits [beta_level][level+k][N]; x0 NULL (zero), an extended polynomial
 * [level+k][N] (lift_x0 = 0) or a Q-only polynomial [level][N] lifted to
 * P*x0 (lift_x0 = 1, Alg. 2 line 2).  accumulate = 1 adds the result to
 * out0/out1 instead of overwriting them (Alg. 2 lines 17-18). */
ckks_status ckks_ks_inner(ckks_ctx* ctx, uint32_t level, const uint64_t* digits, int32_t key_rot,
                          int32_t rot, const uint64_t* x0, int lift_x0, uint64_t* out0, uint64_t* out1,
                          int accumulate, void* stream);

/* ModDown, Eq. (4): x [level+k][N] -> out [level][N]. */
ckks_status ckks_moddown(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream);

/* ModDown merged with rescale (Alg. 2 line 19): x [level+k][N] ->
 * out [level-1][N], dividing by P * q_{level-1} (Eq. 4 over the basis
 * {q_{level-1}, p_0..p_{k-1}}). */
ckks_status ckks_moddown_rescale(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out,
                                 void* stream);

/* ModDown exactly as ckks_moddown, for host programs that cannot let the
 * library allocate device memory while it runs: an application that owns
 * every byte of the GPU through its own allocator or memory budget (a
 * library-side cudaMalloc would take memory outside that budget), or a
 * latency-bound path where a cudaMalloc and the device synchronisation it
 * may imply are not acceptable.  The caller passes x and out.
 * The paper has no counterpart: this is a deployment variant.  Its scratch is
 * a fixed device array inside the library of 8 limbs at N = 2^16 (4 MiB,
 * k * N <= 524288 words); every GPU that loads the library holds it until
 * the process exits.  Larger k * N, level > 64 or k > 8 fail with
 * CKKS_EINVAL, and so does a level whose constant tables do not exist yet
 * (any earlier call at that level on this context creates them).  The call
 * allocates nothing: its first call on a device looks up the array's device
 * address once (make that first call before any stream capture).  All calls
 * share the one array, so calls whose work overlaps on the GPU (other
 * streams, other contexts on the same device) race; serialise them.  The
 * scratch is fully rewritten before it is read, so leftover contents from
 * an earlier call do not matter. */
ckks_status ckks_moddown_noalloc(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream);

/* Rescale, Eq. (1): x [level][N] -> out [level-1][N]. */
ckks_status ckks_rescale(ckks_ctx* ctx, uint32_t level, const uint64_t* x, uint64_t* out, void* stream);

/* Automorphism phi_rot in the NTT domain (Eq. 7) of n_limbs limbs that hold
 * any moduli (a pure index gather): out[s] = in[src(s)]. */
ckks_status ckks_automorphism(ckks_ctx* ctx, uint32_t n_limbs, const uint64_t* in, int32_t rot,
                              uint64_t* out, void* stream);

/* ------------------------------------------------------------------ misc */

/* Waits for the context's device and reports whether any device-side wait
 * gave up since the last check (CKKS_ETIMEOUT; the flag is then cleared and
 * the results computed since the last check must be discarded).  Kernels
 * that stage operands through asynchronous copies bound every wait on them
 * (about one second) instead of spinning forever.  ckks_ct_download performs
 * the same check. */
ckks_status ckks_device_status(ckks_ctx* ctx);

/* Failure-detection self-test: queues one kernel that waits, with the same
 * bounded wait, on a device barrier that nothing completes, for limit_ms
 * (1..5000) milliseconds.  The next ckks_device_status then reports
 * CKKS_ETIMEOUT and the context stays usable.  Faults nothing. */
ckks_status ckks_selftest_bounded_wait(ckks_ctx* ctx, uint32_t limit_ms, void* stream);

/* Failure-detection test hook of the TMA-staged diagonal multiply-accumulate
 * kernel (Alg. 2 lines 8-14; the bounded waits have no counterpart in the
 * paper).  From the next LT call on, that kernel's per-step waits give up
 * after wait_limit_ns (0 = the default of about one second; at most 5 s),
 * and its step starve_step is never issued, so that the wait on that
 * step's barrier runs out in every CTA (0xFFFFFFFF = no step is starved).
 * A CTA whose wait gives up stops, waits with the default limit for the
 * copies it has in flight, and raises the context's device flag: the next
 * ckks_device_status reports CKKS_ETIMEOUT and the results are garbage.
 * Faults nothing.  Reset with (0, 0xFFFFFFFF).  Not for production use; it
 * changes the context like an upload (no evaluation call may overlap it). */
ckks_status ckks_debug_diag_mac_waits(ckks_ctx* ctx, uint64_t wait_limit_ns, uint32_t starve_step);

/* Test hook: every later LT on the context runs the diagonal kernel with this
 * tile (see lt_tuned_tile; outer_per_cta 0 or a power of two up to 8, at
 * most the default; positions_per_cta 0, 128, 256 or 512), instead of the tuned or
 * default one; (0, 0) restores the normal choice.  Results do not depend on
 * the tile, which is what the test checks.  It changes the context like an
 * upload (no evaluation call may overlap it). */
ckks_status ckks_debug_diag_mac_tile(ckks_ctx* ctx, uint32_t outer_per_cta, uint32_t positions_per_cta);

const char* ckks_last_error(void);
size_t ckks_device_bytes_in_use(const ckks_ctx* ctx);
/* Number of CUDA kernels this library has launched in this process. */
uint64_t ckks_kernel_launch_count(void);

/* Live per-kernel timing.  Kernel classes: "diag_mac" (plaintext-diagonal
 * multiply-accumulate with the fused middle key-switch layer), "ks_inner"
 * (switching-key inner product), "ntt_fwd_cols", "ntt_fwd_rows",
 * "ntt_inv_rows", "ntt_inv_cols" (the two passes of the forward and inverse
 * NTT), "automorphism", "add_gather".  While a class is enabled every launch
 * of it is bracketed by CUDA events on its own stream.  ckks_profile_read
 * waits for the recorded events and returns the summed device time (ms) and
 * the number of launches since the last reset.  EINVAL on an unknown name. */
ckks_status ckks_profile_enable(const char* kernel_class, int on);
ckks_status ckks_profile_read(const char* kernel_class, double* total_ms, uint64_t* launches);
void ckks_profile_reset(void);

/* Algorithmic integer work of the launches that ckks_profile_read times
 * (same classes, same enable and reset), for the integer-ALU roofline:
 * `macs` counts 128-bit multiply-accumulates of a residue by a residue
 * ("diag_mac": two per diagonal product plus 2 beta per middle-layer step,
 * Alg. 2 lines 8-14; "ks_inner": 2 beta per output word, the key inner
 * product of Sec. II-A; "ntt_fwd_cols": the basis conversion of Eq. 3 fused
 * into it, one per source limb and output word), `butterflies` counts NTT
 * butterflies (N/2 per stage and limb, the stages of the pass).  EINVAL on
 * an unknown name or a null output. */
ckks_status ckks_profile_work(const char* kernel_class, double* macs, double* butterflies);

/* Integer-rate probe, the denominator of that roofline: register-only loops
 * of the library's own 128-bit multiply-accumulate and of its forward NTT
 * butterfly (the growing Cooley-Tukey form of Sec. II-A's transform) on every
 * SM of `device`, 8 CTAs of 256 threads per SM, best of two timed runs after
 * a warm-up.  Returns multiply-accumulates and butterflies per second.
 * Synchronous; allocates and frees a few KB of device memory and a stream of
 * its own, so it must not be called while a stream of the device is being
 * captured.  ECUDA on a CUDA error, EINVAL on a null output. */
ckks_status ckks_probe_int_rates(int device, double* macs_per_s, double* butterflies_per_s);

#ifdef __cplusplus
}
#endif
#endif /* CKKS_LT_H */
