/*
 * corutv.h -- C ABI of libcorutv, a single-GPU (sm_103a) implementation of
 * Compressed Randomized UTV (CoR-UTV) with the power method and of the
 * ALM-CoRUTV robust-PCA solver (Kaloorazi & de Lamare, "Study of Compressed
 * Randomized UTV Decompositions for Low-Rank Matrix Approximations in Data
 * Science").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are row-major; `ld*` is the row stride in elements (>= columns).
 *  - A pointer argument may be host or device memory; the library asks the
 *    CUDA runtime which. All pointers of one call must be in the same space,
 *    except `opts->psi`, which may be either.
 *  - Device-pointer calls are stream-ordered on the context's stream
 *    (corutv_set_stream) and return once enqueued; corutv_sync waits and
 *    reports any status raised on the device. Host-pointer calls copy in,
 *    compute, copy out and synchronise before returning.
 *  - Inputs are borrowed and never written. Outputs are caller-owned. The
 *    context owns its workspace and streams.
 *  - Errors are reported only through the returned status; nothing aborts or
 *    exits. corutv_last_error gives a one-line message for the calling thread.
 *  - ell = k + p must satisfy 1 <= k <= ell < min(m, n) (Sec. 3.1: "an
 *    integer k <= ell < min{m, n}"), and ell <= 128 for the tensor-core
 *    sketch precisions (BF16, TF32), ell <= 320 for FP64 and FP32 sketches;
 *    q >= 0.
 *  - Every step of every call runs in this library's CUDA kernels; there is
 *    no CPU fallback. Without a usable GPU, corutv_create returns CORUTV_ECUDA.
 */
#ifndef CORUTV_H
#define CORUTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CORUTV_OK = 0,
    CORUTV_EINVAL = 1,      /* bad argument or unsupported combination */
    CORUTV_ENOMEM = 2,      /* device memory or the context's budget exhausted */
    CORUTV_ECUDA = 3,       /* a CUDA runtime / driver call failed */
    CORUTV_EPENDING = 4,    /* corutv_poll: the request has not finished */
    CORUTV_ETIMEDOUT = 5,   /* corutv_poll: timeout elapsed; or a device wait gave up */
    CORUTV_ENOTCONV = 6,    /* corutv_rpca: max_iter reached with zeta >= tol */
    CORUTV_EBREAKDOWN = 7   /* Cholesky of a sketch Gram failed even after the shift */
} corutv_status;

/* Element type of A / M and of every floating-point output of the call. */
typedef enum { CORUTV_F64 = 0, CORUTV_F32 = 1 } corutv_dtype;

/* Arithmetic of the 2q+2 sketch / power products A X and A^T Y.
 * F64: FP64 FMA. F32: FP32 FMA. TF32 / BF16: tensor cores (tcgen05) with FP32
 * accumulation; BF16 first writes a bf16 copy of A. The projection D of
 * eq. 7 always has FP32 accuracy (dtype F32) or runs in FP64 (dtype F64);
 * with BF16 sketches and FP32 input it runs on the tensor cores with
 * exact three-way bf16 splits of A and Q2 (see BF16X3). The Gram Cholesky
 * factorisations and the pivoted QR of D always run in FP64.
 * BF16X3 (corutv_sketch only, FP32 A, trans = 0): A X from the exact splits
 * A = A_h + A_m + A_l, X = X_h + X_m + X_l into bf16 parts, all nine part
 * products on the tensor cores with FP32 accumulation -- the rounding of an
 * FP32 dot product at the memory traffic of 1.5 FP32 passes. */
typedef enum { CORUTV_P_F64 = 0, CORUTV_P_F32 = 1, CORUTV_P_TF32 = 2, CORUTV_P_BF16 = 3,
               CORUTV_P_BF16X3 = 4 } corutv_prec;

typedef struct {
    int64_t k;            /* target rank */
    int64_t p;            /* oversampling; ell = k + p */
    int64_t q;            /* power iterations (Algorithm 1 runs its loop q+1 times) */
    int32_t sketch_prec;  /* corutv_prec */
    int32_t d_mode;       /* 0: D = Q1^T A Q2 (eq. 7), a third pass over A (FP32-accurate on
                             the mixed paths); 1: the single-pass core of Sec. 3.1,
                             D_approx = Q1^T C1 (Q2^T X)^+ with X the matrix the last C1 was
                             formed from, which with C2 = A^T Q1 = Q2 R2 equals R2^T: formed
                             from the factors of the final thin QR, no third pass (on the
                             mixed paths D then carries the sketch products' rounding);
                             other values -> CORUTV_EINVAL */
    uint64_t seed;        /* Philox-4x32-10 key for Psi when psi == NULL */
    uint32_t stream;      /* Philox counter word 2 (independent draws per call) */
    uint32_t t_lower;     /* 0: T upper triangular (Algorithm 1 on A, any shape); 1: T lower
                             triangular, the variant Sec. 3 gives for m < n: Algorithm 1 on
                             A^T, whose A^T ~ U' T' V'^T is returned as U = V' (its Q2 P: perm
                             permutes the columns of U), T = T'^T, V = U' (any shape);
                             other values -> CORUTV_EINVAL */
    const double* psi;    /* optional row-major FP64 Gaussian test matrix: n x ell, or
                             m x ell when t_lower = 1 */
    uint32_t power_form;  /* 0: every sketch is re-orthonormalised before its next use (C1 -> Q1,
                             C2 -> X); 1: one thin QR per power round, X = qr(A^T (A X)) -- the
                             power step of Algorithm 1 with C1 used as it is, the form the
                             paper's loop has between A and A^T (Sec. 3.2); in exact arithmetic
                             the same Q1, Q2. Loses the weak directions of C1 to rounding when
                             C1 is an operand of reduced precision (BF16 sketches). Other values
                             -> CORUTV_EINVAL */
    uint32_t bf16_last_round; /* BF16 sketches of FP32 input with d_mode 0: 0 (default) every
                             round multiplies by A_h = bf16(A); 1: the two products of the last
                             power round multiply by A_h + A_m, the first two exact bf16 parts of
                             A (16 significant bits; two more bf16 reads of A). Ignored otherwise;
                             other values -> CORUTV_EINVAL */
} corutv_opts;

typedef struct corutv_ctx corutv_ctx;

/* Create a context on CUDA device `device`. mem_budget_bytes caps the
 * device workspace the context may hold (0 = 90 % of the free memory at
 * creation). max_slots caps how many serving requests are resident at once
 * (<= 0 selects 8). */
corutv_status corutv_create(corutv_ctx** out, int device, size_t mem_budget_bytes, int max_slots);

/* Waits for outstanding work, frees all device memory of the context. */
corutv_status corutv_destroy(corutv_ctx* ctx);

/* Message of the last failing call made by this thread; never NULL. */
const char* corutv_last_error(const corutv_ctx* ctx);

/* Use `cuda_stream` (a cudaStream_t, may be NULL for the legacy stream) for
 * subsequent stream-ordered calls. The caller keeps the stream alive. Work
 * enqueued afterwards waits (on the device, through an event) for the work
 * already queued on the previous stream, since every call of the context
 * shares its workspace: alternating streams never lets two calls overlap. */
corutv_status corutv_set_stream(corutv_ctx* ctx, void* cuda_stream);

/* Wait for all work enqueued on the context's stream; returns the first
 * device-side status raised since the previous corutv_sync
 * (CORUTV_EBREAKDOWN, CORUTV_ETIMEDOUT) or a CUDA error. */
corutv_status corutv_sync(corutv_ctx* ctx);

/* CoR-UTV with power method (Algorithm 1; eqs. 4-9):
 *   Psi (n x ell, Gaussian) -> for i = 0..q: C1 = A X, Q1 = qr(C1),
 *   C2 = A^T Q1, X = qr(C2) (i < q) -> Q2 = qr(C2) -> D = Q1^T A Q2 ->
 *   D P = Qt Rt (column-pivoted QR) -> U = Q1 Qt, T = Rt, V = Q2 P.
 *   With opts->t_lower = 1 the same steps run on A^T (the lower-T variant of
 *   Sec. 3 for m < n): U = Q2 P, T = Rt^T, V = Q1 Qt of that run.
 * Each sketch is re-orthonormalised before its next use (CholeskyQR2); in
 * exact arithmetic this gives the same Q1, Q2 as the printed loop.
 * A: m x n (lda). U: m x ell (ldu), T: ell x ell upper triangular (row
 * stride ell, strictly lower part written as 0, diag >= 0 and
 * non-increasing), V: n x ell (ldv), perm: ell int32, the 0-based column of
 * D placed at position j. U, V, perm may be NULL; T may not. */
corutv_status corutv_factor(corutv_ctx* ctx, corutv_dtype dtype, const void* A, int64_t m, int64_t n,
                            int64_t lda, const corutv_opts* opts, void* U, int64_t ldu, void* T,
                            void* V, int64_t ldv, int32_t* perm);

/* Row-partitioned CoR-UTV: the form of Algorithm 1 for a matrix whose rows are
 * spread over several processes (GPUs), A = [A_1; A_2; ...], each rank holding
 * A_i (m_local x n, lda) on its own device. Every pass over A is local; the
 * only exchanges are the sums that reduce over A's rows, which the library
 * hands to the caller's `allreduce`:
 *   - the ell x ell Gram matrix of each thin QR of C1 = A X (eq. 4; C1 stays
 *     row-distributed, Q1_i = C1_i R^-1), FP64;
 *   - C2 = sum_i A_i^T Q1_i (eq. 5; n x ell, then replicated), in the panel
 *     arithmetic (FP32 with FP32 data and F32/TF32/BF16 sketches, else FP64);
 *   - D = sum_i Q1_i^T (A_i Q2) (eq. 7; ell x ell), FP64.
 * Everything else (Psi, the thin QRs of C2, the pivoted QR of D, T, V) is
 * computed identically on every rank. Per factorisation the exchanged volume
 * is (q+1) n ell + (2q+3) ell^2 values (one Gram per CholeskyQR pass), against
 * (2q+3) m_local n elements of A read locally.
 * allreduce(buf, count, dtype, user) must replace the `count` values of
 * `dtype` at `buf` (pinned host memory owned by the library) by their sum over
 * all ranks, in the same order on every rank, and return CORUTV_OK; the
 * library calls it synchronously (the device work producing buf has finished)
 * and the same number of times on every rank.
 * m_total = sum of the ranks' m_local; each rank needs m_local > ell. U:
 * this rank's rows of U (m_local x ell, ldu); T, V, perm as in corutv_factor,
 * identical on all ranks. opts->seed / stream must agree across ranks (Psi is
 * drawn, not passed); d_mode, t_lower and power_form must be 0.
 * Device pointers only; returns once enqueued (corutv_sync waits). */
typedef corutv_status (*corutv_allreduce_fn)(void* buf, int64_t count, corutv_dtype dtype, void* user);
corutv_status corutv_factor_rows(corutv_ctx* ctx, corutv_dtype dtype, const void* A, int64_t m_local, int64_t n,
                                 int64_t lda, int64_t m_total, const corutv_opts* opts, corutv_allreduce_fn allreduce,
                                 void* user, void* U, int64_t ldu, void* T, void* V, int64_t ldv, int32_t* perm);

/* ALM-CoRUTV (Algorithm 2; eq. 13): M = L + S by inexact augmented
 * Lagrange multipliers with the CoR-UTV thresholding operator
 * C_delta(B) = U(:,1:r) T(1:r,:) V^T, r = #{i : T_ii > delta}, and the
 * shrinkage S_delta(x) = sgn(x) max(|x| - delta, 0) (Sec. 4). opts->k is the
 * rank guess, 1 <= k <= 160 and ell = 2k <= 128 for tensor-core sketches
 * (CORUTV_EINVAL otherwise); the low-rank step uses
 * ell = 2k and q = 1 (Sec. 5.3) and a fresh Psi per iteration (Philox stream
 * opts->stream + j + 1).
 * Y_0 = S_0 = 0; mu_{j+1} = min(rho mu_j, mu_bar); stop after the first
 * iteration with zeta = ||M - L - S||_F / ||M||_F < tol or after max_iter.
 * Parameters <= 0 select: lambda = 1/sqrt(max(m, n)), mu0 = 1.25/||M||_2
 * (estimated on the device by 50 power iterations), rho = 1.6,
 * mu_bar = 1e7 mu0, tol = 1e-5, max_iter = 100.
 * L, S: m x n with row stride n. iters, zeta, rank: optional outputs (host
 * pointers), valid after the call (device calls synchronise at the end).
 * Returns CORUTV_ENOTCONV if max_iter was reached with zeta >= tol. */
corutv_status corutv_rpca(corutv_ctx* ctx, corutv_dtype dtype, const void* M, int64_t m, int64_t n,
                          int64_t ldm, const corutv_opts* opts, double lambda, double mu0,
                          double mu_bar, double rho, double tol, int max_iter, void* L, void* S,
                          int* iters, double* zeta, int* rank);

/* ---- serving: asynchronous factorisations with continuous admission ---- */
typedef struct {
    corutv_dtype dtype;
    const void* A;
    int64_t m, n, lda;
    corutv_opts opts;
    void *U, *T, *V;
    int64_t ldu, ldv;
    int32_t* perm;
} corutv_request;

/* Queue one corutv_factor request; the descriptor is copied, the buffers
 * are borrowed until corutv_poll returns something other than
 * CORUTV_EPENDING. Requests are admitted in arrival order as slots and
 * workspace memory free up, and run concurrently on the device; the memory
 * idle slots and idle batch lanes hold is given back when the request at the
 * head would not fit beside it. Returns CORUTV_ENOMEM only if the request
 * could never fit the budget.
 * Device inputs: submit records an event on the context's stream
 * (corutv_set_stream) and the request's work waits for it, so A and psi may
 * still be in production on that stream when the caller submits (no host
 * synchronisation needed). Host inputs must be complete at submit. */
corutv_status corutv_submit(corutv_ctx* ctx, const corutv_request* req, uint64_t* ticket);

/* Continuous batching of the serving stream. With max_batch > 0, queued
 * requests that the grouped path takes (device FP32 A, BF16 sketches,
 * d_mode / t_lower / power_form / bf16_last_round 0, psi NULL, ell <= 128:
 * see corutv_factor_batch) are admitted as batches instead of one per slot:
 * whenever one of two batch lanes is free, it takes the batchable requests at
 * the head of the queue (arrival order, up to max_batch, as many as the
 * memory budget allows) and runs them with grouped launches, while requests
 * that arrive meanwhile queue for the other lane. Each result is bitwise the
 * one the same request gives alone through corutv_factor_batch. A batch's
 * device status words are shared: a breakdown or timeout in one problem is
 * reported for every request of its batch. Other requests keep the slots.
 * max_batch = 0 (the default) returns to one request per slot; 0 .. 4096. */
corutv_status corutv_set_batching(corutv_ctx* ctx, int max_batch);

/* Wait up to timeout_us (0 = do not wait, < 0 = forever) for a ticket.
 * CORUTV_EPENDING / CORUTV_ETIMEDOUT while unfinished; otherwise the
 * request's own status, with latency_s (optional) = completion - submit. */
corutv_status corutv_poll(corutv_ctx* ctx, uint64_t ticket, int64_t timeout_us, double* latency_s);

/* ---- batched factorisation: grouped launches over uneven shapes ----------
 * Algorithm 1 (eqs. 4-9) for `count` requests (1 .. 4096) of different m, n,
 * k, p, q at once, every step of the method one kernel launch over all of
 * them: the sketch, power and projection products as one grouped tcgen05
 * launch (each problem its own stream-K tiles, panel width and tensor map),
 * the Grams, FP64 Choleskys, triangular solves, pivoted QRs of D and the
 * assembly of U, T, V each as one launch with a block range per problem.
 * Power rounds are aligned at the end (a problem with q < max q joins the
 * later rounds), so a round's launches cover the problems still iterating.
 * Requests: FP32 A and device pointers only (A, T required; U, V, perm
 * optional, FP32 outputs as in corutv_factor); opts.sketch_prec BF16 with
 * the FP32-accurate split projection; d_mode, t_lower, power_form and
 * bf16_last_round 0; psi NULL (Psi from seed and stream); ell = k + p <= 128.
 * The arithmetic of each step is that of corutv_factor's BF16 path; each
 * problem's launch shapes (stream-K grid, Gram split) depend on its own sizes
 * only, so a problem's results are bitwise the same alone and in any batch
 * (they differ from a corutv_factor call in the order of FP32 partial sums
 * and in forming U from the QRCP's reflectors). Stream-ordered on the
 * context's stream; returns once the work is enqueued (corutv_sync gives the
 * device status). The batch's buffers are held by the context until the next
 * batch call or corutv_destroy. */
corutv_status corutv_factor_batch(corutv_ctx* ctx, const corutv_request* reqs, int count);

/* ---- per-stage device timers and launch counter --------------------------
 * Not part of the method: instrumentation for roofline measurements. With
 * profiling enabled, corutv_factor / corutv_rpca record a CUDA event pair on
 * the context's stream around every kernel of a stage:
 *   CORUTV_STAGE_SKETCH  the 2q+2 sketch / power products (eqs. 4, 5)
 *   CORUTV_STAGE_PROJECT the product W = A Q2 of the projection (eq. 7)
 *   CORUTV_STAGE_ORTH    each thin QR (CholeskyQR2), all of its kernels
 *   CORUTV_STAGE_QRCP    the pivoted QR of D (eq. 8)
 *   CORUTV_STAGE_FACTOR  one whole factorisation (Algorithm 1)
 * corutv_profile_read synchronises the stream and returns the summed
 * duration (ms) and the number of timed intervals of `stage`, and, for
 * CORUTV_STAGE_ALL, the number of kernels this library launched (in any
 * context) since profiling was last enabled. Enabling resets all counters. */
enum { CORUTV_STAGE_SKETCH = 0, CORUTV_STAGE_PROJECT = 1, CORUTV_STAGE_ORTH = 2, CORUTV_STAGE_QRCP = 3,
       CORUTV_STAGE_FACTOR = 4, CORUTV_STAGE_COUNT = 5, CORUTV_STAGE_ALL = -1 };
corutv_status corutv_profile_enable(corutv_ctx* ctx, int enable);

/* CUDA-graph replay of repeated factorisations (not part of the method).
 * With enable = 1, a corutv_factor call on device pointers whose arguments
 * (dtype, A, m, n, lda, every option, the output pointers and leading
 * dimensions) equal those of an earlier call on this context is captured,
 * on its second occurrence, into a CUDA graph of all its launches, and that
 * graph is replayed for every later occurrence: the same kernels on the same
 * buffers, one launch call instead of one per kernel. Results are bitwise
 * those of the direct calls. Up to 16 argument sets are kept; a workspace
 * growth or enable = 0 drops them. Ignored while profiling is enabled and
 * for host pointers. Returns CORUTV_EINVAL for a bad context. */
corutv_status corutv_set_graphs(corutv_ctx* ctx, int enable);

/* Autotuning of the tensor-core products' stage shape (process-wide, all
 * contexts; not part of the method). With enable = 1, the first launch of
 * each product shape (its M and K extents, K segments, operand kind, panel
 * width, direction, output handling and grid) times the candidate shapes --
 * one or two 128-byte K boxes of A per pipeline stage, each with the deepest
 * ring that fits and with half of it -- with CUDA events on the caller's
 * stream (three launches each; the call then synchronises that stream) and
 * keeps the fastest for the process; later launches of that shape use it.
 * enable = 0 (the default) returns to the fixed rule; choices made are kept.
 * Results change only in the order of FP32 partial sums. */
corutv_status corutv_set_autotune(int enable);
/* Returns the number of tuned shapes; for 0 <= index < that number, also
 * the shape (M extent, K extent, panel columns, 1 for A^T Y) and its choice
 * (K boxes per stage, stages, best launch time in microseconds). */
int corutv_autotune_entry(int index, int64_t* mtot, int64_t* ktot, int* nb, int* trans, int* kgroup, int* stages,
                          float* us);
corutv_status corutv_profile_read(corutv_ctx* ctx, int stage, double* total_ms, int64_t* count);

/* ---- single steps of Algorithm 1, for testing and composition ----------
 * Device pointers only, stream-ordered on the context's stream. */

/* Step 1: psi[i*ldpsi + j] = N(0,1) draw for entry (i, j) of the n x ell
 * test matrix: Philox-4x32-10 with counter (i, j, stream, 0) and key
 * (seed_lo, seed_hi); the four words give two 53-bit uniforms
 * u1 in (0,1], u2 in [0,1); z = sqrt(-2 ln u1) cos(2 pi u2). FP64 output. */
corutv_status corutv_gaussian(corutv_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t ell,
                              double* psi, int64_t ldpsi);

/* Eq. 4 / eq. 5 / the first half of eq. 7: C = A X (trans = 0, X n x ell,
 * C m x ell) or C = A^T X (trans = 1, X m x ell, C n x ell) in arithmetic
 * `prec`. A has element type dtype; X and C are FP64. */
corutv_status corutv_sketch(corutv_ctx* ctx, corutv_dtype dtype, corutv_prec prec, int trans,
                            const void* A, int64_t m, int64_t n, int64_t lda, const double* X,
                            int64_t ldx, int64_t ell, double* C, int64_t ldc);

/* Sec. 3.1 "C = Q R": thin QR of the rows x ell FP64 matrix C (rows >= ell)
 * by CholeskyQR2 (Gram in FP64, Cholesky in FP64, shifted once if the
 * first Gram is not numerically positive definite). Q: rows x ell (ldq),
 * R: ell x ell upper (optional), diag(R) > 0. 1 <= ell <= 320 (beyond 128
 * the Cholesky runs in global memory and the triangular solve as R^-1 and a
 * product). */
corutv_status corutv_orth(corutv_ctx* ctx, const double* C, int64_t rows, int64_t ell, int64_t ldc,
                          double* Q, int64_t ldq, double* R);

/* Failure detection of the device waits (not part of the method): enqueue on
 * the context's stream a kernel that holds tensor memory while it waits on an
 * mbarrier nothing arrives on, gives up after about limit_ns (0 .. 1e10),
 * raises the device timeout status, frees the tensor memory and returns --
 * the bounded-wait path every tcgen05 kernel of the library takes. The next
 * corutv_sync returns CORUTV_ETIMEDOUT; the context stays usable. */
corutv_status corutv_selftest_wait(corutv_ctx* ctx, int64_t limit_ns);

/* Eq. 8: D P = Qt Rt for the ell x ell FP64 matrix D (row stride ell), one
 * thread block, FP64, Businger-Golub pivoting on recomputed column norms
 * (lowest index on ties), diag(Rt) >= 0. Qt, Rt: ell x ell, 1 <= ell <= 320:
 * up to 128 in shared memory, where norms within 2^-45 relative of each other
 * count as ties; beyond, in global memory with an exact comparison. */
corutv_status corutv_qrcp(corutv_ctx* ctx, const double* D, int64_t ell, double* Qt, double* Rt,
                          int32_t* perm);

/* ---- allocation-free thin QR --------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: a host framework that owns all device
 * memory through its own pool, a real-time or certified process that forbids
 * allocation after start-up, or a plug-in running inside another library's
 * step. It computes exactly what corutv_orth computes (CholeskyQR2 with the
 * shifted fallback pass) but takes no context, allocates nothing and keeps
 * every temporary in one fixed 16 MiB device array owned by the library
 * (every GPU that loads the library holds it until the process exits).
 *   C: rows x ell (ldc), Q: rows x ell (ldq), R: ell x ell upper (optional),
 *   info: optional device int, set to 1 if the Cholesky broke down even
 *   after the shift, else 0; all device pointers; cuda_stream: the
 *   cudaStream_t to enqueue on (NULL = legacy stream). Stream-ordered: it
 *   returns once the work is enqueued.
 * Limits: 1 <= ell <= 128, rows >= ell and round_up(rows, 64) * ell <= 524288
 *   (e.g. 4096 x 128); larger problems return CORUTV_EINVAL before any work.
 * The first call on each device looks up the fixed array's device address
 *   (with that device current) and caches it; make that first call before
 *   any stream capture. All calls share the array: calls that overlap on the
 *   GPU race and corrupt each other's results, so order them on one stream.
 * Errors: status only; corutv_last_error(NULL) gives the message. */
corutv_status corutv_orth_noalloc(const double* C, int64_t rows, int64_t ell, int64_t ldc, double* Q,
                                  int64_t ldq, double* R, int* info, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CORUTV_H */
