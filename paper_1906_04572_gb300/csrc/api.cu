// C ABI of libcorutv (include/corutv.h): context, workspace, the CoR-UTV
// pipeline of Algorithm 1, the ALM-CoRUTV loop of Algorithm 2 and the
// serving queue. Host code only orchestrates; every arithmetic step runs in
// the kernels of k_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/corutv.h"
#include "internal.cuh"
#include "tc.cuh"

using namespace corutv;

namespace {
std::atomic<long long> g_launches{0};
// while this thread captures a CUDA graph, its launches are counted here (they
// run when the graph is launched, and are counted then)
thread_local long long* t_capture_count = nullptr;
}  // namespace

void corutv::count_launch() {
    if (t_capture_count) ++*t_capture_count;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}

namespace {

// Per-stage CUDA event timers of one context (see corutv_profile_enable).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> open;
    double ms[CORUTV_STAGE_COUNT] = {0};
    long long count[CORUTV_STAGE_COUNT] = {0};
    long long launch_base = 0;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    int begin(int stage, cudaStream_t st) {
        if (!on) return -1;
        cudaEvent_t a = get(), b = get();
        cudaEventRecord(a, st);
        open.push_back({stage, {a, b}});
        return (int)open.size() - 1;
    }
    void end(int token, cudaStream_t st) {
        if (token < 0) return;
        cudaEventRecord(open[token].second.second, st);
    }
    // requires the stream to have been synchronised
    void collect() {
        for (auto& r : open) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.second.first, r.second.second) == cudaSuccess) {
                ms[r.first] += t;
                count[r.first] += 1;
            } else {
                cudaGetLastError();
            }
            pool.push_back(r.second.first);
            pool.push_back(r.second.second);
        }
        open.clear();
    }
    void reset() {
        for (int i = 0; i < CORUTV_STAGE_COUNT; ++i) {
            ms[i] = 0;
            count[i] = 0;
        }
        launch_base = g_launches.load();
    }
    ~Profiler() {
        for (auto& r : open) pool.push_back(r.second.first), pool.push_back(r.second.second);
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct ProfScope {
    Profiler* p;
    int tok;
    cudaStream_t st;
    ProfScope(Profiler* p_, int stage, cudaStream_t s) : p(p_), tok(p_ ? p_->begin(stage, s) : -1), st(s) {}
    ~ProfScope() {
        if (p) p->end(tok, st);
    }
};

thread_local std::string g_last_error = "no error";

corutv_status fail(corutv_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(CORUTV_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                  \
    } while (0)

#define CKS(expr)                          \
    do {                                   \
        corutv_status s_ = (expr);         \
        if (s_ != CORUTV_OK) return s_;    \
    } while (0)

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

void corutv::record_error(const char* msg) { g_last_error = msg; }

namespace {

// Bump allocator over one device buffer; the same code measures (base ==
// nullptr) and carves.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(int64_t count) {
        const size_t bytes = (size_t)round_up((int64_t)(count * (int64_t)sizeof(T)), 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

struct DeviceBuffer {
    void* ptr = nullptr;
    size_t cap = 0;
};

// ---------------------------------------------------------------------------
// Plan and buffers of one factorisation.
// ---------------------------------------------------------------------------
struct FactorPlan {
    // m, n (and the panel strides ldm, ldn) are those of the matrix Algorithm 1
    // runs on: A, or A^T for the lower-T variant (tr); ma, na are A's own
    // rows and columns and ldma, ldna the strides of panels with ma / na rows
    int64_t m, n, lda, k, p, q, ell, ellp, ldm, ldn;
    bool tr;
    int64_t ma, na, ldma, ldna;
    ElemType ta;
    corutv_prec prec;
    ElemType tcomp;   // element type of the B operand of the sketch products
    ElemType tdproj;  // arithmetic of the projection pass (eq. 7)
    ElemType torth;   // arithmetic of the Gram products and triangular solves of the thin QRs
    ElemType tp;      // element type of the tall-skinny panels (X, C1, Q1, C2, Q2, W)
    bool tensor;      // sketch products on tcgen05
    bool split;       // projection by exact bf16 splits on tcgen05 (BF16 / TF32 sketches, FP32 input)
    bool copy_a;      // TF32: A is not a TMA source as is (base or row stride not 16-byte aligned)
    int dmode;        // 0: D = Q1^T A Q2 (eq. 7, a third pass); 1: the single-pass core (= R2^T)
    int power_form;   // 0: every sketch re-orthonormalised; 1: one thin QR per power round (C1 used as is)
    bool x2_last;     // the last power round's products multiply by A_h + A_m (bf16 split copy)
    int64_t ldc32;    // row stride of that padded FP32 copy of A
    int sp_ax, sp_aty, gs_m, gs_n;  // SIMT split counts (sizing the partial buffers)
    int64_t part_elems;
    int num_sms;
};

struct FactorBufs {
    void *x, *c1, *q1, *c2, *q2, *w, *tmp;   // panels of type FactorPlan::tp
    double *gpart, *g, *r, *d, *qt, *rt, *upanel, *zpanel;
    double* refl;     // reflectors of the QRCP of D (V, tau, signs)
    double *racc, *racc2;  // products of CholeskyQR pass factors (single-pass core)
    int* defic;       // columns found numerically dependent in the extra CholeskyQR pass
    float* rinv;      // FP32 inverse of a CholeskyQR factor (triangular solves of FP32 panels)
    void *xc, *q1c, *q2c, *part;
    void* abf;        // bf16 copy of A for CORUTV_P_BF16, or its bf16 splits for the projection
    float* at;        // TF32: A^T (n rows, row stride ldm), so that A^T Y has K-major operands
    float* a32;       // TF32: padded copy of A when A itself is not TMA-aligned
    int *perm, *skip;
    int* tcnt;        // per-tile counters of the tensor-core products, then gcnt
    int* gcnt;        // counters of the FP32 Gram kernel
};

// a_aligned: the device copy of A that the factorisation reads starts on a
// 16-byte boundary (only TF32 sketches read A itself through TMA).
// t_lower: the variant with a lower triangular T (Algorithm 1 on A^T).
corutv_status make_plan(FactorPlan& pl, ElemType ta, int64_t m, int64_t n, int64_t lda, int64_t k,
                        int64_t p, int64_t q, corutv_prec prec, int num_sms, bool a_aligned = true,
                        int d_mode = 0, bool t_lower = false, uint32_t power_form = 0,
                        uint32_t bf16_last_round = 0) {
    pl.tr = t_lower;
    pl.ma = m; pl.na = n;
    pl.m = t_lower ? n : m; pl.n = t_lower ? m : n;
    pl.lda = lda; pl.k = k; pl.p = p; pl.q = q;
    pl.ell = k + p;
    pl.ta = ta;
    pl.prec = prec;
    pl.num_sms = num_sms;
    if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0)
        return fail(CORUTV_EINVAL, "invalid sizes m=%lld n=%lld k=%lld p=%lld q=%lld", (long long)m,
                    (long long)n, (long long)k, (long long)p, (long long)q);
    if (pl.ell >= std::min(m, n))
        return fail(CORUTV_EINVAL, "ell = k + p = %lld must be < min(m, n) = %lld", (long long)pl.ell,
                    (long long)std::min(m, n));
    if (lda < n) return fail(CORUTV_EINVAL, "lda = %lld < n = %lld", (long long)lda, (long long)n);
    if (prec < CORUTV_P_F64 || prec > CORUTV_P_BF16) return fail(CORUTV_EINVAL, "unknown sketch precision %d", (int)prec);
    pl.tensor = (prec == CORUTV_P_TF32 || prec == CORUTV_P_BF16);
    // tensor-core sketches up to 128 columns; FP64 / FP32 sketches up to 320
    if (pl.ell > (pl.tensor ? 128 : kMaxEllSimt))
        return fail(CORUTV_EINVAL, "ell = %lld exceeds the supported maximum %d for this sketch precision",
                    (long long)pl.ell, pl.tensor ? 128 : kMaxEllSimt);
    if (prec == CORUTV_P_TF32 && ta != T_F32) return fail(CORUTV_EINVAL, "TF32 sketches need FP32 input");
    if (d_mode != 0 && d_mode != 1) return fail(CORUTV_EINVAL, "d_mode %d is not supported (0 exact D, 1 single-pass core)", d_mode);
    pl.dmode = d_mode;
    pl.split = pl.tensor && ta == T_F32 && d_mode == 0;  // the bf16 splits serve the projection only
    if (power_form > 1) return fail(CORUTV_EINVAL, "power_form %u is not supported (0 or 1)", power_form);
    if (bf16_last_round > 1) return fail(CORUTV_EINVAL, "bf16_last_round %u is not supported (0 or 1)", bf16_last_round);
    pl.power_form = (int)power_form;
    pl.x2_last = pl.split && prec == CORUTV_P_BF16 && bf16_last_round == 1;
    pl.copy_a = prec == CORUTV_P_TF32 && (!a_aligned || lda % 4 != 0);
    pl.ldc32 = round_up(n, 4);
    pl.ellp = pl.tensor ? round_up(pl.ell, 16) : pl.ell;
    pl.ldm = round_up(pl.m, 64);
    pl.ldn = round_up(pl.n, 64);
    pl.ldma = t_lower ? pl.ldn : pl.ldm;
    pl.ldna = t_lower ? pl.ldm : pl.ldn;
    pl.tcomp = pl.tensor ? (prec == CORUTV_P_BF16 ? T_BF16 : T_F32) : (prec == CORUTV_P_F64 ? T_F64 : T_F32);
    pl.tdproj = (ta == T_F64) ? T_F64 : T_F32;
    pl.torth = (prec == CORUTV_P_F64) ? T_F64 : T_F32;
    pl.tp = (ta == T_F32 && prec != CORUTV_P_F64) ? T_F32 : T_F64;
    pl.sp_ax = gemm_simt_splits(pl.m, pl.n, num_sms);
    pl.sp_aty = gemm_simt_splits(pl.n, pl.m, num_sms);
    pl.gs_m = gemm_simt_splits(pl.ell, m, num_sms);
    pl.gs_n = gemm_simt_splits(pl.ell, n, num_sms);
    int64_t part = std::max((int64_t)pl.sp_ax * pl.ellp * pl.ldm, (int64_t)pl.sp_aty * pl.ellp * pl.ldn);
    if (pl.tensor) part = std::max(part, tc_partial_elems(pl.m, pl.n, pl.ellp, pl.ldm, pl.ldn, num_sms));
    pl.part_elems = part;
    return CORUTV_OK;
}

int64_t factor_counters(const FactorPlan& pl) {
    return tc_counter_elems(pl.m, pl.n) + gram_f32_counters(std::max(pl.m, pl.n), (int)pl.ell, pl.num_sms);
}

template <class C>
void carve_factor(C& cv, const FactorPlan& pl, FactorBufs& b) {
    const int64_t pm = pl.ellp * pl.ldm, pn = pl.ellp * pl.ldn, ll = pl.ellp * pl.ellp;
    const int es_c = elem_size(pl.tcomp), es_d = elem_size(pl.tdproj), es_p = elem_size(pl.tp);
    b.x = cv.template take<char>(pn * es_p);
    b.c1 = cv.template take<char>(pm * es_p);
    b.q1 = cv.template take<char>(pm * es_p);
    b.c2 = cv.template take<char>(pn * es_p);
    b.q2 = cv.template take<char>(pn * es_p);
    b.w = cv.template take<char>(std::max(pm, pn) * es_p);  // A Q2, or A Q1 for the lower-T variant
    b.tmp = cv.template take<char>(std::max(pm, pn) * es_p);
    b.upanel = cv.template take<double>(pm);
    b.zpanel = cv.template take<double>(pn);
    b.gpart = cv.template take<double>(std::max((int64_t)std::max(pl.gs_m, pl.gs_n) * ll,
                                                (gram_f32_work_floats(std::max(pl.m, pl.n), (int)pl.ell,
                                                                      pl.num_sms) + 1) / 2));
    b.g = cv.template take<double>(ll);
    b.r = cv.template take<double>(ll);
    b.d = cv.template take<double>(ll);
    b.qt = cv.template take<double>(ll);
    b.rt = cv.template take<double>(ll);
    b.refl = cv.template take<double>(pl.ellp * (pl.ellp + 2));
    b.racc = pl.dmode == 1 ? cv.template take<double>(ll) : nullptr;
    b.racc2 = pl.dmode == 1 ? cv.template take<double>(ll) : nullptr;
    b.defic = cv.template take<int>(pl.ellp);
    b.rinv = reinterpret_cast<float*>(cv.template take<double>(trsm_rinv_floats(pl.ellp)));  // FP64 for wide FP64 panels
    b.xc = cv.template take<char>(pn * es_c);
    b.q1c = cv.template take<char>(pm * es_c);
    b.q2c = cv.template take<char>(pl.split ? 3 * std::max(pm, pn) * 2 : std::max(pm, pn) * es_d);
    b.part = cv.template take<char>(pl.part_elems * std::max(8, std::max(es_c, es_d)));
    b.abf = (pl.prec == CORUTV_P_BF16 || pl.split) ? cv.template take<char>((pl.split ? 3 : 1) *
                                                                            tiled_part_bytes(pl.ma, pl.na))
                                                   : nullptr;
    b.at = pl.prec == CORUTV_P_TF32 ? cv.template take<float>(pl.na * pl.ldma) : nullptr;
    b.a32 = pl.copy_a ? cv.template take<float>(pl.ma * pl.ldc32) : nullptr;
    b.perm = cv.template take<int>(pl.ellp);
    b.skip = cv.template take<int>(8);
    b.tcnt = cv.template take<int>(factor_counters(pl));
    b.gcnt = b.tcnt + tc_counter_elems(pl.m, pl.n);
}

size_t factor_bytes(const FactorPlan& pl) {
    Carver cv(nullptr);
    FactorBufs b;
    carve_factor(cv, pl, b);
    return cv.off;
}

// The exchange of a row-partitioned factorisation (corutv_factor_rows): sums
// over the ranks through the caller's callback, on pinned host buffers.
struct Exchange {
    corutv_allreduce_fn fn = nullptr;
    void* user = nullptr;
    void* host = nullptr;      // pinned staging buffer
    int64_t total_rows = 0;    // rows of the whole matrix (sizes the Cholesky shift)
};

// The bf16 splits A_m, A_l of the tiled copy (needed only by the projection,
// eq. 7) cast on a side stream in row chunks while the main stream runs the
// thin QRs' single-SM FP64 steps: one chunk is forked at the first Gram of
// every thin QR and joined before the next product over A, the rest forked
// and joined before the projection. The critical path casts A_h alone.
struct CastOverlap {
    cudaStream_t side = nullptr;
    cudaEvent_t* ev = nullptr;   // 2 per chunk: fork (main) and done (side)
    const void* a = nullptr;
    ElemType ta = T_F32;
    int64_t m = 0, n = 0, lda = 0;
    void* out = nullptr;
    const int* cancel = nullptr;
    int parts = 2;               // 2: A_m, A_l (A_h is on the critical path); 3: all three (TF32 sketches)
    int chunks = 0, issued = 0, joined = 0;
    cudaEvent_t psi_fork = nullptr, psi_done = nullptr;  // the test matrix formed on the side stream
    bool psi_pending = false;
    cudaEvent_t emit_fork = nullptr, emit_done = nullptr;  // T, V, perm written on the side stream
    corutv_status issue(cudaStream_t main) {
        if (issued >= chunks) return CORUTV_OK;
        const int64_t mt = (m + 127) / 128;
        const int64_t rb0 = mt * issued / chunks, rb1 = mt * (issued + 1) / chunks;
        CK(cudaEventRecord(ev[2 * issued], main));
        CK(cudaStreamWaitEvent(side, ev[2 * issued], 0));
        if (rb1 > rb0) CK(launch_cast_tiled_rows(a, ta, m, n, lda, out, parts, rb0, rb1, cancel, side));
        CK(cudaEventRecord(ev[2 * issued + 1], side));
        ++issued;
        return CORUTV_OK;
    }
    corutv_status join(cudaStream_t main) {
        if (psi_pending) {
            CK(cudaStreamWaitEvent(main, psi_done, 0));
            psi_pending = false;
        }
        for (; joined < issued; ++joined) CK(cudaStreamWaitEvent(main, ev[2 * joined + 1], 0));
        return CORUTV_OK;
    }
    corutv_status finish(cudaStream_t main) {
        while (issued < chunks) CKS(issue(main));
        return join(main);
    }
};
constexpr int kMaxCastChunks = 8;

struct Exec {
    cudaStream_t st;
    int* flags;
    const int* cancel;
    int num_sms;
    Profiler* prof = nullptr;
    const Exchange* xch = nullptr;  // set for the rows of a row-partitioned matrix
    CastOverlap* ov = nullptr;      // set: A_m, A_l are cast on a side stream (run_factor)
};

// buf (device, count elements of type t) <- its sum over the ranks: copied to
// the pinned staging buffer once the stream has produced it, summed in place by
// the caller's callback, copied back in stream order.
corutv_status exchange_sum(const Exec& ex, void* buf, int64_t count, ElemType t) {
    const size_t bytes = (size_t)count * elem_size(t);
    CK(cudaMemcpyAsync(ex.xch->host, buf, bytes, cudaMemcpyDeviceToHost, ex.st));
    CK(cudaStreamSynchronize(ex.st));
    const corutv_status st = ex.xch->fn(ex.xch->host, count, t == T_F64 ? CORUTV_F64 : CORUTV_F32, ex.xch->user);
    if (st != CORUTV_OK) return fail(st, "the all-reduce callback returned status %d", (int)st);
    CK(cudaMemcpyAsync(buf, ex.xch->host, bytes, cudaMemcpyHostToDevice, ex.st));
    return CORUTV_OK;
}

// C = A X (am = A_ROWS, R = m, K = n) or A^T Y (am = A_COLS, R = n, K = m) on
// SIMT cores for A's own m x n, written to the panel `out` (type pl.tp).
corutv_status sketch_simt(const Exec& ex, const FactorPlan& pl, const FactorBufs& b, AMode am,
                          const void* a, ElemType ta, const void* bop, ElemType tc, void* out,
                          int64_t ldout) {
    const int64_t R = am == A_ROWS ? pl.ma : pl.na;
    const int64_t K = am == A_ROWS ? pl.na : pl.ma;
    const int splits = gemm_simt_splits(R, K, ex.num_sms);
    const int64_t ldb = am == A_ROWS ? pl.ldna : pl.ldma;
    GemmArgs g{am, B_PANEL, O_PANEL, ta, tc, a, pl.lda, bop, ldb, b.part, ldout, pl.ellp * ldout,
               R, K, pl.ell, splits, ex.cancel};
    {
        ProfScope ps(ex.prof, CORUTV_STAGE_SKETCH, ex.st);
        CK(launch_gemm_simt(g, ex.st));
    }
    CK(launch_reduce_splits(b.part, tc, splits, pl.ellp * ldout, out, pl.tp, ldout, R, pl.ell, ldout, ex.cancel,
                            ex.st));
    return CORUTV_OK;
}

// G = X^T Y (ell x ell, written as FP64) for two panels of type pl.tp and
// `len` rows; products and split sums in arithmetic tg.
// px / py: pieces of a tensor-core product still to be added to X / Y (the
// Gram is their first reader; writeback completes the panel for later ones).
corutv_status gram(const Exec& ex, const FactorPlan& pl, const FactorBufs& b, const void* x,
                   int64_t ldx, const void* y, int64_t ldy, int64_t len, double* out,
                   const int* cancel, ElemType tg, const TcPieces* px = nullptr, const TcPieces* py = nullptr,
                   bool writeback = false) {
    if (tg == T_F32 && pl.tp == T_F32 && b.gcnt) {
        // one launch, split sums reduced in the kernel
        CK(launch_gram_f32(static_cast<const float*>(x), ldx, static_cast<const float*>(y), ldy, len, (int)pl.ell,
                           out, reinterpret_cast<float*>(b.gpart), b.gcnt, ex.num_sms, cancel, ex.st,
                           px ? *px : TcPieces(), py ? *py : TcPieces(), writeback));
        return CORUTV_OK;
    }
    if ((px && px->part) || (py && py->part)) return fail(CORUTV_ECUDA, "pending product pieces need the FP32 Gram");
    const int gs = gemm_simt_splits(pl.ell, len, ex.num_sms);
    const int64_t ll = pl.ell * pl.ell;
    GemmArgs g{A_PANEL_T, B_PANEL, O_ROWMAJ, pl.tp, tg, x, ldx, y, ldy, b.gpart, pl.ell, ll,
               pl.ell, len, pl.ell, gs, cancel};
    g.tb = pl.tp;
    CK(launch_gemm_simt(g, ex.st));
    CK(launch_reduce_splits(b.gpart, tg, gs, ll, out, T_F64, pl.ell, pl.ell, pl.ell, pl.ell, cancel, ex.st));
    return CORUTV_OK;
}

// Thin QR of the panel c (len x ell, type pl.tp) by CholeskyQR: `passes` = 2
// gives CholeskyQR2 (used for the bases Q1, Q2 that leave the power loop, and
// everywhere on the FP64 path); `passes` = 1 is used for the intermediate
// bases of the power iteration on the mixed paths, where only the span
// matters. A pass whose Gram needed the shift is followed by one more pass
// (shifted CholeskyQR3). Gram products and triangular solves run in
// pl.torth; every Cholesky factorisation runs in FP64. Writes the panel q
// (type pl.tp) and, if qc != nullptr, a copy of type tqc.
corutv_status orth(const Exec& ex, const FactorPlan& pl, const FactorBufs& b, const void* c,
                   int64_t ld, int64_t len, void* q, void* qc, ElemType tqc, int passes = 2,
                   double* rt_out = nullptr, const TcPieces* pieces = nullptr, bool dist = false) {
    const int64_t ell = pl.ell;
    const ElemType tw = pl.torth, tp = pl.tp;
    ProfScope ps(ex.prof, CORUTV_STAGE_ORTH, ex.st);
    // a panel whose rows are spread over ranks: each Gram is the sum of the
    // ranks' Gram matrices, and the shift counts all rows
    const bool sum = dist && ex.xch;
    const int64_t rows_all = sum ? ex.xch->total_rows : len;
    void* p1 = passes == 1 ? q : b.tmp;
    void* p1c = passes == 1 ? qc : nullptr;
    // pass 1 (the first reader of c: it adds any pieces the product left and completes c)
    CKS(gram(ex, pl, b, c, ld, c, ld, len, b.g, ex.cancel, tw, pieces, pieces, true));
    if (ex.ov) CKS(ex.ov->issue(ex.st));  // a chunk of A_m, A_l beside the Cholesky and the solves
    if (sum) CKS(exchange_sum(ex, b.g, ell * ell, T_F64));
    const double u = tw == T_F64 ? 0x1p-53 : 0x1p-24;  // unit roundoff of the Gram arithmetic
    CK(launch_cholesky(b.g, ell, rows_all, b.r, ex.flags, b.skip, ex.cancel, ex.st, u));
    if (rt_out) CK(launch_trimul(b.r, nullptr, b.racc, ell, false, nullptr, ex.cancel, ex.st));
    CK(launch_trsm_rows(c, tp, ld, len, ell, b.r, tw, p1, ld, p1c, tqc, ld, ex.cancel, ex.st, nullptr, b.rinv));
    // extra pass, only after a shifted pass 1. Directions the shifted pass left
    // at rounding level (a numerically rank-deficient C) cannot be restored
    // from C: their columns get a seeded random completion, orthonormalised by
    // the following pass (and well conditioned as they stand for a
    // one-pass intermediate basis).
    CKS(gram(ex, pl, b, p1, ld, p1, ld, len, b.g, b.skip, tw));
    if (sum) CKS(exchange_sum(ex, b.g, ell * ell, T_F64));  // (summed but unused when the pass is skipped)
    CK(launch_cholesky(b.g, ell, rows_all, b.r, ex.flags, nullptr, b.skip, ex.st, u, b.defic, 10.0 * (double)ell * u));
    // the extra pass's factor joins the product only if that pass ran
    if (rt_out) CK(launch_trimul(b.r, b.racc, b.racc2, ell, false, b.skip, ex.cancel, ex.st));
    CK(launch_trsm_rows(p1, tp, ld, len, ell, b.r, tw, p1, ld, p1c, tqc, ld, b.skip, ex.st, b.defic, b.rinv));
    if (passes == 1) return rt_out ? fail(CORUTV_EINVAL, "the R factor needs two passes") : CORUTV_OK;
    // pass 2
    CKS(gram(ex, pl, b, b.tmp, ld, b.tmp, ld, len, b.g, ex.cancel, tw));
    if (sum) CKS(exchange_sum(ex, b.g, ell * ell, T_F64));
    CK(launch_cholesky(b.g, ell, rows_all, b.r, ex.flags, nullptr, ex.cancel, ex.st, u));
    // C = Q (R_2 R_extra R_1): rt_out receives that product transposed
    if (rt_out) CK(launch_trimul(b.r, b.racc2, rt_out, ell, true, nullptr, ex.cancel, ex.st));
    CK(launch_trsm_rows(b.tmp, tp, ld, len, ell, b.r, tw, q, ld, qc, tqc, ld, ex.cancel, ex.st, nullptr, b.rinv));
    return CORUTV_OK;
}

// U = Q1 Qt is formed from the explicit Qt (qform) for FP32 panels wider than 64
// columns; otherwise from the reflectors.
bool explicit_qt(const FactorPlan& pl, ElemType tout) {
    return pl.ell > 128 || (pl.tp == T_F32 && tout == T_F32 && pl.ell > 64);
}

// Algorithm 1 on device data; leaves Q1, Q2, D, Qt, Rt, perm in the buffers.
// psi_dev: optional n x ell row-major FP64 test matrix.
corutv_status run_factor(const Exec& ex, const FactorPlan& pl, const FactorBufs& b, const void* a,
                         const double* psi_dev, uint64_t seed, uint32_t sid) {
    const int64_t m = pl.m, n = pl.n, ell = pl.ell;
    ProfScope ps_all(ex.prof, CORUTV_STAGE_FACTOR, ex.st);
    // Step 1: X = Psi (panel n x ellp, padding columns zero); with a side stream
    // it is formed there, beside the cast of A, and joined before the first product
    const bool side_psi = ex.ov && pl.tensor && pl.split && ex.ov->psi_fork;
    cudaStream_t pst = ex.st;
    if (side_psi) {
        CK(cudaEventRecord(ex.ov->psi_fork, ex.st));
        CK(cudaStreamWaitEvent(ex.ov->side, ex.ov->psi_fork, 0));
        pst = ex.ov->side;
    }
    if (psi_dev) CK(launch_rowmajor_to_panel(psi_dev, ell, n, ell, pl.ellp, b.x, pl.tp, pl.ldn, pst));
    else CK(launch_gaussian_panel(seed, sid, n, ell, pl.ellp, b.x, pl.tp, pl.ldn, ex.cancel, pst));
    // the workspace is shared with other entry points: start the kernels' counters at zero
    CK(cudaMemsetAsync(b.tcnt, 0, sizeof(int) * (size_t)factor_counters(pl), ex.st));
    if (pl.tensor) {
        // padding columns of the bf16 / fp32 operand panels must read as zero
        CK(cudaMemsetAsync(b.q1c, 0, (size_t)pl.ellp * pl.ldm * elem_size(pl.tcomp), ex.st));
        CK(launch_panel_convert(b.x, pl.tp, pl.ldn, n, pl.ellp, b.xc, pl.tcomp, pl.ldn, ex.cancel, pst));
        if (side_psi) {
            CK(cudaEventRecord(ex.ov->psi_done, pst));
            ex.ov->psi_pending = true;
        }
        if (pl.prec == CORUTV_P_TF32 && pl.split && ex.ov) {
            // A^T (and the padded copy) now; the bf16 splits for eq. 7 in row chunks on the side stream
            CK(launch_prep_f32(static_cast<const float*>(a), pl.ma, pl.na, pl.lda, b.at, pl.ldma, nullptr, b.a32,
                               pl.ldc32, ex.cancel, ex.st));
            CastOverlap& ov = *ex.ov;
            ov.a = a;
            ov.ta = pl.ta;
            ov.m = pl.ma;
            ov.n = pl.na;
            ov.lda = pl.lda;
            ov.out = b.abf;
            ov.cancel = ex.cancel;
            ov.parts = 3;
            ov.chunks = (int)std::min<int64_t>(kMaxCastChunks, std::max<int64_t>(1, 2 * pl.q + 2));
            ov.issued = ov.joined = 0;
        } else if (pl.prec == CORUTV_P_TF32)
            // one pass over A: A^T for the K-major A^T Y, the tiled bf16 splits for eq. 7
            CK(launch_prep_f32(static_cast<const float*>(a), pl.ma, pl.na, pl.lda, b.at, pl.ldma, b.abf, b.a32,
                               pl.ldc32, ex.cancel, ex.st));
        else if (pl.prec == CORUTV_P_BF16 && pl.split && ex.ov) {
            // A_h now; A_m, A_l for eq. 7 in row chunks on the side stream (CastOverlap)
            CK(launch_cast_tiled(a, pl.ta, pl.ma, pl.na, pl.lda, b.abf, 1, ex.cancel, ex.st));
            CastOverlap& ov = *ex.ov;
            ov.a = a;
            ov.ta = pl.ta;
            ov.m = pl.ma;
            ov.n = pl.na;
            ov.lda = pl.lda;
            ov.out = b.abf;
            ov.cancel = ex.cancel;
            ov.chunks = (int)std::min<int64_t>(kMaxCastChunks, std::max<int64_t>(1, 2 * pl.q + 2));
            ov.issued = ov.joined = 0;
        } else if (pl.prec == CORUTV_P_BF16)
            // the tiled bf16 copy the products read (A_h), with A_m, A_l for eq. 7 when split
            CK(launch_cast_tiled(a, pl.ta, pl.ma, pl.na, pl.lda, b.abf, pl.split ? 3 : 1, ex.cancel, ex.st));
    } else {
        CK(launch_panel_convert(b.x, pl.tp, pl.ldn, n, ell, b.xc, pl.tcomp, pl.ldn, ex.cancel, ex.st));
    }
    // split tiles of a tensor-core product stay pieces until the Gram that
    // first reads the panel adds them (no fix-up tail in the product)
    TcPieces pieces;
    // (a row-partitioned run sums its panels over ranks: no pieces left for a consumer).
    // Measured: the deferral pays up to about 10^4 rows (8000 x 6000, ell = 60:
    // 1.139 against 1.144 ms; 8000 x 8000, ell = 110: equal); beyond, the Gram's
    // per-row piece loads cost more than the products' own fix-up (20000 x 20000,
    // ell = 110: 4.28 against 4.19 ms). Bitwise the same sums either way.
    TcPieces* defer = (pl.tp == T_F32 && pl.torth == T_F32 && pl.tdproj == T_F32 && !ex.xch &&
                       std::max(pl.m, pl.n) <= 12000)
                          ? &pieces
                          : nullptr;
    // A X (a_rows: the output has A's rows, the operand is a panel with A's
    // columns) or A^T Y (the other way round). Algorithm 1's C1 = A X is the
    // first, C2 = A^T Q1 the second; on A^T (the lower-T variant) the two swap.
    auto product = [&](bool a_rows, const void* opnd, void* out, TcPieces* pc, int nsegs = 1) -> corutv_status {
        const int64_t ldo = a_rows ? pl.ldna : pl.ldma, ldout = a_rows ? pl.ldma : pl.ldna;
        if (!pl.tensor) return sketch_simt(ex, pl, b, a_rows ? A_ROWS : A_COLS, a, pl.ta, opnd, pl.tcomp, out, ldout);
        if (ex.ov && (ex.ov->chunks || ex.ov->psi_pending)) CKS(ex.ov->join(ex.st));  // nothing beside a product
        ProfScope ps(ex.prof, CORUTV_STAGE_SKETCH, ex.st);
        if (pl.prec == CORUTV_P_BF16) {
            // the tiled bf16 copy (its first part, A_h) serves both directions
            CK(launch_sketch_tc_tiled(b.abf, pl.ma, pl.na, a_rows ? 0 : 1, opnd, ldo, ell, pl.ellp, b.part, b.tcnt,
                                      out, pl.tp, ldout, ex.num_sms, ex.flags, ex.cancel, ex.st, pc, nsegs));
        } else if (a_rows) {
            const void* aop = pl.copy_a ? static_cast<const void*>(b.a32) : a;
            const int64_t lda_op = pl.copy_a ? pl.ldc32 : pl.lda;
            CK(launch_sketch_tc(aop, pl.tcomp, pl.ma, pl.na, lda_op, /*trans=*/0, opnd, ldo, ell, pl.ellp, b.part,
                                b.tcnt, out, pl.tp, ldout, ex.num_sms, ex.flags, ex.cancel, ex.st, pc));
        } else {  // TF32: (A^T) Y with the transposed copy, both operands K-major
            CK(launch_sketch_tc(b.at, pl.tcomp, pl.na, pl.ma, pl.ldma, /*trans=*/0, opnd, ldo, ell, pl.ellp, b.part,
                                b.tcnt, out, pl.tp, ldout, ex.num_sms, ex.flags, ex.cancel, ex.st, pc));
        }
        return CORUTV_OK;
    };
    for (int64_t it = 0; it <= pl.q; ++it) {
        // the last round's products read A_h + A_m when asked (the rounding of A's
        // bf16 copy there is what limits the captured subspace)
        const int nsegs = (pl.x2_last && it == pl.q) ? 2 : 1;
        // one thin QR per power round: C1 = A X is the operand of A^T as it is
        const bool raw_c1 = pl.power_form == 1 && it < pl.q;
        // eq. 4: C1 = A X
        CKS(product(!pl.tr, b.xc, b.c1, raw_c1 ? nullptr : defer, nsegs));
        const int inner = (pl.prec == CORUTV_P_F64) ? 2 : 1;  // passes for the intermediate bases
        if (raw_c1) {
            CK(launch_panel_convert(b.c1, pl.tp, pl.ldm, m, ell, b.q1c, pl.tcomp, pl.ldm, ex.cancel, ex.st));
        } else {
            CKS(orth(ex, pl, b, b.c1, pl.ldm, m, b.q1, b.q1c, pl.tcomp, it < pl.q ? inner : 2, nullptr, &pieces,
                     /*dist=*/true));
        }
        pieces = TcPieces();
        // eq. 5 (with C1 -> Q1): C2 = A^T Q1
        CKS(product(pl.tr, b.q1c, b.c2, defer, nsegs));
        // row-partitioned: C2 = sum over the ranks of A_i^T Q1_i (eq. 5), then replicated
        if (ex.xch) CKS(exchange_sum(ex, b.c2, ell * pl.ldn, pl.tp));
        if (it < pl.q) {
            CKS(orth(ex, pl, b, b.c2, pl.ldn, n, b.x, b.xc, pl.tcomp, inner, nullptr, &pieces));
            pieces = TcPieces();
        }
    }
    // Q2 = qr(C2), with a copy in the projection's arithmetic
    // single-pass core (Sec. 3.1): D_approx = Q1^T C1 (Q2^T X)^+, and with
    // C2 = A^T Q1 = Q2 R2 that is R2^T (Q2^T X)(Q2^T X)^+ = R2^T: the transposed
    // product of this thin QR's pass factors, with no third pass over A
    if (pl.dmode == 1) {
        CKS(orth(ex, pl, b, b.c2, pl.ldn, n, b.q2, nullptr, pl.tdproj, 2, b.d, &pieces));
        ProfScope ps(ex.prof, CORUTV_STAGE_QRCP, ex.st);
        CK(launch_qrcp(b.d, ell, b.qt, b.rt, b.perm, b.refl, ex.cancel, ex.st, explicit_qt(pl, pl.tp) && !ex.ov));
        return CORUTV_OK;
    }
    // the non-split projection multiplies A by Q2 in its own arithmetic (a copy
    // made here), or by Q1 for the lower-T variant (converted below)
    CKS(orth(ex, pl, b, b.c2, pl.ldn, n, b.q2, (pl.split || pl.tr) ? nullptr : b.q2c, pl.tdproj, 2, nullptr,
             &pieces));
    pieces = TcPieces();
    // eq. 7: W = A Q2 (FP64, or FP32-accurate from the original A), D = Q1^T W.
    // Lower-T variant (Algorithm 1 on A^T): D = Q1^T A^T Q2 = (A Q1)^T Q2, so W = A Q1
    // and D = W^T Q2 -- the same product with A, Q1 in the place of Q2.
    const void* pan = pl.tr ? b.q1 : b.q2;  // the operand panel (A's columns)
    if (pl.split) {
        if (ex.ov && ex.ov->chunks) CKS(ex.ov->finish(ex.st));  // all of A_m, A_l before eq. 7
        CK(launch_split_panel(static_cast<const float*>(pan), pl.ldna, pl.na, ell, pl.ellp, b.q2c, pl.ldna,
                              ex.cancel, ex.st));
        ProfScope ps(ex.prof, CORUTV_STAGE_PROJECT, ex.st);
        CK(launch_project_split_tc_tiled(b.abf, pl.ma, pl.na, b.q2c, pl.ldna, ell, pl.ellp, b.part, b.tcnt, b.w,
                                         pl.tp, pl.ldma, ex.num_sms, ex.flags, ex.cancel, ex.st, defer));
    } else {
        const void* opnd = b.q2c;
        if (pl.tr) {
            if (pl.tp == pl.tdproj) opnd = b.q1;
            else CK(launch_panel_convert(b.q1, pl.tp, pl.ldna, pl.na, ell, b.q2c, pl.tdproj, pl.ldna, ex.cancel, ex.st));
        }
        const int sp = gemm_simt_splits(pl.ma, pl.na, ex.num_sms);
        GemmArgs g{A_ROWS, B_PANEL, O_PANEL, pl.ta, pl.tdproj, a, pl.lda, opnd, pl.ldna, b.part, pl.ldma,
                   pl.ellp * pl.ldma, pl.ma, pl.na, ell, sp, ex.cancel};
        {
            ProfScope ps(ex.prof, CORUTV_STAGE_PROJECT, ex.st);
            CK(launch_gemm_simt(g, ex.st));
        }
        CK(launch_reduce_splits(b.part, pl.tdproj, sp, pl.ellp * pl.ldma, b.w, pl.tp, pl.ldma, pl.ma, ell, pl.ldma,
                                ex.cancel, ex.st));
    }
    if (pl.tr) CKS(gram(ex, pl, b, b.w, pl.ldn, b.q2, pl.ldn, n, b.d, ex.cancel, pl.tdproj, &pieces, nullptr));
    else CKS(gram(ex, pl, b, b.q1, pl.ldm, b.w, pl.ldm, m, b.d, ex.cancel, pl.tdproj, nullptr, &pieces));
    // row-partitioned: D = sum over the ranks of Q1_i^T (A_i Q2) (eq. 7)
    if (ex.xch) CKS(exchange_sum(ex, b.d, ell * ell, T_F64));
    // eq. 8: D P = Qt Rt
    {
        ProfScope ps(ex.prof, CORUTV_STAGE_QRCP, ex.st);
        CK(launch_qrcp(b.d, ell, b.qt, b.rt, b.perm, b.refl, ex.cancel, ex.st, explicit_qt(pl, pl.tp) && !ex.ov));
    }
    return CORUTV_OK;
}

// Eq. 9 into caller buffers (device): U = Q1 Qt, T = Rt, V = Q2 P, perm. For
// the lower-T variant the run was on A^T: A's U is that run's Q2 P (the
// permutation acts on U's columns), V its Q1 Qt and T = Rt^T.
corutv_status emit_user(const Exec& ex, const FactorPlan& pl, const FactorBufs& b, ElemType tout, void* u,
                        int64_t ldu, void* t, void* v, int64_t ldv, int32_t* perm) {
    const int64_t ell = pl.ell;
    void* uq = pl.tr ? v : u;  // receives Q1 Qt
    void* vq = pl.tr ? u : v;  // receives Q2 P
    const int64_t lduq = pl.tr ? ldv : ldu, ldvq = pl.tr ? ldu : ldv;
    // with a side stream: T, V = Q2 P and perm there, beside the formation of Qt
    // (run_factor left it to this step) and U = Q1 Qt on the main stream
    cudaStream_t sst = ex.st;
    if (ex.ov && ex.ov->emit_fork) {
        CK(cudaEventRecord(ex.ov->emit_fork, ex.st));
        CK(cudaStreamWaitEvent(ex.ov->side, ex.ov->emit_fork, 0));
        sst = ex.ov->side;
        CK(launch_copy_small(b.rt, ell, t, tout, ex.cancel, sst, pl.tr));
        if (vq) CK(launch_gather_v(b.q2, pl.tp, pl.ldn, pl.n, ell, b.perm, vq, tout, ldvq, ex.cancel, sst));
        if (perm) CK(cudaMemcpyAsync(perm, b.perm, sizeof(int32_t) * ell, cudaMemcpyDeviceToDevice, sst));
        CK(cudaEventRecord(ex.ov->emit_done, sst));
    }
    if (ex.ov && explicit_qt(pl, pl.tp)) CK(launch_qform(b.refl, ell, b.qt, ex.cancel, ex.st));
    if (uq && explicit_qt(pl, tout) && pl.tp == T_F64) {
        // Q1 Qt as an FP64 product with the explicit Qt (widths beyond the
        // reflector kernel's shared memory)
        GemmArgs g{A_PANEL, B_SMALL, O_ROWMAJ, T_F64, tout, b.q1, pl.ldm, b.qt, ell, uq, lduq, 0,
                   pl.m, ell, ell, 1, ex.cancel, T_F64};
        CK(launch_gemm_simt(g, ex.st));
    } else if (uq && explicit_qt(pl, tout)) {
        // Q1 Qt as a product with the explicit Qt (FP32): for wide Qt the reflector
        // form below is a long per-row chain (ell reflectors of ell entries each)
        float* qt32 = static_cast<float*>(b.tmp);
        CK(launch_copy_small(b.qt, ell, qt32, T_F32, ex.cancel, ex.st));
        GemmArgs g{A_PANEL, B_SMALL, O_ROWMAJ, T_F32, T_F32, b.q1, pl.ldm, qt32, ell, uq, lduq, 0,
                   pl.m, ell, ell, 1, ex.cancel};
        CK(launch_gemm_simt(g, ex.st));
    } else if (uq) {
        // Q1 Qt, applied as the QRCP's reflectors to the rows of Q1
        CK(launch_apply_reflectors(b.q1, pl.tp, pl.ldm, pl.m, ell, b.refl, uq, tout, lduq, false, ex.cancel, ex.st));
    }
    if (sst != ex.st) {
        CK(cudaStreamWaitEvent(ex.st, ex.ov->emit_done, 0));  // joined: the call ends on the main stream
        return CORUTV_OK;
    }
    CK(launch_copy_small(b.rt, ell, t, tout, ex.cancel, ex.st, pl.tr));
    if (vq) CK(launch_gather_v(b.q2, pl.tp, pl.ldn, pl.n, ell, b.perm, vq, tout, ldvq, ex.cancel, ex.st));
    if (perm) CK(cudaMemcpyAsync(perm, b.perm, sizeof(int32_t) * ell, cudaMemcpyDeviceToDevice, ex.st));
    return CORUTV_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device's view of page-locked host memory (UVA), or null for pageable
// memory and device pointers: kernels may read such memory directly.
const void* pinned_host_view(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct ServingSlot {
    cudaStream_t st = nullptr;
    DeviceBuffer ws;
    int* flags = nullptr;   // device
    int* hflags = nullptr;  // pinned host mirror
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    int32_t* perm_host = nullptr;
};

struct PendingReq {
    uint64_t ticket;
    corutv_request req;
    std::chrono::steady_clock::time_point t0;
    size_t bytes;
    bool host;
    cudaEvent_t ready = nullptr;  // device inputs: recorded on the caller's stream at submit
};

struct ReqResult {
    bool done = false;
    corutv_status status = CORUTV_EPENDING;
    double latency = 0.0;
    std::chrono::steady_clock::time_point t0;
    std::string msg;  // the dispatcher's message for a failed request
};

// State of the grouped executor (corutv_factor_batch): the problems'
// buffers, the launch records and their pinned staging copy.
struct BatchState {
    DeviceBuffer ws, desc;
    char* host = nullptr;         // pinned staging of the records
    size_t hcap = 0;
    cudaEvent_t copied = nullptr;  // recorded after the records' copy: `host` may be rewritten
    std::vector<char> rec;        // records being built
};

// A serving lane of the batching dispatcher (corutv_set_batching): runs one
// batch of admitted requests at a time with grouped launches on its stream.
struct BatchLane {
    cudaStream_t st = nullptr;
    BatchState bs;
    int* flags = nullptr;   // device
    int* hflags = nullptr;  // pinned host mirror
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
};

struct corutv_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t switch_ev = nullptr;  // orders a newly set stream after the previous one
    std::mutex call_mu;
    DeviceBuffer ws;
    int* flags = nullptr;
    Profiler prof;
    // serving
    int max_slots = 8;
    std::vector<ServingSlot> slots;
    std::mutex smu;
    std::condition_variable scv;
    std::deque<PendingReq> queue;
    std::map<uint64_t, ReqResult> results;
    std::thread worker;
    bool stop = false;
    bool worker_started = false;
    uint64_t next_ticket = 1;
    size_t serving_bytes = 0;
    std::vector<cudaEvent_t> ev_pool;  // events for submit-time ordering (under smu)
    void* xhost = nullptr;             // pinned staging of the row-partitioned exchanges
    size_t xcap = 0;
    // CUDA-graph replay of repeated factorisations (corutv_set_graphs)
    bool graphs = false;
    struct GraphEntry {
        int seen = 0;                    // direct runs so far (captured on the second)
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;           // library kernels in the graph
    };
    std::map<std::string, GraphEntry> graph_cache;
    cudaStream_t cap_stream = nullptr;   // captures run here (the caller's stream may be the legacy one)
    cudaStream_t side = nullptr;         // the A_m, A_l cast chunks (CastOverlap)
    cudaEvent_t ov_ev[2 * kMaxCastChunks + 4] = {};  // chunk fork / done, the test matrix's, the outputs'
    BatchState batch;                    // corutv_factor_batch
    int batch_max = 0;                   // serving: largest batch (0: one request per slot)
    std::vector<BatchLane> lanes;        // serving: batch lanes (corutv_set_batching)
};

namespace {

// The arguments of a call as bytes (the key of its captured graph).
struct KeyBytes {
    std::string s;
    template <typename T>
    KeyBytes& add(const T& v) {
        s.append(reinterpret_cast<const char*>(&v), sizeof(T));
        return *this;
    }
};

void drop_graphs(corutv_ctx* ctx) {
    for (auto& kv : ctx->graph_cache)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graph_cache.clear();
}

corutv_status ensure_ws(corutv_ctx* ctx, DeviceBuffer& buf, size_t bytes, cudaStream_t st) {
    if (buf.cap >= bytes) return CORUTV_OK;
    if (bytes > ctx->budget)
        return fail(CORUTV_ENOMEM, "workspace of %zu bytes exceeds the context budget %zu", bytes, ctx->budget);
    if (buf.ptr) {
        CK(cudaStreamSynchronize(st));
        if (&buf == &ctx->ws) drop_graphs(ctx);  // the captured graphs use the old workspace
        CK(cudaFree(buf.ptr));
        buf.ptr = nullptr;
        buf.cap = 0;
    }
    cudaError_t e = cudaMalloc(&buf.ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        buf.ptr = nullptr;
        return fail(CORUTV_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    buf.cap = bytes;
    return CORUTV_OK;
}

// ---------------------------------------------------------------------------
// Grouped execution of a batch of factorisations (corutv_factor_batch):
// Algorithm 1 for every problem of the batch with each step one launch over
// all problems (the grouped kernels), on BF16 sketches of FP32 input as in
// run_factor's split path. The problems run their power rounds aligned at the
// end: sorted by q (largest first), problem i joins at round qmax - q_i, so
// the problems of round r are a prefix of the sorted order and every launch
// of that round covers the first cnt_r records of its array. The records
// (arguments and grids of every launch, tensor maps of the products) are
// built on the host once per batch and copied to the device in one transfer.
// ---------------------------------------------------------------------------

// One array of launch records in the records buffer.
struct RecArr {
    size_t off = 0;
    int count = 0;
    unsigned gx = 0, gy = 0;  // largest grid of the records (kAnyGrid records excluded)
    int max_ell = 0;
    size_t smem = 0;          // grouped products: largest shared memory
    int64_t stride_total = 0; // grid-stride kernels: largest element count
};

struct RecBuilder {
    std::vector<char>& h;
    explicit RecBuilder(std::vector<char>& buf) : h(buf) { h.clear(); }
    size_t reserve(size_t bytes) {
        const size_t off = (h.size() + 127) & ~size_t(127);
        h.resize(off + bytes);
        return off;
    }
    template <class A>
    RecArr add(const std::vector<GroupItem<A>>& items, const std::vector<int>& ells, int64_t stride_total = 0) {
        RecArr r;
        r.count = (int)items.size();
        r.off = reserve(sizeof(GroupItem<A>) * items.size());
        if (!items.empty()) std::memcpy(h.data() + r.off, items.data(), sizeof(GroupItem<A>) * items.size());
        for (size_t i = 0; i < items.size(); ++i) {
            if (items[i].gx != kAnyGrid) r.gx = std::max(r.gx, items[i].gx);
            r.gy = std::max(r.gy, items[i].gy);
            if (i < ells.size()) r.max_ell = std::max(r.max_ell, ells[i]);
        }
        r.stride_total = stride_total;
        return r;
    }
};

// The arrays of one thin QR (orth: CholeskyQR with one or two passes and the
// dependence-check pass) over the problems.
struct OrthRecs {
    int passes = 1;
    RecArr gram[3], chol[3], rinv[3], trsm[3];
    bool qc_bf16[3] = {false, false, false};
};

struct BatchProblem {
    FactorPlan pl;
    FactorBufs b;
    const corutv_request* req;
};

enum OrthKind { ORTH_C1_1 = 0, ORTH_C1_2 = 1, ORTH_C2_1 = 2, ORTH_C2_2 = 3 };

void build_orth(RecBuilder& rb, const std::vector<BatchProblem>& P, OrthKind kind, int* flags, int num_sms,
                OrthRecs& o) {
    const bool c1 = kind == ORTH_C1_1 || kind == ORTH_C1_2;
    o.passes = (kind == ORTH_C1_2 || kind == ORTH_C2_2) ? 2 : 1;
    const double u = 0x1p-24;  // FP32 Grams
    std::vector<int> ells;
    for (auto& pb : P) ells.push_back((int)pb.pl.ell);
    for (int pass = 0; pass < (o.passes == 2 ? 3 : 2); ++pass) {
        std::vector<GroupItem<GramArgs>> g;
        std::vector<GroupItem<CholArgs>> ch;
        std::vector<GroupItem<RinvArgs>> ri;
        std::vector<GroupItem<TrsmArgs>> tr;
        for (auto& pb : P) {
            const FactorPlan& pl = pb.pl;
            const FactorBufs& b = pb.b;
            const int ell = (int)pl.ell, ldri = (ell + 7) & ~7;
            const int64_t ld = c1 ? pl.ldm : pl.ldn, len = c1 ? pl.m : pl.n;
            float* c = static_cast<float*>(c1 ? b.c1 : b.c2);
            float* q = static_cast<float*>(c1 ? b.q1 : (kind == ORTH_C2_1 ? b.x : b.q2));
            void* qc = c1 ? b.q1c : (kind == ORTH_C2_1 ? b.xc : nullptr);
            float* tmp = static_cast<float*>(b.tmp);
            float* p1 = o.passes == 1 ? q : tmp;
            void* p1c = o.passes == 1 ? qc : nullptr;
            float* in = pass == 0 ? c : (pass == 1 ? p1 : tmp);
            float* out = pass == 2 ? q : p1;
            void* outc = pass == 2 ? qc : p1c;
            const int* cancel = pass == 1 ? b.skip : nullptr;  // the dependence-check pass runs only after a shift
            g.push_back(gram_group_item(in, ld, in, ld, len, ell, b.g, reinterpret_cast<float*>(b.gpart), b.gcnt,
                                        cancel, num_sms));
            CholArgs ca{b.g, ell, len, b.r, flags, pass == 0 ? b.skip : nullptr, cancel, u,
                        pass == 1 ? b.defic : nullptr, pass == 1 ? 10.0 * (double)ell * u : 0.0};
            ch.push_back(cholesky_item(ca));
            ri.push_back(rinv_item(RinvArgs{b.r, ell, b.rinv, ldri, cancel}));
            tr.push_back(trsm_item(TrsmArgs{in, ld, len, ell, b.rinv, ldri, out, ld, outc, ld, cancel,
                                            pass == 1 ? b.defic : nullptr}));
            o.qc_bf16[pass] = outc != nullptr;
        }
        o.gram[pass] = rb.add(g, ells);
        o.chol[pass] = rb.add(ch, ells);
        o.rinv[pass] = rb.add(ri, ells);
        o.trsm[pass] = rb.add(tr, ells);
    }
}

// The records of the products (one TcGroupItem each) in the records buffer.
struct ProdRecs {
    RecArr arr;
    int max_grid = 0;
};

corutv_status build_products(RecBuilder& rb, const std::vector<BatchProblem>& P, int which, int* flags,
                             int num_sms, ProdRecs& out) {
    const size_t isz = tc_group_item_bytes();
    out.arr.count = (int)P.size();
    out.arr.off = rb.reserve(isz * P.size());
    for (size_t i = 0; i < P.size(); ++i) {
        const FactorPlan& pl = P[i].pl;
        const FactorBufs& b = P[i].b;
        void* item = rb.h.data() + out.arr.off + i * isz;
        int grid = 0;
        size_t smem = 0;
        int64_t pf = 0;
        cudaError_t e;
        if (which == 0)  // eq. 4: C1 = A X
            e = tc_group_sketch_item(item, b.abf, pl.m, pl.n, 0, b.xc, pl.ldn, pl.ell, pl.ellp, b.part, b.tcnt, b.c1,
                                     T_F32, pl.ldm, num_sms, flags, nullptr, &grid, &smem, &pf);
        else if (which == 1)  // eq. 5: C2 = A^T Q1
            e = tc_group_sketch_item(item, b.abf, pl.m, pl.n, 1, b.q1c, pl.ldm, pl.ell, pl.ellp, b.part, b.tcnt,
                                     b.c2, T_F32, pl.ldn, num_sms, flags, nullptr, &grid, &smem, &pf);
        else  // eq. 7: W = A Q2 from the exact splits
            e = tc_group_project_item(item, b.abf, pl.m, pl.n, b.q2c, pl.ldn, pl.ell, pl.ellp, b.part, b.tcnt, b.w,
                                      T_F32, pl.ldm, num_sms, flags, nullptr, &grid, &smem, &pf);
        if (e != cudaSuccess) return fail(CORUTV_ECUDA, "grouped product record %zu: %s", i, cudaGetErrorString(e));
        if (pf > pl.part_elems) return fail(CORUTV_EINVAL, "grouped product %zu needs more partial storage", i);
        out.max_grid = std::max(out.max_grid, grid);
        out.arr.smem = std::max(out.arr.smem, smem);
    }
    return CORUTV_OK;
}

// Algorithm 1 for the requests of a batch (validated; device pointers) with
// grouped launches on `st`.
corutv_status run_batch(corutv_ctx* ctx, BatchState& bs, const corutv_request* reqs, int count, cudaStream_t st,
                        int* flags) {
    const int num_sms = ctx->num_sms;
    // problems sorted by q, largest first (stable: equal q keep the caller's order)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return reqs[x].opts.q > reqs[y].opts.q; });
    std::vector<BatchProblem> P(count);
    size_t bytes = 0;
    for (int i = 0; i < count; ++i) {
        const corutv_request& r = reqs[order[i]];
        P[i].req = &r;
        CKS(make_plan(P[i].pl, T_F32, r.m, r.n, r.lda, r.opts.k, r.opts.p, r.opts.q, CORUTV_P_BF16, num_sms,
                      reinterpret_cast<uintptr_t>(r.A) % 16 == 0));
        if (!P[i].pl.split) return fail(CORUTV_EINVAL, "batch request %d: the grouped path needs FP32 A", order[i]);
        // the grouped products' own stream-K grids may split a tile into more pieces
        P[i].pl.part_elems = std::max(P[i].pl.part_elems,
                                      tc_group_partial_elems(P[i].pl.m, P[i].pl.n, P[i].pl.ellp, num_sms));
        bytes += factor_bytes(P[i].pl);
    }
    CKS(ensure_ws(ctx, bs.ws, bytes, st));
    Carver cv(bs.ws.ptr);
    for (auto& pb : P) carve_factor(cv, pb.pl, pb.b);
    const int qmax = (int)P[0].pl.q;
    std::vector<int> ells;
    for (auto& pb : P) ells.push_back((int)pb.pl.ell);

    RecBuilder rb(bs.rec);
    // zero: the products' and Grams' counters, the padding columns of Q1's bf16 copy
    std::vector<GroupItem<ZeroArgs>> zi;
    int64_t zmax = 0;
    for (auto& pb : P) {
        const int64_t cb = (int64_t)sizeof(int) * factor_counters(pb.pl);
        const int64_t qb = pb.pl.ellp * pb.pl.ldm * 2;
        zi.push_back(zero_item(pb.b.tcnt, (cb + 3) & ~int64_t(3)));
        zi.push_back(zero_item(pb.b.q1c, qb));
        zmax = std::max(zmax, std::max(cb, qb) / 16);
    }
    const RecArr rz = rb.add(zi, {}, zmax);
    std::vector<GroupItem<GaussArgs>> gi;
    std::vector<GroupItem<CastArgs>> ci;
    std::vector<GroupItem<SplitArgs>> si;
    std::vector<GroupItem<GramArgs>> di;
    std::vector<GroupItem<QrcpArgs>> qi;
    std::vector<GroupItem<ReflArgs>> ui, ur;
    std::vector<GroupItem<GatherArgs>> vi;
    std::vector<GroupItem<EmitArgs>> ei;
    int64_t gmax = 0, smax = 0;
    bool want_u = false, want_v = false;
    for (auto& pb : P) {
        const FactorPlan& pl = pb.pl;
        const FactorBufs& b = pb.b;
        const corutv_request& r = *pb.req;
        const int ell = (int)pl.ell;
        gi.push_back(gaussian_item(GaussArgs{r.opts.seed, r.opts.stream, pl.n, pl.ell, pl.ellp, b.xc, pl.ldn, nullptr}));
        gmax = std::max(gmax, pl.n * pl.ellp);
        ci.push_back(cast3_item(CastArgs{static_cast<const float*>(r.A), pl.m, pl.n, pl.lda, b.abf, nullptr}));
        si.push_back(split_item(SplitArgs{static_cast<const float*>(b.q2), pl.ldn, pl.n, ell, (int)pl.ellp, b.q2c,
                                          pl.ldn, nullptr}));
        smax = std::max(smax, pl.n * pl.ellp);
        di.push_back(gram_group_item(static_cast<const float*>(b.q1), pl.ldm, static_cast<const float*>(b.w), pl.ldm,
                                     pl.m, ell, b.d, reinterpret_cast<float*>(b.gpart), b.gcnt, nullptr, num_sms));
        qi.push_back(qrcp_item(QrcpArgs{b.d, ell, b.refl, b.rt, b.perm, nullptr}));
        if (r.U) want_u = true;
        if (r.V) want_v = true;
        const ReflArgs ra{static_cast<const float*>(b.q1), pl.ldm, r.U ? pl.m : 0, ell, b.refl,
                          static_cast<float*>(r.U), r.ldu, nullptr};
        // U = Q1 Qt from the reflectors: one row per thread up to ell = 64, else the shared-memory form
        ur.push_back(refl_rows_item(ra));
        ui.push_back(refl_item(ra));
        if (ell <= 64) ui.back().gx = 0;
        vi.push_back(gather_item(GatherArgs{static_cast<const float*>(b.q2), pl.ldn, r.V ? pl.n : 0, ell, b.perm,
                                            static_cast<float*>(r.V), r.ldv, nullptr}));
        ei.push_back(emit_item(EmitArgs{b.rt, ell, static_cast<float*>(r.T), b.perm, r.perm, nullptr}));
    }
    const RecArr rg = rb.add(gi, ells, gmax), rc = rb.add(ci, ells), rs = rb.add(si, ells, smax);
    const RecArr rd = rb.add(di, ells), rq = rb.add(qi, ells), ru = rb.add(ui, ells), rur = rb.add(ur, ells);
    const RecArr rvv = rb.add(vi, ells);
    const RecArr re = rb.add(ei, ells, (int64_t)128 * 129);
    ProdRecs pax, paty, pproj;
    CKS(build_products(rb, P, 0, flags, num_sms, pax));
    CKS(build_products(rb, P, 1, flags, num_sms, paty));
    CKS(build_products(rb, P, 2, flags, num_sms, pproj));
    OrthRecs o_c1_1, o_c1_2, o_c2_1, o_c2_2;
    if (qmax > 0) {
        build_orth(rb, P, ORTH_C1_1, flags, num_sms, o_c1_1);
        build_orth(rb, P, ORTH_C2_1, flags, num_sms, o_c2_1);
    }
    build_orth(rb, P, ORTH_C1_2, flags, num_sms, o_c1_2);
    build_orth(rb, P, ORTH_C2_2, flags, num_sms, o_c2_2);

    // the records to the device: pinned staging (reused once its previous copy has run), one copy
    const size_t rbytes = bs.rec.size();
    if (!bs.copied) CK(cudaEventCreateWithFlags(&bs.copied, cudaEventDisableTiming));
    CK(cudaEventSynchronize(bs.copied));
    if (bs.hcap < rbytes) {
        if (bs.host) CK(cudaFreeHost(bs.host));
        bs.host = nullptr;
        bs.hcap = 0;
        CK(cudaMallocHost(reinterpret_cast<void**>(&bs.host), rbytes));
        bs.hcap = rbytes;
    }
    std::memcpy(bs.host, bs.rec.data(), rbytes);
    CKS(ensure_ws(ctx, bs.desc, rbytes, st));
    CK(cudaMemcpyAsync(bs.desc.ptr, bs.host, rbytes, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(bs.copied, st));
    char* dr = static_cast<char*>(bs.desc.ptr);
    auto at = [&](const RecArr& r) { return dr + r.off; };
    auto items = [&](const RecArr& r, auto tag) { return reinterpret_cast<const GroupItem<decltype(tag)>*>(at(r)); };

    // round r covers the problems with q >= qmax - r: a prefix of the sorted order
    auto active = [&](int r) {
        int c = 0;
        while (c < count && P[c].pl.q >= qmax - r) ++c;
        return c;
    };
    auto product = [&](const ProdRecs& pr, int cnt) -> corutv_status {
        CK(launch_sketch_tc_grouped(at(pr.arr), cnt, pr.max_grid, pr.arr.smem, st));
        return CORUTV_OK;
    };
    auto orth = [&](const OrthRecs& o, int cnt) -> corutv_status {
        for (int pass = 0; pass < (o.passes == 2 ? 3 : 2); ++pass) {
            CK(launch_gram_grouped(items(o.gram[pass], GramArgs{}), cnt, o.gram[pass].gx, o.gram[pass].gy, st));
            CK(launch_cholesky_grouped(items(o.chol[pass], CholArgs{}), cnt, o.chol[pass].max_ell, pass == 1, st));
            CK(launch_rinv_grouped(items(o.rinv[pass], RinvArgs{}), cnt, o.rinv[pass].gx, o.rinv[pass].max_ell, st));
            CK(launch_trsm_grouped(items(o.trsm[pass], TrsmArgs{}), cnt, o.trsm[pass].gx, o.trsm[pass].max_ell,
                                   o.qc_bf16[pass], st));
        }
        return CORUTV_OK;
    };
    CK(launch_zero_grouped(items(rz, ZeroArgs{}), rz.count, stride_grid(rz.stride_total), st));
    // Step 1 (Psi as the bf16 operand panel) and the tiled bf16 splits of A
    CK(launch_gaussian_grouped(items(rg, GaussArgs{}), count, stride_grid(rg.stride_total), st));
    CK(launch_cast3_grouped(items(rc, CastArgs{}), count, rc.gx, rc.gy, st));
    for (int r = 0; r <= qmax; ++r) {
        const int cnt = active(r);
        CKS(product(pax, cnt));                                  // eq. 4
        CKS(orth(r < qmax ? o_c1_1 : o_c1_2, cnt));              // Q1 = qr(C1)
        CKS(product(paty, cnt));                                 // eq. 5
        if (r < qmax) CKS(orth(o_c2_1, cnt));                    // X = qr(C2)
    }
    CKS(orth(o_c2_2, count));  // Q2 = qr(C2)
    // eq. 7: W = A Q2 from the exact splits, D = Q1^T W
    CK(launch_split_grouped(items(rs, SplitArgs{}), count, stride_grid(rs.stride_total), st));
    CKS(product(pproj, count));
    CK(launch_gram_grouped(items(rd, GramArgs{}), count, rd.gx, rd.gy, st));
    // eq. 8, then eq. 9: U = Q1 Qt, T = Rt, V = Q2 P
    CK(launch_qrcp_grouped(items(rq, QrcpArgs{}), count, rq.max_ell, st));
    if (want_u && rur.gx) CK(launch_refl_rows_grouped(items(rur, ReflArgs{}), count, rur.gx, st));
    if (want_u && ru.gx) CK(launch_refl_grouped(items(ru, ReflArgs{}), count, ru.gx, ru.max_ell, st));
    if (want_v) CK(launch_gather_grouped(items(rvv, GatherArgs{}), count, rvv.gx, st));
    CK(launch_emit_grouped(items(re, EmitArgs{}), count, stride_grid(re.stride_total), st));
    return CORUTV_OK;
}

// Runs `enqueue(stream)` (all launches of one call, stream-ordered) directly
// on ctx->stream at the first occurrence of `key`, captured into a CUDA graph
// on the second (on a stream of the context's own, as the caller's may be the
// legacy stream, which cannot be captured) and launched on ctx->stream, and
// as that graph's replay afterwards. A capture that fails (an unsupported call
// inside) leaves the key on direct runs.
template <class F>
corutv_status graph_run(corutv_ctx* ctx, const std::string& key, F&& enqueue) {
    auto it = ctx->graph_cache.find(key);
    if (it == ctx->graph_cache.end()) {
        if (ctx->graph_cache.size() >= 16) drop_graphs(ctx);
        it = ctx->graph_cache.emplace(key, corutv_ctx::GraphEntry{}).first;
    }
    corutv_ctx::GraphEntry& g = it->second;
    if (g.exec) {
        CK(cudaGraphLaunch(g.exec, ctx->stream));
        g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
        return CORUTV_OK;
    }
    if (g.seen++ != 1) return enqueue(ctx->stream);  // first occurrence, or a capture that failed before
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    long long kernels = 0;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    t_capture_count = &kernels;
    const corutv_status st = enqueue(ctx->cap_stream);
    t_capture_count = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaErrorUnknown;
    if (st == CORUTV_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != CORUTV_OK) {
        cudaGetLastError();
        return st;
    }
    if (ce != cudaSuccess || ie != cudaSuccess) {
        cudaGetLastError();  // not capturable here: stay on direct runs
        return enqueue(ctx->stream);
    }
    g.exec = exec;
    g.kernels = kernels;
    CK(cudaGraphLaunch(g.exec, ctx->stream));
    g_launches.fetch_add(kernels, std::memory_order_relaxed);
    return CORUTV_OK;
}

corutv_status check_ctx(const corutv_ctx* ctx) {
    if (!ctx) return fail(CORUTV_EINVAL, "null context");
    return CORUTV_OK;
}

corutv_status read_flags(corutv_ctx* ctx, int* hf) {
    CK(cudaMemcpyAsync(hf, ctx->flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CORUTV_OK;
}

corutv_status flags_status(const int* hf) {
    if (hf[FLAG_BREAKDOWN]) return fail(CORUTV_EBREAKDOWN, "Cholesky of a sketch Gram matrix broke down");
    if (hf[FLAG_TIMEOUT]) return fail(CORUTV_ETIMEDOUT, "a bounded device wait gave up");
    return CORUTV_OK;
}

}  // namespace

extern "C" {

corutv_status corutv_create(corutv_ctx** out, int device, size_t mem_budget_bytes, int max_slots) {
    if (!out) return fail(CORUTV_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(CORUTV_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    if (device < 0 || device >= count) return fail(CORUTV_EINVAL, "device %d out of range [0, %d)", device, count);
    DeviceGuard guard(device);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(CORUTV_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a only", device,
                    prop.major, prop.minor);
    auto* ctx = new corutv_ctx();
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * (double)free_b);
    ctx->max_slots = max_slots > 0 ? max_slots : 8;
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return fail(CORUTV_ECUDA, "cudaStreamCreate failed");
    }
    ctx->own_stream = true;
    if (cudaEventCreateWithFlags(&ctx->switch_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return fail(CORUTV_ECUDA, "cudaEventCreate failed");
    }
    if (cudaMalloc(&ctx->flags, sizeof(int) * FLAG_COUNT) != cudaSuccess ||
        cudaMemset(ctx->flags, 0, sizeof(int) * FLAG_COUNT) != cudaSuccess) {
        cudaEventDestroy(ctx->switch_ev);
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return fail(CORUTV_ENOMEM, "cannot allocate the status words");
    }
    *out = ctx;
    return CORUTV_OK;
}

corutv_status corutv_destroy(corutv_ctx* ctx) {
    if (!ctx) return CORUTV_OK;
    DeviceGuard guard(ctx->device);
    if (ctx->worker_started) {
        {
            std::lock_guard<std::mutex> lk(ctx->smu);
            ctx->stop = true;
        }
        ctx->scv.notify_all();
        ctx->worker.join();
    }
    for (auto& pr : ctx->queue)
        if (pr.ready) cudaEventDestroy(pr.ready);
    for (auto& s : ctx->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.ws.ptr) cudaFree(s.ws.ptr);
        if (s.flags) cudaFree(s.flags);
        if (s.hflags) cudaFreeHost(s.hflags);
        if (s.done) cudaEventDestroy(s.done);
        if (s.st) cudaStreamDestroy(s.st);
    }
    for (auto& l : ctx->lanes) {
        if (l.st) cudaStreamSynchronize(l.st);
        if (l.bs.ws.ptr) cudaFree(l.bs.ws.ptr);
        if (l.bs.desc.ptr) cudaFree(l.bs.desc.ptr);
        if (l.bs.host) cudaFreeHost(l.bs.host);
        if (l.bs.copied) cudaEventDestroy(l.bs.copied);
        if (l.flags) cudaFree(l.flags);
        if (l.hflags) cudaFreeHost(l.hflags);
        if (l.done) cudaEventDestroy(l.done);
        if (l.st) cudaStreamDestroy(l.st);
    }
    for (auto ev : ctx->ev_pool) cudaEventDestroy(ev);
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    for (auto ev : ctx->ov_ev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ws.ptr) cudaFree(ctx->ws.ptr);
    if (ctx->batch.ws.ptr) cudaFree(ctx->batch.ws.ptr);
    if (ctx->batch.desc.ptr) cudaFree(ctx->batch.desc.ptr);
    if (ctx->batch.host) cudaFreeHost(ctx->batch.host);
    if (ctx->batch.copied) cudaEventDestroy(ctx->batch.copied);
    if (ctx->flags) cudaFree(ctx->flags);
    if (ctx->switch_ev) cudaEventDestroy(ctx->switch_ev);
    if (ctx->xhost) cudaFreeHost(ctx->xhost);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return CORUTV_OK;
}

const char* corutv_last_error(const corutv_ctx* ctx) {
    (void)ctx;
    return g_last_error.c_str();
}

corutv_status corutv_set_stream(corutv_ctx* ctx, void* cuda_stream) {
    CKS(check_ctx(ctx));
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    cudaStream_t next = static_cast<cudaStream_t>(cuda_stream);
    if (next == ctx->stream) return CORUTV_OK;
    // every call of the context shares its workspace and status words: work
    // enqueued from now on, on the new stream, must not start before the work
    // already queued on the previous stream has finished with them
    CK(cudaEventRecord(ctx->switch_ev, ctx->stream));
    CK(cudaStreamWaitEvent(next, ctx->switch_ev, 0));
    if (ctx->own_stream) {
        // released by the runtime once its queued work has completed
        CK(cudaStreamDestroy(ctx->stream));
        ctx->own_stream = false;
    }
    ctx->stream = next;
    return CORUTV_OK;
}

corutv_status corutv_sync(corutv_ctx* ctx) {
    CKS(check_ctx(ctx));
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    int hf[FLAG_COUNT];
    CKS(read_flags(ctx, hf));
    CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * FLAG_COUNT, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return flags_status(hf);
}

corutv_status corutv_set_graphs(corutv_ctx* ctx, int enable) {
    CKS(check_ctx(ctx));
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    if (!enable) {
        CK(cudaStreamSynchronize(ctx->stream));
        drop_graphs(ctx);
    }
    ctx->graphs = enable != 0;
    return CORUTV_OK;
}

corutv_status corutv_set_autotune(int enable) {
    tc_set_autotune(enable != 0);
    return CORUTV_OK;
}

int corutv_autotune_entry(int index, int64_t* mtot, int64_t* ktot, int* nb, int* trans, int* kgroup, int* stages,
                          float* us) {
    long long mt = 0, kt = 0;
    int b = 0, tr = 0, kg = 0, st = 0;
    float t = 0.f;
    const int count = tc_autotune_entry(index, &mt, &kt, &b, &tr, &kg, &st, &t);
    if (index >= 0 && index < count) {
        if (mtot) *mtot = mt;
        if (ktot) *ktot = kt;
        if (nb) *nb = b;
        if (trans) *trans = tr;
        if (kgroup) *kgroup = kg;
        if (stages) *stages = st;
        if (us) *us = t;
    }
    return count;
}

corutv_status corutv_profile_enable(corutv_ctx* ctx, int enable) {
    CKS(check_ctx(ctx));
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof.collect();
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    return CORUTV_OK;
}

corutv_status corutv_profile_read(corutv_ctx* ctx, int stage, double* total_ms, int64_t* count) {
    CKS(check_ctx(ctx));
    if (stage < CORUTV_STAGE_ALL || stage >= CORUTV_STAGE_COUNT) return fail(CORUTV_EINVAL, "unknown stage %d", stage);
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof.collect();
    if (stage == CORUTV_STAGE_ALL) {
        if (total_ms) *total_ms = 0.0;
        if (count) *count = g_launches.load() - ctx->prof.launch_base;
    } else {
        if (total_ms) *total_ms = ctx->prof.ms[stage];
        if (count) *count = ctx->prof.count[stage];
    }
    return CORUTV_OK;
}

corutv_status corutv_factor(corutv_ctx* ctx, corutv_dtype dtype, const void* A, int64_t m, int64_t n,
                            int64_t lda, const corutv_opts* opts, void* U, int64_t ldu, void* T, void* V,
                            int64_t ldv, int32_t* perm) {
    CKS(check_ctx(ctx));
    if (!A || !opts || !T) return fail(CORUTV_EINVAL, "A, opts and T must not be NULL");
    if (dtype != CORUTV_F64 && dtype != CORUTV_F32) return fail(CORUTV_EINVAL, "unknown dtype %d", (int)dtype);
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    const ElemType ta = dtype == CORUTV_F64 ? T_F64 : T_F32;
    const int es = elem_size(ta);
    const bool dev = is_device_ptr(A);
    if (lda < n) return fail(CORUTV_EINVAL, "lda = %lld < n = %lld", (long long)lda, (long long)n);
    FactorPlan pl;
    if (opts->t_lower > 1) return fail(CORUTV_EINVAL, "t_lower %u is not supported (0 upper T, 1 lower T)", opts->t_lower);
    // host input is staged with row stride n into the (256-byte aligned) workspace
    CKS(make_plan(pl, ta, m, n, dev ? lda : n, opts->k, opts->p, opts->q, (corutv_prec)opts->sketch_prec,
                  ctx->num_sms, !dev || reinterpret_cast<uintptr_t>(A) % 16 == 0, opts->d_mode, opts->t_lower == 1,
                  opts->power_form, opts->bf16_last_round));
    const int64_t ell = pl.ell;
    if (U && ldu < ell) return fail(CORUTV_EINVAL, "ldu < ell");
    if (V && ldv < ell) return fail(CORUTV_EINVAL, "ldv < ell");
    if ((U && is_device_ptr(U) != dev) || is_device_ptr(T) != dev || (V && is_device_ptr(V) != dev) ||
        (perm && is_device_ptr(perm) != dev))
        return fail(CORUTV_EINVAL, "A and the outputs must all be host or all be device memory");
    const bool psi_dev = opts->psi && is_device_ptr(opts->psi);
    // workspace: factor buffers + staging for host calls / host psi
    size_t bytes = factor_bytes(pl);
    Carver extra_measure(nullptr);
    // pinned host A on the bf16 path: the three-part cast reads it in place
    // (one pass over the host copy instead of a copy to the device and a cast)
    const void* a_view = (!dev && pl.split && pl.prec == CORUTV_P_BF16 && !pl.tr) ? pinned_host_view(A) : nullptr;
    if (!dev) {
        if (!a_view) extra_measure.take<char>(m * n * es);
        extra_measure.take<char>(m * ell * es);
        extra_measure.take<char>(n * ell * es);
        extra_measure.take<char>(ell * ell * es);
        extra_measure.take<int>(ell);
    }
    if (opts->psi && !psi_dev) extra_measure.take<double>(pl.n * ell);  // Psi has the rows of pl.n
    CKS(ensure_ws(ctx, ctx->ws, bytes + extra_measure.off, ctx->stream));
    Carver cv(ctx->ws.ptr);
    FactorBufs b;
    carve_factor(cv, pl, b);
    const void* a_dev = A;
    void *u_dev = U, *t_dev = T, *v_dev = V;
    int32_t* perm_dev = perm;
    int64_t ldu_dev = ldu, ldv_dev = ldv;
    if (!dev) {
        void* as = a_view ? nullptr : cv.take<char>(m * n * es);
        u_dev = U ? cv.take<char>(m * ell * es) : nullptr;
        v_dev = V ? cv.take<char>(n * ell * es) : nullptr;
        t_dev = cv.take<char>(ell * ell * es);
        perm_dev = perm ? cv.take<int>(ell) : nullptr;
        if (!U) cv.take<char>(m * ell * es);
        if (!V) cv.take<char>(n * ell * es);
        if (!perm) cv.take<int>(ell);
        if (a_view) {
            a_dev = a_view;
            pl.lda = lda;  // read in place with the caller's row stride
        } else {
            CK(cudaMemcpy2DAsync(as, n * es, A, lda * es, n * es, m, cudaMemcpyHostToDevice, ctx->stream));
            a_dev = as;
            pl.lda = n;
        }
        ldu_dev = ell;
        ldv_dev = ell;
    }
    const double* psi = nullptr;
    if (opts->psi) {
        if (psi_dev) {
            psi = opts->psi;
        } else {
            double* ps = cv.take<double>(pl.n * ell);
            CK(cudaMemcpyAsync(ps, opts->psi, sizeof(double) * pl.n * ell, cudaMemcpyHostToDevice, ctx->stream));
            psi = ps;
        }
    }
    // A_m, A_l of the projection cast beside the thin QRs (device input, bf16 sketches)
    CastOverlap ov;
    // (host input: its staged copy; not for A read in place from host memory, cast whole in one pass)
    const bool overlap = pl.split && (pl.prec == CORUTV_P_BF16 || pl.prec == CORUTV_P_TF32) && !a_view;
    if (overlap && !ctx->side) {
        CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        for (auto& ev : ctx->ov_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    auto enqueue = [&](cudaStream_t st) -> corutv_status {
        Exec ex{st, ctx->flags, nullptr, ctx->num_sms, &ctx->prof};
        if (overlap) {
            ov = CastOverlap();
            ov.side = ctx->side;
            ov.ev = ctx->ov_ev;
            ov.psi_fork = ctx->ov_ev[2 * kMaxCastChunks];
            ov.psi_done = ctx->ov_ev[2 * kMaxCastChunks + 1];
            ov.emit_fork = ctx->ov_ev[2 * kMaxCastChunks + 2];
            ov.emit_done = ctx->ov_ev[2 * kMaxCastChunks + 3];
            ex.ov = &ov;
        }
        CKS(run_factor(ex, pl, b, a_dev, psi, opts->seed, opts->stream));
        return emit_user(ex, pl, b, ta, u_dev, ldu_dev, t_dev, v_dev, ldv_dev, perm_dev);
    };
    if (dev && ctx->graphs && !ctx->prof.on) {
        KeyBytes key;
        key.add(dtype).add(A).add(m).add(n).add(lda).add(opts->k).add(opts->p).add(opts->q);
        key.add(opts->sketch_prec).add(opts->d_mode).add(opts->seed).add(opts->stream).add(opts->t_lower);
        key.add(opts->psi).add(opts->power_form).add(opts->bf16_last_round);
        key.add(U).add(ldu).add(T).add(V).add(ldv).add(perm).add(ctx->ws.ptr).add(ctx->stream);
        return graph_run(ctx, key.s, enqueue);
    }
    CKS(enqueue(ctx->stream));
    if (!dev) {
        if (U) CK(cudaMemcpy2DAsync(U, ldu * es, u_dev, ell * es, ell * es, m, cudaMemcpyDeviceToHost, ctx->stream));
        if (V) CK(cudaMemcpy2DAsync(V, ldv * es, v_dev, ell * es, ell * es, n, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(T, t_dev, ell * ell * es, cudaMemcpyDeviceToHost, ctx->stream));
        if (perm) CK(cudaMemcpyAsync(perm, perm_dev, sizeof(int32_t) * ell, cudaMemcpyDeviceToHost, ctx->stream));
        int hf[FLAG_COUNT];
        CKS(read_flags(ctx, hf));
        CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * FLAG_COUNT, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return flags_status(hf);
    }
    CK(cudaGetLastError());
    return CORUTV_OK;
}

corutv_status corutv_factor_rows(corutv_ctx* ctx, corutv_dtype dtype, const void* A, int64_t m_local, int64_t n,
                                 int64_t lda, int64_t m_total, const corutv_opts* opts, corutv_allreduce_fn allreduce,
                                 void* user, void* U, int64_t ldu, void* T, void* V, int64_t ldv, int32_t* perm) {
    CKS(check_ctx(ctx));
    if (!A || !opts || !T || !allreduce) return fail(CORUTV_EINVAL, "A, opts, T and allreduce must not be NULL");
    if (dtype != CORUTV_F64 && dtype != CORUTV_F32) return fail(CORUTV_EINVAL, "unknown dtype %d", (int)dtype);
    if (opts->d_mode != 0 || opts->t_lower != 0 || opts->power_form != 0 || opts->psi)
        return fail(CORUTV_EINVAL, "the row-partitioned form takes d_mode 0, t_lower 0, power_form 0 and a seeded Psi");
    if (m_total < m_local || m_local < 1) return fail(CORUTV_EINVAL, "need 1 <= m_local <= m_total");
    if (opts->k + opts->p >= std::min(m_total, n))
        return fail(CORUTV_EINVAL, "ell = k + p must be < min(m_total, n)");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    if (!is_device_ptr(A) || !is_device_ptr(T) || (U && !is_device_ptr(U)) || (V && !is_device_ptr(V)) ||
        (perm && !is_device_ptr(perm)))
        return fail(CORUTV_EINVAL, "corutv_factor_rows takes device pointers only");
    const ElemType ta = dtype == CORUTV_F64 ? T_F64 : T_F32;
    FactorPlan pl;
    // the local block must itself be taller than ell (its thin QR panels hold m_local rows)
    CKS(make_plan(pl, ta, m_local, n, lda, opts->k, opts->p, opts->q, (corutv_prec)opts->sketch_prec, ctx->num_sms,
                  reinterpret_cast<uintptr_t>(A) % 16 == 0, 0, false, 0, opts->bf16_last_round));
    const int64_t ell = pl.ell;
    if ((U && ldu < ell) || (V && ldv < ell)) return fail(CORUTV_EINVAL, "ldu, ldv must be >= ell");
    CKS(ensure_ws(ctx, ctx->ws, factor_bytes(pl), ctx->stream));
    const size_t xbytes = sizeof(double) * (size_t)std::max(ell * ell, ell * pl.ldn);
    if (ctx->xcap < xbytes) {
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->xhost) CK(cudaFreeHost(ctx->xhost));
        ctx->xhost = nullptr;
        ctx->xcap = 0;
        CK(cudaMallocHost(&ctx->xhost, xbytes));
        ctx->xcap = xbytes;
    }
    Carver cv(ctx->ws.ptr);
    FactorBufs b;
    carve_factor(cv, pl, b);
    Exchange xch{allreduce, user, ctx->xhost, m_total};
    Exec ex{ctx->stream, ctx->flags, nullptr, ctx->num_sms, &ctx->prof, &xch};
    CKS(run_factor(ex, pl, b, A, nullptr, opts->seed, opts->stream));
    CKS(emit_user(ex, pl, b, ta, U, ldu, T, V, ldv, perm));
    CK(cudaGetLastError());
    return CORUTV_OK;
}

// ---------------------------------------------------------------------------
// Single steps.
// ---------------------------------------------------------------------------
corutv_status corutv_factor_batch(corutv_ctx* ctx, const corutv_request* reqs, int count) {
    CKS(check_ctx(ctx));
    if (!reqs || count < 1 || count > 4096) return fail(CORUTV_EINVAL, "need 1 <= count <= 4096 requests");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    for (int i = 0; i < count; ++i) {
        const corutv_request& r = reqs[i];
        const corutv_opts& o = r.opts;
        if (r.dtype != CORUTV_F32 || o.sketch_prec != CORUTV_P_BF16)
            return fail(CORUTV_EINVAL, "batch request %d: the grouped path takes FP32 A and BF16 sketches", i);
        if (o.d_mode != 0 || o.t_lower != 0 || o.power_form != 0 || o.bf16_last_round != 0 || o.psi)
            return fail(CORUTV_EINVAL,
                        "batch request %d: the grouped path takes d_mode 0, t_lower 0, power_form 0, "
                        "bf16_last_round 0 and a seeded Psi", i);
        if (!r.A || !r.T) return fail(CORUTV_EINVAL, "batch request %d: A and T must not be NULL", i);
        if (!is_device_ptr(r.A) || !is_device_ptr(r.T) || (r.U && !is_device_ptr(r.U)) ||
            (r.V && !is_device_ptr(r.V)) || (r.perm && !is_device_ptr(r.perm)))
            return fail(CORUTV_EINVAL, "batch request %d: corutv_factor_batch takes device pointers only", i);
        if (o.k < 1 || o.p < 0 || o.q < 0 || o.k + o.p > 128 || o.k + o.p >= std::min(r.m, r.n) || r.lda < r.n)
            return fail(CORUTV_EINVAL, "batch request %d: need 1 <= k, ell = k + p <= 128, ell < min(m, n), lda >= n",
                        i);
        if ((r.U && r.ldu < o.k + o.p) || (r.V && r.ldv < o.k + o.p))
            return fail(CORUTV_EINVAL, "batch request %d: ldu, ldv must be >= ell", i);
    }
    CKS(run_batch(ctx, ctx->batch, reqs, count, ctx->stream, ctx->flags));
    CK(cudaGetLastError());
    return CORUTV_OK;
}

corutv_status corutv_gaussian(corutv_ctx* ctx, uint64_t seed, uint32_t stream, int64_t n, int64_t ell,
                              double* psi, int64_t ldpsi) {
    CKS(check_ctx(ctx));
    if (!psi || n < 1 || ell < 1 || ldpsi < ell) return fail(CORUTV_EINVAL, "bad gaussian arguments");
    if (!is_device_ptr(psi)) return fail(CORUTV_EINVAL, "psi must be device memory");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    CK(launch_gaussian_rowmajor(seed, stream, n, ell, psi, ldpsi, ctx->stream));
    return CORUTV_OK;
}

corutv_status corutv_sketch(corutv_ctx* ctx, corutv_dtype dtype, corutv_prec prec, int trans, const void* A,
                            int64_t m, int64_t n, int64_t lda, const double* X, int64_t ldx, int64_t ell,
                            double* C, int64_t ldc) {
    CKS(check_ctx(ctx));
    if (!A || !X || !C) return fail(CORUTV_EINVAL, "null pointer");
    if (!is_device_ptr(A) || !is_device_ptr(X) || !is_device_ptr(C))
        return fail(CORUTV_EINVAL, "corutv_sketch takes device pointers only");
    const int64_t xrows = trans ? m : n, crows = trans ? n : m;
    const bool tc_prec = prec == CORUTV_P_TF32 || prec == CORUTV_P_BF16 || (int)prec == CORUTV_P_BF16X3;
    if (ell < 1 || ell > (tc_prec ? 128 : kMaxEllSimt) || ldx < ell || ldc < ell || lda < n || m < 1 || n < 1)
        return fail(CORUTV_EINVAL, "bad sketch sizes");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    const ElemType ta = dtype == CORUTV_F64 ? T_F64 : T_F32;
    if ((int)prec == CORUTV_P_BF16X3) {
        // FP32-accurate A X from exact bf16 splits (tensor cores)
        if (ta != T_F32 || trans) return fail(CORUTV_EINVAL, "BF16X3 needs FP32 A and trans = 0");
        const int64_t ellp = round_up(ell, 16), ldn = round_up(n, 64), ldm = round_up(m, 64);
        const int64_t part_elems = tc_partial_elems(m, n, ellp, ldm, ldn, ctx->num_sms);
        Carver measure(nullptr);
        measure.take<float>(ellp * ldn);
        measure.take<char>(3 * ellp * ldn * 2);
        measure.take<double>(ellp * ldm);
        measure.take<float>(part_elems);
        measure.take<char>(3 * tiled_part_bytes(m, n));
        measure.take<int>(tc_counter_elems(m, n));
        CKS(ensure_ws(ctx, ctx->ws, measure.off, ctx->stream));
        Carver cv(ctx->ws.ptr);
        float* xp = cv.take<float>(ellp * ldn);
        void* x3 = cv.take<char>(3 * ellp * ldn * 2);
        double* cp = cv.take<double>(ellp * ldm);
        void* part = cv.take<float>(part_elems);
        void* a3 = cv.take<char>(3 * tiled_part_bytes(m, n));
        int* tcnt = cv.take<int>(tc_counter_elems(m, n));
        CK(cudaMemsetAsync(tcnt, 0, sizeof(int) * (size_t)tc_counter_elems(m, n), ctx->stream));
        CK(launch_rowmajor_to_panel(X, ldx, n, ell, ellp, xp, T_F32, ldn, ctx->stream));
        CK(launch_split_panel(xp, ldn, n, ell, ellp, x3, ldn, nullptr, ctx->stream));
        CK(launch_cast_tiled(A, T_F32, m, n, lda, a3, 3, nullptr, ctx->stream));
        CK(launch_project_split_tc_tiled(a3, m, n, x3, ldn, ell, ellp, part, tcnt, cp, T_F64, ldm, ctx->num_sms,
                                         ctx->flags, nullptr, ctx->stream));
        CK(launch_panel_to_rowmajor(cp, ldm, m, ell, C, T_F64, ldc, nullptr, ctx->stream));
        return CORUTV_OK;
    }
    FactorPlan pl;
    // plan with k = ell, p = 0, q = 0; sizes m, n need ell < min(m, n) only for the full pipeline
    pl.m = m; pl.n = n; pl.lda = lda; pl.k = ell; pl.p = 0; pl.q = 0; pl.ell = ell; pl.ta = ta; pl.prec = prec;
    pl.num_sms = ctx->num_sms;
    pl.tensor = (prec == CORUTV_P_TF32 || prec == CORUTV_P_BF16);
    if (prec == CORUTV_P_TF32 && ta != T_F32) return fail(CORUTV_EINVAL, "TF32 needs FP32 input");
    pl.ellp = pl.tensor ? round_up(ell, 16) : ell;
    pl.ldm = round_up(m, 64);
    pl.ldn = round_up(n, 64);
    pl.tr = false;
    pl.ma = m; pl.na = n; pl.ldma = pl.ldm; pl.ldna = pl.ldn;
    pl.tcomp = pl.tensor ? (prec == CORUTV_P_BF16 ? T_BF16 : T_F32) : (prec == CORUTV_P_F64 ? T_F64 : T_F32);
    pl.tdproj = pl.tcomp;
    pl.tp = T_F64;
    pl.sp_ax = gemm_simt_splits(m, n, ctx->num_sms);
    pl.sp_aty = gemm_simt_splits(n, m, ctx->num_sms);
    pl.gs_m = pl.gs_n = 1;
    pl.part_elems = std::max((int64_t)pl.sp_ax * pl.ellp * pl.ldm, (int64_t)pl.sp_aty * pl.ellp * pl.ldn);
    if (pl.tensor) pl.part_elems = std::max(pl.part_elems, tc_partial_elems(m, n, pl.ellp, pl.ldm, pl.ldn, ctx->num_sms));
    const int64_t ldxp = trans ? pl.ldm : pl.ldn, ldcp = trans ? pl.ldn : pl.ldm;
    Carver measure(nullptr);
    measure.take<double>(pl.ellp * ldxp);
    measure.take<char>(pl.ellp * ldxp * 8);
    measure.take<double>(pl.ellp * ldcp);
    measure.take<char>(pl.part_elems * 8);
    if (prec == CORUTV_P_BF16) measure.take<char>(tiled_part_bytes(m, n));
    // TF32 A^T X runs as (A^T) X on a transposed copy: both operands K-major
    const bool tf32_t = prec == CORUTV_P_TF32 && trans;
    const bool tf32_copy = prec == CORUTV_P_TF32 && !trans && !tma_rows_aligned(A, lda, 4);
    if (tf32_copy) measure.take<float>(m * round_up(n, 4));
    if (tf32_t) measure.take<float>(n * pl.ldm);
    if (pl.tensor) measure.take<int>(tc_counter_elems(m, n));
    CKS(ensure_ws(ctx, ctx->ws, measure.off, ctx->stream));
    Carver cv(ctx->ws.ptr);
    double* xp = cv.take<double>(pl.ellp * ldxp);
    void* xc = cv.take<char>(pl.ellp * ldxp * 8);
    double* cp = cv.take<double>(pl.ellp * ldcp);
    FactorBufs b{};
    b.part = cv.take<char>(pl.part_elems * 8);
    b.abf = prec == CORUTV_P_BF16 ? cv.take<char>(tiled_part_bytes(m, n)) : nullptr;
    float* a32 = tf32_copy ? cv.take<float>(m * round_up(n, 4)) : nullptr;
    float* at = tf32_t ? cv.take<float>(n * pl.ldm) : nullptr;
    b.tcnt = pl.tensor ? cv.take<int>(tc_counter_elems(m, n)) : nullptr;
    if (pl.tensor) CK(cudaMemsetAsync(b.tcnt, 0, sizeof(int) * (size_t)tc_counter_elems(m, n), ctx->stream));
    CK(launch_rowmajor_to_panel(X, ldx, xrows, ell, pl.ellp, xp, T_F64, ldxp, ctx->stream));
    CK(launch_panel_convert(xp, T_F64, ldxp, xrows, pl.ellp, xc, pl.tcomp, ldxp, nullptr, ctx->stream));
    Exec ex{ctx->stream, ctx->flags, nullptr, ctx->num_sms};
    if (pl.tensor) {
        const void* aop = A;
        int64_t lda_op = lda;
        if (prec == CORUTV_P_BF16) {
            CK(launch_cast_tiled(A, ta, m, n, lda, b.abf, 1, nullptr, ctx->stream));
            aop = b.abf;
        } else if (tf32_copy) {
            CK(launch_copy_f32_padded(static_cast<const float*>(A), m, n, lda, a32, round_up(n, 4), ctx->stream));
            aop = a32;
            lda_op = round_up(n, 4);
        }
        if (tf32_t) {
            CK(launch_prep_f32(static_cast<const float*>(A), m, n, lda, at, pl.ldm, nullptr, nullptr, 0, nullptr,
                               ctx->stream));
            CK(launch_sketch_tc(at, T_F32, n, m, pl.ldm, 0, xc, ldxp, ell, pl.ellp, b.part, b.tcnt, cp, T_F64, ldcp,
                                ctx->num_sms, ctx->flags, nullptr, ctx->stream));
        } else if (prec == CORUTV_P_BF16) {
            CK(launch_sketch_tc_tiled(aop, m, n, trans, xc, ldxp, ell, pl.ellp, b.part, b.tcnt, cp, T_F64, ldcp,
                                      ctx->num_sms, ctx->flags, nullptr, ctx->stream));
        } else {
            CK(launch_sketch_tc(aop, pl.tcomp, m, n, lda_op, trans, xc, ldxp, ell, pl.ellp, b.part, b.tcnt, cp, T_F64,
                                ldcp, ctx->num_sms, ctx->flags, nullptr, ctx->stream));
        }
    } else {
        CKS(sketch_simt(ex, pl, b, trans ? A_COLS : A_ROWS, A, ta, xc, pl.tcomp, cp, ldcp));
    }
    CK(launch_panel_to_rowmajor(cp, ldcp, crows, ell, C, T_F64, ldc, nullptr, ctx->stream));
    return CORUTV_OK;
}

corutv_status corutv_orth(corutv_ctx* ctx, const double* C, int64_t rows, int64_t ell, int64_t ldc, double* Q,
                          int64_t ldq, double* R) {
    CKS(check_ctx(ctx));
    if (!C || !Q) return fail(CORUTV_EINVAL, "null pointer");
    if (!is_device_ptr(C) || !is_device_ptr(Q) || (R && !is_device_ptr(R)))
        return fail(CORUTV_EINVAL, "corutv_orth takes device pointers only");
    if (ell < 1 || ell > kMaxEllSimt || rows < ell || ldc < ell || ldq < ell) return fail(CORUTV_EINVAL, "bad orth sizes");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    FactorPlan pl{};
    pl.ell = ell; pl.ellp = ell; pl.m = rows; pl.ldm = round_up(rows, 64);
    pl.gs_m = gemm_simt_splits(ell, rows, ctx->num_sms);
    pl.gs_n = pl.gs_m;
    const int64_t pm = ell * pl.ldm;
    Carver measure(nullptr);
    measure.take<double>(pm);
    measure.take<double>(pm);
    measure.take<double>(pm);
    measure.take<double>((int64_t)pl.gs_m * ell * ell);
    measure.take<double>(ell * ell);
    measure.take<double>(ell * ell);
    measure.take<int>(8);
    measure.take<double>(trsm_rinv_floats(ell));
    CKS(ensure_ws(ctx, ctx->ws, measure.off, ctx->stream));
    Carver cv(ctx->ws.ptr);
    double* cp = cv.take<double>(pm);
    double* qp = cv.take<double>(pm);
    FactorBufs b{};
    b.tmp = cv.take<double>(pm);
    b.gpart = cv.take<double>((int64_t)pl.gs_m * ell * ell);
    b.g = cv.take<double>(ell * ell);
    b.r = cv.take<double>(ell * ell);
    b.skip = cv.take<int>(8);
    b.rinv = reinterpret_cast<float*>(cv.take<double>(trsm_rinv_floats(ell)));  // wide panels only
    CK(launch_rowmajor_to_panel(C, ldc, rows, ell, ell, cp, T_F64, pl.ldm, ctx->stream));
    Exec ex{ctx->stream, ctx->flags, nullptr, ctx->num_sms};
    pl.torth = T_F64;
    pl.tp = T_F64;
    CKS(orth(ex, pl, b, cp, pl.ldm, rows, qp, nullptr, T_F64, 2));
    CK(launch_panel_to_rowmajor(qp, pl.ldm, rows, ell, Q, T_F64, ldq, nullptr, ctx->stream));
    if (R) {
        // R of C = Q R: R = Q^T C (exact in exact arithmetic; upper triangular)
        CKS(gram(ex, pl, b, qp, pl.ldm, cp, pl.ldm, rows, b.g, nullptr, T_F64));
        CK(cudaMemcpyAsync(R, b.g, sizeof(double) * ell * ell, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return CORUTV_OK;
}

corutv_status corutv_selftest_wait(corutv_ctx* ctx, int64_t limit_ns) {
    CKS(check_ctx(ctx));
    if (limit_ns < 0 || limit_ns > 10000000000LL) return fail(CORUTV_EINVAL, "limit_ns must be in [0, 1e10]");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    CK(launch_wait_probe(ctx->flags, (unsigned long long)limit_ns, ctx->stream));
    return CORUTV_OK;
}

corutv_status corutv_qrcp(corutv_ctx* ctx, const double* D, int64_t ell, double* Qt, double* Rt, int32_t* perm) {
    CKS(check_ctx(ctx));
    if (!D || !Qt || !Rt || !perm) return fail(CORUTV_EINVAL, "null pointer");
    if (!is_device_ptr(D) || !is_device_ptr(Qt) || !is_device_ptr(Rt) || !is_device_ptr(perm))
        return fail(CORUTV_EINVAL, "corutv_qrcp takes device pointers only");
    if (ell < 1 || ell > kMaxEllSimt) return fail(CORUTV_EINVAL, "ell must be in [1, %d]", kMaxEllSimt);
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    const size_t work_bytes = sizeof(double) * (size_t)(ell * (ell + 2));
    CKS(ensure_ws(ctx, ctx->ws, work_bytes, ctx->stream));
    CK(launch_qrcp(D, ell, Qt, Rt, perm, static_cast<double*>(ctx->ws.ptr), nullptr, ctx->stream));
    return CORUTV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ALM-CoRUTV
// ---------------------------------------------------------------------------
namespace {

corutv_status normest(corutv_ctx* ctx, const FactorPlan& pl, const FactorBufs& b, const void* mat,
                      ElemType tm, int64_t ldm_user, double* out_norm2) {
    const int64_t m = pl.m, n = pl.n;
    // FP64 vectors carved from the panel buffers (each holds at least ell >= 2
    // panel columns, i.e. >= 2 x rows x 4 bytes)
    double* v = static_cast<double*>(b.x);    // n
    double* u = static_cast<double*>(b.c1);   // m
    double* w = static_cast<double*>(b.c2);   // n
    double* lam = b.g;                        // scalar
    CK(launch_vec_fill(v, n, 1.0 / std::sqrt((double)n), ctx->stream));
    // M^T u as row-chunk partials (added in chunk order) that fit the partial buffer
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)32, pl.part_elems / pl.ldn, m}));
    for (int it = 0; it < 50; ++it) {
        CK(launch_gemv_rows(mat, tm, ldm_user, m, n, v, u, ctx->stream));
        CK(launch_gemv_cols_partial(mat, tm, ldm_user, m, n, u, static_cast<double*>(b.part), pl.ldn, chunks,
                                    ctx->stream));
        CK(launch_reduce_splits(b.part, T_F64, chunks, pl.ldn, w, T_F64, pl.ldn, n, 1, pl.ldn, nullptr, ctx->stream));
        CK(launch_vec_normalize(w, v, n, lam, ctx->stream));
    }
    double h = 0.0;
    CK(cudaMemcpyAsync(&h, lam, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out_norm2 = std::sqrt(h);
    return CORUTV_OK;
}

}  // namespace

extern "C" corutv_status corutv_rpca(corutv_ctx* ctx, corutv_dtype dtype, const void* M, int64_t m, int64_t n,
                                     int64_t ldm, const corutv_opts* opts, double lambda, double mu0,
                                     double mu_bar, double rho, double tol, int max_iter, void* L, void* S,
                                     int* iters, double* zeta, int* rank) {
    CKS(check_ctx(ctx));
    if (!M || !opts || !L || !S) return fail(CORUTV_EINVAL, "M, opts, L and S must not be NULL");
    if (dtype != CORUTV_F64 && dtype != CORUTV_F32) return fail(CORUTV_EINVAL, "unknown dtype");
    const int64_t k = opts->k;
    if (k < 1 || 2 * k > kMaxEllSimt)
        return fail(CORUTV_EINVAL, "rank guess k must be in [1, %d] (ell = 2k <= %d)", kMaxEllSimt / 2, kMaxEllSimt);
    if (ldm < n) return fail(CORUTV_EINVAL, "ldm < n");
    const bool dev = is_device_ptr(M);
    if (is_device_ptr(L) != dev || is_device_ptr(S) != dev)
        return fail(CORUTV_EINVAL, "M, L and S must all be host or all be device memory");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DeviceGuard guard(ctx->device);
    const ElemType tm = dtype == CORUTV_F64 ? T_F64 : T_F32;
    const int es = elem_size(tm);
    corutv_prec prec = (corutv_prec)opts->sketch_prec;
    if (prec != CORUTV_P_F64 && prec != CORUTV_P_F32 && prec != CORUTV_P_TF32 && prec != CORUTV_P_BF16)
        return fail(CORUTV_EINVAL, "unknown sketch precision");
    if (max_iter <= 0) max_iter = 100;
    if (tol <= 0) tol = 1e-5;
    if (rho <= 0) rho = 1.6;
    if (lambda <= 0) lambda = 1.0 / std::sqrt((double)std::max(m, n));
    FactorPlan pl;
    CKS(make_plan(pl, tm, m, n, n, k, k, 1, prec, ctx->num_sms, true, 0, false, opts->power_form,
                  opts->bf16_last_round));
    const int64_t mn = m * n;
    const int nup = rpca_update_blocks(m, n);
    size_t bytes = factor_bytes(pl);
    Carver measure(nullptr);
    measure.take<char>(mn * es);  // Y
    measure.take<char>(mn * es);  // B
    measure.take<double>(std::max(nup, 1184));  // residual partials
    measure.take<double>(1184);  // ||M||_F partials
    measure.take<double>(max_iter);
    measure.take<int>(4);
    if (!dev) {
        measure.take<char>(mn * es);  // M
        measure.take<char>(mn * es);  // L
        measure.take<char>(mn * es);  // S
    }
    CKS(ensure_ws(ctx, ctx->ws, bytes + measure.off, ctx->stream));
    Carver cv(ctx->ws.ptr);
    FactorBufs b;
    carve_factor(cv, pl, b);
    void* y = cv.take<char>(mn * es);
    void* bmat = cv.take<char>(mn * es);
    double* res_part = cv.take<double>(std::max(nup, 1184));
    double* fro_part = cv.take<double>(1184);
    double* zhist = cv.take<double>(max_iter);
    int* rank_dev = cv.take<int>(4);
    const void* m_dev = M;
    int64_t ldm_dev = ldm;
    void *l_dev = L, *s_dev = S;
    if (!dev) {
        void* ms = cv.take<char>(mn * es);
        l_dev = cv.take<char>(mn * es);
        s_dev = cv.take<char>(mn * es);
        CK(cudaMemcpy2DAsync(ms, n * es, M, ldm * es, n * es, m, cudaMemcpyHostToDevice, ctx->stream));
        m_dev = ms;
        ldm_dev = n;
    }
    CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * FLAG_COUNT, ctx->stream));
    CK(cudaMemsetAsync(rank_dev, 0, sizeof(int) * 4, ctx->stream));
    int nfro = 0;
    CK(launch_rpca_init(m_dev, tm, ldm_dev, m, n, static_cast<float*>(s_dev), static_cast<float*>(y),
                        static_cast<float*>(bmat), static_cast<double*>(s_dev), static_cast<double*>(y),
                        static_cast<double*>(bmat), fro_part, &nfro, ctx->stream));
    if (mu0 <= 0) {
        double nrm = 0.0;
        CKS(normest(ctx, pl, b, m_dev, tm, ldm_dev, &nrm));
        if (!(nrm > 0)) return fail(CORUTV_EINVAL, "M has zero spectral norm");
        mu0 = 1.25 / nrm;
    }
    if (mu_bar <= 0) mu_bar = 1e7 * mu0;
    std::vector<double> mus(max_iter + 1);
    mus[0] = mu0;
    for (int j = 1; j <= max_iter; ++j) mus[j] = std::min(rho * mus[j - 1], mu_bar);
    const int* done = ctx->flags + FLAG_RPCA_DONE;
    Exec ex{ctx->stream, ctx->flags, done, ctx->num_sms, &ctx->prof};
    for (int j = 0; j < max_iter; ++j) {
        // L_{j+1} = C_{1/mu_j}(B_j): CoR-UTV of B_j with ell = 2k, q = 1, fresh Psi
        CKS(run_factor(ex, pl, b, bmat, nullptr, opts->seed, opts->stream + (uint32_t)j + 1u));
        // U = Q1 Qt (FP64 panel) from the QRCP's reflectors
        if (pl.ell > 128) {
            // wide sketches: U = Q1 Qt as an FP64 product with the explicit Qt
            GemmArgs g{A_PANEL, B_SMALL, O_PANEL, pl.tp, T_F64, b.q1, pl.ldm, b.qt, pl.ell, b.upanel, pl.ldm, 0,
                       m, pl.ell, pl.ell, 1, done, T_F64};
            CK(launch_gemm_simt(g, ctx->stream));
        } else {
            CK(launch_apply_reflectors(b.q1, pl.tp, pl.ldm, m, pl.ell, b.refl, b.upanel, T_F64, pl.ldm, true, done,
                                       ctx->stream));
        }
        CK(launch_rpca_rank_z(b.rt, b.q2, pl.tp, pl.ldn, b.perm, n, pl.ell, 1.0 / mus[j], rank_dev, b.zpanel,
                              pl.ldn, done, ctx->stream));
        RpcaIterArgs ua{m_dev, tm, ldm_dev, m, n,
                        static_cast<float*>(s_dev), static_cast<float*>(y), static_cast<float*>(bmat),
                        static_cast<double*>(s_dev), static_cast<double*>(y), static_cast<double*>(bmat),
                        b.upanel, pl.ldm, b.zpanel, pl.ldn, pl.ell, rank_dev, mus[j], mus[j + 1], lambda,
                        res_part, done};
        int nparts = 0;
        CK(launch_rpca_update(ua, &nparts, ctx->stream));
        CK(launch_rpca_finish_iter(res_part, nparts, fro_part, nfro, tol, j, zhist, ctx->flags, rank_dev,
                                   ctx->stream));
    }
    CK(launch_rpca_reconstruct(b.upanel, pl.ldm, b.zpanel, pl.ldn, rank_dev, pl.ell, m, n, l_dev, tm, n,
                               ctx->stream));
    int hf[FLAG_COUNT];
    CKS(read_flags(ctx, hf));
    const int it_done = hf[FLAG_RPCA_ITERS];
    double z_last = 0.0;
    if (it_done > 0)
        CK(cudaMemcpyAsync(&z_last, zhist + (it_done - 1), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (!dev) {
        CK(cudaMemcpyAsync(L, l_dev, mn * es, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(S, s_dev, mn * es, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * FLAG_COUNT, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (iters) *iters = it_done;
    if (zeta) *zeta = z_last;
    if (rank) *rank = hf[FLAG_RPCA_RANK];
    CKS(flags_status(hf));
    if (!hf[FLAG_RPCA_DONE]) return fail(CORUTV_ENOTCONV, "ALM-CoRUTV reached max_iter=%d with zeta=%.3e", max_iter, z_last);
    return CORUTV_OK;
}

// ---------------------------------------------------------------------------
// Serving: a dispatcher thread admits queued requests into slots (each with
// its own stream, workspace and status words) as slots and memory free up;
// admitted requests run concurrently on the device.
// ---------------------------------------------------------------------------
namespace {

size_t request_bytes(const corutv_request& r, bool host, int num_sms, FactorPlan* plan_out, corutv_status* st) {
    FactorPlan pl;
    const ElemType ta = r.dtype == CORUTV_F64 ? T_F64 : T_F32;
    if (r.opts.t_lower > 1) {
        *st = fail(CORUTV_EINVAL, "t_lower %u is not supported (0 upper T, 1 lower T)", r.opts.t_lower);
        return 0;
    }
    *st = make_plan(pl, ta, r.m, r.n, host ? r.n : r.lda, r.opts.k, r.opts.p, r.opts.q,
                    (corutv_prec)r.opts.sketch_prec, num_sms, host || reinterpret_cast<uintptr_t>(r.A) % 16 == 0,
                    r.opts.d_mode, r.opts.t_lower == 1, r.opts.power_form, r.opts.bf16_last_round);
    if (*st != CORUTV_OK) return 0;
    size_t bytes = factor_bytes(pl);
    const int es = elem_size(ta);
    const int64_t ell = pl.ell;
    if (host) {
        Carver c(nullptr);
        c.take<char>(r.m * r.n * es);
        c.take<char>(r.m * ell * es);
        c.take<char>(r.n * ell * es);
        c.take<char>(ell * ell * es);
        c.take<int>(ell);
        bytes += c.off;
    }
    if (r.opts.psi) bytes += (size_t)round_up(pl.n * ell * 8, 256);
    if (plan_out) *plan_out = pl;
    return bytes;
}

corutv_status launch_request(corutv_ctx* ctx, ServingSlot& s, const PendingReq& pr) {
    const corutv_request& r = pr.req;
    FactorPlan pl;
    corutv_status st;
    request_bytes(r, pr.host, ctx->num_sms, &pl, &st);
    if (st != CORUTV_OK) return st;
    const ElemType ta = r.dtype == CORUTV_F64 ? T_F64 : T_F32;
    const int es = elem_size(ta);
    const int64_t m = r.m, n = r.n, ell = pl.ell;
    // device inputs: nothing of this request starts before the work the caller
    // had queued on its stream when it submitted (the producer of A, psi)
    if (pr.ready) CK(cudaStreamWaitEvent(s.st, pr.ready, 0));
    Carver cv(s.ws.ptr);
    FactorBufs b;
    carve_factor(cv, pl, b);
    const void* a_dev = r.A;
    void *u_dev = r.U, *t_dev = r.T, *v_dev = r.V;
    int32_t* perm_dev = r.perm;
    int64_t ldu = r.ldu, ldv = r.ldv;
    if (pr.host) {
        void* as = cv.take<char>(m * n * es);
        u_dev = cv.take<char>(m * ell * es);
        v_dev = cv.take<char>(n * ell * es);
        t_dev = cv.take<char>(ell * ell * es);
        perm_dev = cv.take<int>(ell);
        CK(cudaMemcpy2DAsync(as, n * es, r.A, r.lda * es, n * es, m, cudaMemcpyHostToDevice, s.st));
        a_dev = as;
        ldu = ell;
        ldv = ell;
    }
    const double* psi = nullptr;
    if (r.opts.psi) {
        double* ps = cv.take<double>(pl.n * ell);
        CK(cudaMemcpyAsync(ps, r.opts.psi, sizeof(double) * pl.n * ell, cudaMemcpyDefault, s.st));
        psi = ps;
    }
    CK(cudaMemsetAsync(s.flags, 0, sizeof(int) * FLAG_COUNT, s.st));
    Exec ex{s.st, s.flags, nullptr, ctx->num_sms};
    CKS(run_factor(ex, pl, b, a_dev, psi, r.opts.seed, r.opts.stream));
    CKS(emit_user(ex, pl, b, ta, r.U ? u_dev : nullptr, ldu, t_dev, r.V ? v_dev : nullptr, ldv,
                  r.perm ? perm_dev : nullptr));
    if (pr.host) {
        if (r.U) CK(cudaMemcpy2DAsync(r.U, r.ldu * es, u_dev, ell * es, ell * es, m, cudaMemcpyDeviceToHost, s.st));
        if (r.V) CK(cudaMemcpy2DAsync(r.V, r.ldv * es, v_dev, ell * es, ell * es, n, cudaMemcpyDeviceToHost, s.st));
        CK(cudaMemcpyAsync(r.T, t_dev, ell * ell * es, cudaMemcpyDeviceToHost, s.st));
        if (r.perm) CK(cudaMemcpyAsync(r.perm, perm_dev, sizeof(int32_t) * ell, cudaMemcpyDeviceToHost, s.st));
    }
    CK(cudaMemcpyAsync(s.hflags, s.flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, s.st));
    CK(cudaEventRecord(s.done, s.st));
    return CORUTV_OK;
}

// A request the batch lanes take: device FP32 input, BF16 sketches on the
// split path, a seeded test matrix and none of the variants (the grouped
// path's scope); the others run one per slot.
bool batchable(const PendingReq& pr) {
    const corutv_request& r = pr.req;
    const corutv_opts& o = r.opts;
    return !pr.host && r.dtype == CORUTV_F32 && o.sketch_prec == CORUTV_P_BF16 && o.d_mode == 0 &&
           o.t_lower == 0 && o.power_form == 0 && o.bf16_last_round == 0 && !o.psi && o.k + o.p <= 128;
}

// One batch on a lane: its requests' producers first, then the grouped
// launches, the lane's status words to the host and the completion event.
corutv_status launch_batch(corutv_ctx* ctx, BatchLane& l, const std::vector<PendingReq>& prs) {
    for (auto& pr : prs)
        if (pr.ready) CK(cudaStreamWaitEvent(l.st, pr.ready, 0));
    std::vector<corutv_request> reqs;
    reqs.reserve(prs.size());
    for (auto& pr : prs) reqs.push_back(pr.req);
    CK(cudaMemsetAsync(l.flags, 0, sizeof(int) * FLAG_COUNT, l.st));
    CKS(run_batch(ctx, l.bs, reqs.data(), (int)reqs.size(), l.st, l.flags));
    CK(cudaMemcpyAsync(l.hflags, l.flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, l.st));
    CK(cudaEventRecord(l.done, l.st));
    return CORUTV_OK;
}

void finish_lane(corutv_ctx* ctx, BatchLane& l, corutv_status st) {
    const auto now = std::chrono::steady_clock::now();
    for (uint64_t t : l.tickets) {
        auto it = ctx->results.find(t);
        if (it == ctx->results.end()) continue;
        it->second.done = true;
        it->second.status = st;
        if (st != CORUTV_OK) it->second.msg = g_last_error;
        it->second.latency = std::chrono::duration<double>(now - it->second.t0).count();
    }
    l.tickets.clear();
    l.busy = false;
}

void finish_slot(corutv_ctx* ctx, ServingSlot& s, corutv_status st) {
    auto it = ctx->results.find(s.ticket);
    if (it != ctx->results.end()) {
        it->second.done = true;
        it->second.status = st;
        if (st != CORUTV_OK) it->second.msg = g_last_error;
        it->second.latency =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - it->second.t0).count();
    }
    s.busy = false;
}

// Memory held by idle slots and idle batch lanes (other than `keep`) given
// back, so that a request too large for what is left can be admitted; true
// if anything was freed. Slot workspaces are freed in their stream's order,
// a lane's buffers with cudaFree (its stream has no pending work).
bool release_idle(corutv_ctx* ctx, const BatchLane* keep) {
    bool freed = false;
    for (auto& s : ctx->slots) {
        if (s.busy || !s.ws.ptr) continue;
        cudaFreeAsync(s.ws.ptr, s.st);
        ctx->serving_bytes -= s.ws.cap;
        s.ws.ptr = nullptr;
        s.ws.cap = 0;
        freed = true;
    }
    for (auto& l : ctx->lanes) {
        if (l.busy || &l == keep) continue;
        for (DeviceBuffer* b : {&l.bs.ws, &l.bs.desc}) {
            if (!b->ptr) continue;
            cudaFree(b->ptr);
            ctx->serving_bytes -= b->cap;
            b->ptr = nullptr;
            b->cap = 0;
            freed = true;
        }
    }
    cudaGetLastError();
    return freed;
}

void worker_main(corutv_ctx* ctx) {
    DeviceGuard guard(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->smu);
    while (true) {
        bool progressed = false;
        // retire
        for (auto& s : ctx->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaSuccess) {
                corutv_status st = CORUTV_OK;
                if (s.hflags[FLAG_BREAKDOWN]) st = CORUTV_EBREAKDOWN;
                else if (s.hflags[FLAG_TIMEOUT]) st = CORUTV_ETIMEDOUT;
                finish_slot(ctx, s, st);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                finish_slot(ctx, s, CORUTV_ECUDA);
                progressed = true;
            }
        }
        for (auto& l : ctx->lanes) {
            if (!l.busy) continue;
            const cudaError_t q = cudaEventQuery(l.done);
            if (q == cudaSuccess) {
                corutv_status st = CORUTV_OK;
                if (l.hflags[FLAG_BREAKDOWN]) st = fail(CORUTV_EBREAKDOWN, "a Cholesky of the batch broke down");
                else if (l.hflags[FLAG_TIMEOUT]) st = fail(CORUTV_ETIMEDOUT, "a device wait of the batch timed out");
                finish_lane(ctx, l, st);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                fail(CORUTV_ECUDA, "batch lane: %s", cudaGetErrorString(q));
                finish_lane(ctx, l, CORUTV_ECUDA);
                progressed = true;
            }
        }
        // admit in arrival order
        while (!ctx->queue.empty()) {
            PendingReq& head = ctx->queue.front();
            if (ctx->batch_max > 0 && batchable(head)) {
                // continuous batching: a free lane takes the queued batchable
                // requests at the head, up to batch_max and what memory allows
                BatchLane* lane = nullptr;
                for (auto& l : ctx->lanes)
                    if (!l.busy) { lane = &l; break; }
                if (!lane) break;
                const size_t held = lane->bs.ws.cap + lane->bs.desc.cap;
                const size_t others = ctx->serving_bytes - held;
                const size_t avail = ctx->budget > others ? ctx->budget - others : 0;
                std::vector<PendingReq> take;
                size_t sum = 0;
                for (auto it = ctx->queue.begin(); it != ctx->queue.end() && (int)take.size() < ctx->batch_max &&
                                                   batchable(*it);
                     ++it) {
                    if (sum + it->bytes + (size_t)(1 << 20) > avail) break;  // (records: well under 1 MB)
                    sum += it->bytes;
                    take.push_back(*it);
                }
                if (take.empty()) {
                    if (release_idle(ctx, lane)) continue;  // retry with the idle memory given back
                    break;                                   // waits for running work to free memory
                }
                ctx->queue.erase(ctx->queue.begin(), ctx->queue.begin() + (std::ptrdiff_t)take.size());
                lane->busy = true;
                lane->tickets.clear();
                for (auto& pr : take) lane->tickets.push_back(pr.ticket);
                lk.unlock();
                const corutv_status st = launch_batch(ctx, *lane, take);
                lk.lock();
                ctx->serving_bytes = others + lane->bs.ws.cap + lane->bs.desc.cap;
                for (auto& pr : take)
                    if (pr.ready) ctx->ev_pool.push_back(pr.ready);
                if (st != CORUTV_OK) finish_lane(ctx, *lane, st);
                progressed = true;
                continue;
            }
            ServingSlot* pick = nullptr;
            for (auto& s : ctx->slots)
                if (!s.busy && s.ws.cap >= head.bytes) { pick = &s; break; }
            if (!pick) {
                for (auto& s : ctx->slots) {
                    if (s.busy) continue;
                    if (ctx->serving_bytes - s.ws.cap + head.bytes <= ctx->budget) { pick = &s; break; }
                }
                if (pick) {
                    // grow this idle slot's workspace (stream-ordered, no device-wide sync)
                    if (pick->ws.ptr) {
                        cudaFreeAsync(pick->ws.ptr, pick->st);
                        ctx->serving_bytes -= pick->ws.cap;
                        pick->ws.ptr = nullptr;
                        pick->ws.cap = 0;
                    }
                    if (cudaMallocAsync(&pick->ws.ptr, head.bytes, pick->st) != cudaSuccess) {
                        cudaGetLastError();
                        pick->ws.ptr = nullptr;
                        pick = nullptr;
                    } else {
                        pick->ws.cap = head.bytes;
                        ctx->serving_bytes += head.bytes;
                    }
                }
            }
            if (!pick) {
                if (release_idle(ctx, nullptr)) continue;  // retry with the idle memory given back
                break;
            }
            PendingReq pr = head;
            ctx->queue.pop_front();
            pick->busy = true;
            pick->ticket = pr.ticket;
            lk.unlock();
            corutv_status st = launch_request(ctx, *pick, pr);
            lk.lock();
            // the slot stream's wait is enqueued: the event may be recorded again
            if (pr.ready) ctx->ev_pool.push_back(pr.ready);
            if (st != CORUTV_OK) finish_slot(ctx, *pick, st);
            progressed = true;
        }
        if (progressed) ctx->scv.notify_all();
        if (ctx->stop) {
            bool any_busy = false;
            for (auto& s : ctx->slots) any_busy |= s.busy;
            for (auto& l : ctx->lanes) any_busy |= l.busy;
            if (!any_busy) break;
        }
        ctx->scv.wait_for(lk, std::chrono::microseconds(progressed ? 0 : 20));
    }
}

corutv_status start_worker(corutv_ctx* ctx) {
    if (ctx->worker_started) return CORUTV_OK;
    ctx->slots.resize(ctx->max_slots);
    for (auto& s : ctx->slots) {
        CK(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
        CK(cudaMalloc(&s.flags, sizeof(int) * FLAG_COUNT));
        CK(cudaMallocHost(&s.hflags, sizeof(int) * FLAG_COUNT));
        CK(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    }
    ctx->worker = std::thread(worker_main, ctx);
    ctx->worker_started = true;
    return CORUTV_OK;
}

}  // namespace

extern "C" corutv_status corutv_submit(corutv_ctx* ctx, const corutv_request* req, uint64_t* ticket) {
    CKS(check_ctx(ctx));
    if (!req || !ticket || !req->A || !req->T) return fail(CORUTV_EINVAL, "req, ticket, A and T must not be NULL");
    if (req->opts.d_mode != 0 && req->opts.d_mode != 1) return fail(CORUTV_EINVAL, "d_mode must be 0 or 1");
    if (req->lda < req->n) return fail(CORUTV_EINVAL, "lda = %lld < n = %lld", (long long)req->lda, (long long)req->n);
    DeviceGuard guard(ctx->device);
    const bool host = !is_device_ptr(req->A);
    corutv_status st;
    const size_t bytes = request_bytes(*req, host, ctx->num_sms, nullptr, &st);
    if (st != CORUTV_OK) return st;
    if (bytes > ctx->budget)
        return fail(CORUTV_ENOMEM, "request needs %zu bytes of workspace, budget is %zu", bytes, ctx->budget);
    std::lock_guard<std::mutex> lk(ctx->smu);
    CKS(start_worker(ctx));
    cudaEvent_t ready = nullptr;
    if (!host) {
        // mark the caller's stream (the context's stream, corutv_set_stream) at
        // submission: the request's kernels wait for everything queued before it
        if (!ctx->ev_pool.empty()) {
            ready = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
        } else {
            CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        }
        cudaError_t e;
        {
            std::lock_guard<std::mutex> lk2(ctx->call_mu);
            e = cudaEventRecord(ready, ctx->stream);
        }
        if (e != cudaSuccess) {
            ctx->ev_pool.push_back(ready);
            return fail(CORUTV_ECUDA, "cudaEventRecord at submit failed: %s", cudaGetErrorString(e));
        }
    }
    PendingReq pr{ctx->next_ticket++, *req, std::chrono::steady_clock::now(), bytes, host, ready};
    ReqResult rr;
    rr.t0 = pr.t0;
    ctx->results[pr.ticket] = rr;
    ctx->queue.push_back(pr);
    *ticket = pr.ticket;
    ctx->scv.notify_all();
    return CORUTV_OK;
}

extern "C" corutv_status corutv_set_batching(corutv_ctx* ctx, int max_batch) {
    CKS(check_ctx(ctx));
    if (max_batch < 0 || max_batch > 4096) return fail(CORUTV_EINVAL, "max_batch must be in 0 .. 4096");
    DeviceGuard guard(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->smu);
    if (max_batch > 0 && ctx->lanes.empty()) {
        ctx->lanes.resize(2);
        for (auto& l : ctx->lanes) {
            CK(cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking));
            CK(cudaMalloc(&l.flags, sizeof(int) * FLAG_COUNT));
            CK(cudaMallocHost(&l.hflags, sizeof(int) * FLAG_COUNT));
            CK(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming));
        }
    }
    ctx->batch_max = max_batch;
    return CORUTV_OK;
}

extern "C" corutv_status corutv_poll(corutv_ctx* ctx, uint64_t ticket, int64_t timeout_us, double* latency_s) {
    CKS(check_ctx(ctx));
    std::unique_lock<std::mutex> lk(ctx->smu);
    auto it = ctx->results.find(ticket);
    if (it == ctx->results.end()) return fail(CORUTV_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    auto ready = [&] { return ctx->results[ticket].done; };
    if (!ready()) {
        if (timeout_us == 0) return CORUTV_EPENDING;
        if (timeout_us < 0) ctx->scv.wait(lk, ready);
        else if (!ctx->scv.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
            return fail(CORUTV_ETIMEDOUT, "ticket %llu not finished after %lld us", (unsigned long long)ticket,
                        (long long)timeout_us);
    }
    ReqResult rr = ctx->results[ticket];
    ctx->results.erase(ticket);
    if (latency_s) *latency_s = rr.latency;
    if (rr.status != CORUTV_OK && rr.status != CORUTV_EPENDING)
        return fail(rr.status, "request %llu failed with status %d: %s", (unsigned long long)ticket, (int)rr.status,
                    rr.msg.c_str());
    return rr.status;
}
