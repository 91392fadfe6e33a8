// Internal declarations of libcorutv (not part of the public ABI).
//
// Layout conventions inside the library
//  * "panel": a tall-skinny rows x ell matrix stored column-major, element
//    (i, j) at p[j * ld + i], ld a multiple of 32 elements. Sketches C1, C2,
//    the bases Q1, Q2 and the test matrix X all live in this layout, so the
//    coalesced direction of every skinny product is the long one.
//  * "small": an ell x ell matrix stored row-major with row stride ell.
//  * user matrices (A, M, U, V, T, L, S) are row-major with a leading
//    dimension, as in the public header.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>
#include <unordered_set>

namespace corutv {

// Device-side status words, one small array per context / request.
enum FlagIndex {
    FLAG_BREAKDOWN = 0,   // a Cholesky of a Gram matrix failed even after shifting
    FLAG_SHIFTED = 1,     // count of Gram matrices that needed the shift
    FLAG_TIMEOUT = 2,     // a bounded device wait gave up
    FLAG_RPCA_DONE = 3,   // ALM loop converged: later iteration kernels exit at once
    FLAG_RPCA_ITERS = 4,  // iterations executed
    FLAG_RPCA_RANK = 5,   // r of the last executed iteration
    FLAG_COUNT = 16
};

enum ElemType { T_F64 = 0, T_F32 = 1, T_BF16 = 2, T_SAME = 3 };

inline int elem_size(ElemType t) { return t == T_F64 ? 8 : (t == T_F32 ? 4 : 2); }

// How the generic skinny product reads its "A" operand. The product is
//   out[r][j] = sum_k Aop[k][r] * Bop[k][j],  r < R, k < K, j < L (L <= 128).
enum AMode {
    A_ROWS = 0,     // Aop[k][r] = A[r * lda + k]   : C = A X     (r = row of A)
    A_COLS = 1,     // Aop[k][r] = A[k * lda + r]   : C = A^T Y   (r = column of A)
    A_PANEL_T = 2,  // Aop[k][r] = P[r * ldp + k]   : G = X^T Y   (r = panel column)
    A_PANEL = 3     // Aop[k][r] = P[k * ldp + r]   : Q = P B     (r = panel row)
};
enum BMode {
    B_PANEL = 0,    // Bop[k][j] = Y[j * ldb + k]
    B_SMALL = 1     // Bop[k][j] = Bm[k * ldb + j]
};
enum OMode {
    O_PANEL = 0,    // out[j * ldo + r]  (+ split * split_stride)
    O_ROWMAJ = 1    // out[r * ldo + j]  (+ split * split_stride)
};

struct GemmArgs {
    AMode amode;
    BMode bmode;
    OMode omode;
    ElemType ta;          // element type of A (F64 / F32)
    ElemType tc;          // compute type = element type of the output
    const void* a;
    int64_t lda;
    const void* b;
    int64_t ldb;
    void* out;
    int64_t ldo;
    int64_t split_stride; // elements between split outputs
    int64_t R, K, L;
    int splits;           // K is cut into `splits` ranges, each written separately
    const int* cancel;    // optional device flag: kernels return at once when set
    ElemType tb = T_SAME; // element type of B (T_SAME: the compute type)
};

// Number of SMs of the current device (cached per device).
int device_sms();

// Counts every kernel launch issued by this library (instrumentation).
void count_launch();
// Largest sketch width ell on the SIMT paths (FP64 / FP32 sketches): the
// ell x ell steps beyond 128 run in global memory (one block each), the
// products in column groups of at most 128.
constexpr int kMaxEllSimt = 320;

// Programmatic dependent launch. Every kernel of the library is launched with
// programmatic stream serialisation, so the next kernel in a stream can be
// scheduled while the previous one finishes instead of after it. Each kernel
// calls pdl_trigger() first (its successor may then launch once all of its
// blocks are running) and pdl_wait() before it reads anything an earlier
// kernel wrote (the wait returns when the predecessor has completed and its
// writes are visible; it is a no-op for a launch without the attribute).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#ifdef __CUDACC__
// Exact float -> double by integer operations (normal and zero inputs; the
// rest through the conversion instruction). The FP64 conversion instruction
// would take a slot of the FP64 pipe, which this GPU has little of.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;  // zero, subnormal, inf, nan
    const unsigned long long s = (unsigned long long)(u >> 31) << 63;
    const unsigned long long bits = s | ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double f2d_exact(double d) { return d; }
#endif

// Stream-K tile ownership of the tensor-core products: unit u (tile t = u / kc,
// K chunk u % kc) belongs to CTA c with c units / grid <= u < (c + 1) units / grid.
__host__ __device__ __forceinline__ long long unit_owner(long long u, long long units, long long grid) {
    return ((u + 1) * grid + units - 1) / units - 1;
}

// Output of a tensor-core product whose split tiles were left as pieces for
// the consumer (the first kernel to read the panel adds them): tile t of 128
// rows covered by np(t) > 1 CTAs has its FP32 partials at part[((t * maxp +
// pc) * ellp + j) * 128 + (row % 128)], pc = 0 .. np-1, added in that order;
// tiles covered by one CTA are in the panel itself. part == nullptr: the
// panel is complete.
struct TcPieces {
    const float* part = nullptr;
    long long units = 0, kc = 1;
    int grid = 1, maxp = 1, ellp = 0;
};

// Every kernel asks for the largest shared-memory carve-out once, so that the
// switches between the tensor-core products (about 200 KB of shared memory
// per block) and the small kernels around them do not reconfigure the SMs'
// L1 / shared split.
inline void prefer_max_shared(const void* fn) {
    // a per-thread record first: no lock on the launch path once a kernel is known
    thread_local std::unordered_set<const void*> seen;
    if (seen.count(fn)) return;
    static std::mutex mu;
    static std::unordered_set<const void*> done;
    std::lock_guard<std::mutex> lk(mu);
    seen.insert(fn);
    if (done.insert(fn).second)
        if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            cudaGetLastError();  // a preference only: ignore a refusal
}

// Raises the largest dynamic shared memory a launch of `fn` may ask for to
// what the device allows, once per function and device. It is a limit, not a
// reservation: each launch still gets (and is scheduled with) the size it
// asks for. Setting it per launch to that launch's size instead would race
// between host threads that launch the same kernel with different sizes (the
// serving slots), one thread's smaller setting failing the other's launch.
inline cudaError_t allow_max_dynamic_smem(const void* fn) {
    static std::mutex mu;
    static std::unordered_set<unsigned long long> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long key = (reinterpret_cast<unsigned long long>(fn) << 6) ^ (unsigned long long)dev;
    thread_local std::unordered_set<unsigned long long> seen;  // per-thread record: no lock once known
    if (seen.count(key)) return cudaSuccess;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) {
        seen.insert(key);
        return cudaSuccess;
    }
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) {
        done.insert(key);
        seen.insert(key);
    }
    return e;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    prefer_max_shared(reinterpret_cast<const void*>(kernel));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Sets the calling thread's message returned by corutv_last_error().
void record_error(const char* msg);

// ---- launchers (all stream-ordered, never synchronising) ----------------
cudaError_t launch_gemm_simt(const GemmArgs& g, cudaStream_t st);
int gemm_simt_splits(int64_t R, int64_t K, int num_sms);

// out[e] = sum_{s < splits} part[s * stride + e] over a rows x cols region
// with leading dimension ld (panel: rows = R, cols = L; small: rows = L).
cudaError_t launch_reduce_splits(const void* part, ElemType tpart, int splits, int64_t stride, void* out,
                                 ElemType tout, int64_t ld, int64_t rows, int64_t cols, int64_t ld_out,
                                 const int* cancel, cudaStream_t st);

cudaError_t launch_gaussian_panel(uint64_t seed, uint32_t stream_id, int64_t n, int64_t ell,
                                  int64_t ellp, void* x, ElemType tx, int64_t ldx, const int* cancel,
                                  cudaStream_t st);
cudaError_t launch_gaussian_rowmajor(uint64_t seed, uint32_t stream_id, int64_t n, int64_t ell,
                                     double* psi, int64_t ld, cudaStream_t st);

// Layout / type conversions.
cudaError_t launch_rowmajor_to_panel(const double* src, int64_t lds, int64_t rows, int64_t cols,
                                     int64_t colsp, void* dst, ElemType tdst, int64_t ldd, cudaStream_t st);
cudaError_t launch_panel_convert(const void* src, ElemType tsrc, int64_t lds, int64_t rows, int64_t cols,
                                 void* dst, ElemType tdst, int64_t ldd, const int* cancel, cudaStream_t st);
cudaError_t launch_panel_to_rowmajor(const double* src, int64_t lds, int64_t rows, int64_t cols,
                                     void* dst, ElemType tdst, int64_t ldd, const int* cancel,
                                     cudaStream_t st);

// CholeskyQR pieces (k_qr.cu).
// R = chol(G) (upper, R^T R = G + shift I), FP64, one block; flags as above.
// *skip_out (optional) is set to 0 when a shift was needed (so a third
// CholeskyQR pass must run) and to 1 otherwise or when cancelled.
// unit_roundoff: of the arithmetic G was formed in (2^-53 FP64, 2^-24 FP32);
// it scales the shift. With `defic` (ell ints, written), a pivot at most
// tau_rel times the largest diagonal entry marks its column numerically
// dependent (defic[j] = 1, R row j = e_j) instead of failing.
cudaError_t launch_cholesky(const double* g, int64_t ell, int64_t rows, double* r, int* flags,
                            int* skip_out, const int* cancel, cudaStream_t st,
                            double unit_roundoff = 0x1p-53, int* defic = nullptr, double tau_rel = 0.0);
// out = Rn Ra for upper triangular ell x ell FP64 factors (row-major); Ra null:
// out = Rn; *skip set: out = Ra (copy-through for a pass that did not run);
// transpose: out receives the transpose. out must not alias Rn or Ra.
cudaError_t launch_trimul(const double* rn, const double* ra, double* out, int64_t ell, bool transpose,
                          const int* skip, const int* cancel, cudaStream_t st);
// Q = C R^{-1} row by row (forward substitution with R^T), compute type tc;
// c and q are panels of type tp; if qc != nullptr a copy of type tqc is
// written too.
// defic (optional, from launch_cholesky): dependent columns of Q are filled
// with a seeded random completion.
cudaError_t launch_trsm_rows(const void* c, ElemType tp, int64_t ldc, int64_t rows, int64_t ell,
                             const double* r, ElemType tc, void* q, int64_t ldq, void* qc,
                             ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st,
                             const int* defic = nullptr, float* rinv_work = nullptr);
// Size (floats) of the rinv_work buffer that selects, for FP32 panels solved
// in FP32, the inverse-and-product form of the triangular solve.
int64_t trsm_rinv_floats(int64_t ell);
// FP32 Gram G = X^T Y (row-major ell x ell FP64 output) of two FP32 panels
// in one launch; split sums reduced in the kernel in a fixed order. work:
// gram_f32_work_floats floats; cnt: gram_f32_counters ints, zero before the
// first call (every call leaves them zero).
int64_t gram_f32_work_floats(int64_t len, int ell, int num_sms);
int64_t gram_f32_counters(int64_t len, int ell, int num_sms);
// px / py: pieces of X / Y still to be added (TcPieces); with writeback the
// added rows are stored into that panel as well, completing it for later
// kernels.
cudaError_t launch_gram_f32(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len, int ell,
                            double* out, float* work, int* cnt, int num_sms, const int* cancel, cudaStream_t st,
                            const TcPieces& px = TcPieces(), const TcPieces& py = TcPieces(), bool writeback = false);
// Column-pivoted QR of the small ell x ell FP64 matrix d (eq. 8): the
// factorisation in one block, then Qt formed from its reflectors by several
// blocks. work: ell * (ell + 2) doubles of device scratch.
cudaError_t launch_qrcp(const double* d, int64_t ell, double* qt, double* rt, int* perm, double* work,
                        const int* cancel, cudaStream_t st, bool form_q = true);
// Qt (ell x ell, row-major) from the reflectors launch_qrcp left in refl.
cudaError_t launch_qform(const double* refl, int64_t ell, double* qt, const int* cancel, cudaStream_t st);
// U = Q1 Qt from the reflectors the QRCP left in `refl` (its work array),
// without Qt: q1 a panel of type tp (ld ldq, `rows` rows); out row-major
// (ld ldo) or, with out_panel, a panel; element type tout.
cudaError_t launch_apply_reflectors(const void* q1, ElemType tp, int64_t ldq, int64_t rows, int64_t ell,
                                    const double* refl, void* out, ElemType tout, int64_t ldo, bool out_panel,
                                    const int* cancel, cudaStream_t st);
// V[i][j] = Q2[perm[j]] (Q2 a panel of type tq2; row-major output of type tv).
cudaError_t launch_gather_v(const void* q2, ElemType tq2, int64_t ldq2, int64_t n, int64_t ell, const int* perm,
                            void* v, ElemType tv, int64_t ldv, const int* cancel, cudaStream_t st);
cudaError_t launch_copy_small(const double* src, int64_t ell, void* dst, ElemType tdst,
                              const int* cancel, cudaStream_t st, bool transpose = false);

// ---- grouped launches: one launch over the problems of a batch ----------
// Problem z of a grouped launch (blockIdx.z) runs the blocks (x, y) < (gx, gy)
// of its own grid with its own arguments; blocks beyond that grid return at
// once. The launch's grid is the largest over its problems, by the number of
// problems. Kernels with grid-stride loops get gx = the launch's gx (no block
// returns early), so the stride is the launch's own.
template <class A>
struct GroupItem {
    A a;
    unsigned gx, gy;
};

#ifdef __CUDACC__
template <class A, void (*F)(const A&), int kMaxThreads>
__global__ void __launch_bounds__(kMaxThreads) grouped_kernel(const GroupItem<A>* items) {
    const GroupItem<A>& it = items[blockIdx.z];
    if (blockIdx.x >= it.gx || blockIdx.y >= it.gy) return;
    F(it.a);
}
#endif

// Arguments of the grouped kernels (each the argument list of its one-problem
// launch; panels and small matrices as above).
struct ZeroArgs { void* p; int64_t bytes; };
// Gaussian test panel written as bf16 (the FP32 draw of launch_gaussian_panel, rounded)
struct GaussArgs { uint64_t seed; uint32_t sid; int64_t n, ell, ellp; void* x; int64_t ldx; const int* cancel; };
// tiled bf16 splits A_h, A_m, A_l of FP32 A (launch_cast_tiled with three parts)
struct CastArgs { const float* a; int64_t m, n, lda; void* out; const int* cancel; };
// [Q_h | Q_m | Q_l] of an FP32 panel (launch_split_panel)
struct SplitArgs { const float* q; int64_t ldq, rows; int ell, ellp; void* q3; int64_t ldq3; const int* cancel; };
struct CholArgs {
    const double* g; int ell; int64_t rows; double* r; int* flags; int* skip_out; const int* cancel;
    double unit_roundoff; int* defic; double tau_rel;
};
struct RinvArgs { const double* r; int ell; float* ri; int ldri; const int* cancel; };
// Q = C R^{-1} from R^{-1} (FP32 panels); qc: copy of element type bf16 or none
struct TrsmArgs {
    const float* c; int64_t ldc, rows; int ell; const float* ri; int ldri; float* q; int64_t ldq; void* qc;
    int64_t ldqc; const int* cancel; const int* defic;
};
struct QrcpArgs { const double* d; int ell; double* refl; double* rt; int* perm; const int* cancel; };
// U = Q1 Qt from the reflectors (FP32 panel in, FP32 row-major out)
struct ReflArgs { const float* x; int64_t ldx, rows; int ell; const double* refl; float* out; int64_t ldo; const int* cancel; };
struct GatherArgs { const float* q2; int64_t ldq2, n; int ell; const int* perm; float* v; int64_t ldv; const int* cancel; };
// T = Rt as FP32 (row-major ell x ell) and perm copied out
struct EmitArgs { const double* rt; int ell; float* t; const int* perm_src; int* perm_dst; const int* cancel; };
// FP32 Gram X^T Y of two complete panels (no pieces): its plan fields as
// chosen by gram_group_item
struct GramArgs {
    const float* x; int64_t ldx; const float* y; int64_t ldy; int64_t len; int ell; double* out; float* work;
    int* cnt; int ntile, tiles, nc, sym; const int* cancel;
};

// Grid-stride kernels: every block of the launch serves every problem.
constexpr unsigned kAnyGrid = 0xffffffffu;
// Blocks of 256 threads for a grid-stride pass over `total` elements.
inline unsigned stride_grid(int64_t total) {
    const int64_t b = (total + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

// Items with their grids, and the grouped launches (gx, gy: the largest grid
// of the items launched; count: how many items, from the first).
GroupItem<ZeroArgs> zero_item(void* p, int64_t bytes);
GroupItem<GaussArgs> gaussian_item(const GaussArgs& a);
GroupItem<CastArgs> cast3_item(const CastArgs& a);
GroupItem<SplitArgs> split_item(const SplitArgs& a);
GroupItem<CholArgs> cholesky_item(const CholArgs& a);
GroupItem<RinvArgs> rinv_item(const RinvArgs& a);
GroupItem<TrsmArgs> trsm_item(const TrsmArgs& a);
GroupItem<QrcpArgs> qrcp_item(const QrcpArgs& a);
GroupItem<ReflArgs> refl_item(const ReflArgs& a);
// the register-row form for ell <= 64 (gx = 0 for wider problems: refl_item's launch takes those)
GroupItem<ReflArgs> refl_rows_item(const ReflArgs& a);
GroupItem<GatherArgs> gather_item(const GatherArgs& a);
GroupItem<EmitArgs> emit_item(const EmitArgs& a);
// The Gram's plan for a problem of a batch: about 256 rows per CTA, from the
// problem's own sizes only (so a problem's sums do not depend on the batch).
// Its workspace and counters fit gram_f32_work_floats / gram_f32_counters
// for the same num_sms.
GroupItem<GramArgs> gram_group_item(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len, int ell,
                                    double* out, float* work, int* cnt, const int* cancel, int num_sms);
cudaError_t launch_zero_grouped(const GroupItem<ZeroArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_gaussian_grouped(const GroupItem<GaussArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_cast3_grouped(const GroupItem<CastArgs>* it, int count, unsigned gx, unsigned gy, cudaStream_t st);
cudaError_t launch_split_grouped(const GroupItem<SplitArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_cholesky_grouped(const GroupItem<CholArgs>* it, int count, int max_ell, bool defic,
                                    cudaStream_t st);
cudaError_t launch_rinv_grouped(const GroupItem<RinvArgs>* it, int count, unsigned gx, int max_ell, cudaStream_t st);
cudaError_t launch_trsm_grouped(const GroupItem<TrsmArgs>* it, int count, unsigned gx, int max_ell, bool qc_bf16,
                                cudaStream_t st);
cudaError_t launch_qrcp_grouped(const GroupItem<QrcpArgs>* it, int count, int max_ell, cudaStream_t st);
cudaError_t launch_refl_grouped(const GroupItem<ReflArgs>* it, int count, unsigned gx, int max_ell, cudaStream_t st);
cudaError_t launch_refl_rows_grouped(const GroupItem<ReflArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_gather_grouped(const GroupItem<GatherArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_emit_grouped(const GroupItem<EmitArgs>* it, int count, unsigned gx, cudaStream_t st);
cudaError_t launch_gram_grouped(const GroupItem<GramArgs>* it, int count, unsigned gx, unsigned gy, cudaStream_t st);

// RPCA pieces (k_rpca.cu).
struct RpcaIterArgs {
    const void* m; ElemType tm; int64_t ldm;
    int64_t rows, cols;
    float* s; float* y; float* b;           // FP32 state (dtype F32)
    double* s64; double* y64; double* b64;  // FP64 state (dtype F64)
    const double* u; int64_t ldu;           // U panel (rows x ell)
    const double* z; int64_t ldz;           // Z panel (cols x ell): Z = V T(1:r,:)^T
    int64_t ell;
    const int* rank;                        // device r
    double mu, mu_next, lambda;
    double* res_part;                       // per-block partial sums of residual^2
    const int* cancel;
};
cudaError_t launch_rpca_init(const void* m, ElemType tm, int64_t ldm, int64_t rows, int64_t cols,
                             float* s, float* y, float* b, double* s64, double* y64, double* b64,
                             double* fro_part, int* nparts, cudaStream_t st);
cudaError_t launch_rpca_rank_z(const double* rt, const void* vq2, ElemType tq2, int64_t ldv, const int* perm,
                               int64_t cols, int64_t ell, double inv_mu, int* rank, double* z,
                               int64_t ldz, const int* cancel, cudaStream_t st);
cudaError_t launch_rpca_update(const RpcaIterArgs& a, int* nparts, cudaStream_t st);
cudaError_t launch_rpca_finish_iter(const double* res_part, int nparts, const double* fro_part,
                                    int nfro, double tol, int iter, double* zeta_hist,
                                    int* flags, const int* rank, cudaStream_t st);
cudaError_t launch_rpca_reconstruct(const double* u, int64_t ldu, const double* z, int64_t ldz,
                                    const int* rank, int64_t ell, int64_t rows, int64_t cols,
                                    void* lout, ElemType tl, int64_t ldl, cudaStream_t st);

int rpca_update_blocks(int64_t rows, int64_t cols);

// Power iteration helpers for the ||M||_2 estimate: v = value; v = w / ||w||
// with ||w|| stored in *lam (one block).
cudaError_t launch_vec_fill(double* v, int64_t n, double value, cudaStream_t st);
cudaError_t launch_vec_normalize(const double* w, double* v, int64_t n, double* lam, cudaStream_t st);
// y = M x for a row-major m x n matrix M (FP32 or FP64, row stride ldm) and an
// FP64 vector x; FP64 accumulation, one warp per row.
cudaError_t launch_gemv_rows(const void* mat, ElemType tm, int64_t ldm, int64_t m, int64_t n, const double* x,
                             double* y, cudaStream_t st);
// part[q * ldp + c] = sum over rows i of chunk q (chunk_rows rows each) of
// M[i][c] u[i]; FP64 accumulation. The chunks are then added in order.
cudaError_t launch_gemv_cols_partial(const void* mat, ElemType tm, int64_t ldm, int64_t m, int64_t n,
                                     const double* u, double* part, int64_t ldp, int chunks, cudaStream_t st);

}  // namespace corutv
