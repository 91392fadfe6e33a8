// Tensor-core (tcgen05 + TMA) sketch products of libcorutv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace corutv {

// Elements of split-K partial storage the tensor-core products may use
// (FP32 elements; the caller provides at least this many).
int64_t tc_partial_elems(int64_t m, int64_t n, int64_t ellp, int64_t ldm, int64_t ldn, int num_sms);
// Per-tile completion counters the products need (int elements). They must
// be zero before the first product; every product leaves them zero again
// (unless it timed out).
int64_t tc_counter_elems(int64_t m, int64_t n);

// C = A X (trans = 0; C: m x ell panel with ld ldc = ldm) or C = A^T X
// (trans = 1; C: n x ell panel, ldc = ldn). A: m x n row-major of type ta
// (T_BF16 -> kind::f16 with bf16 operands; T_F32 -> kind::tf32), row stride
// lda (lda * elem_size a multiple of 16 bytes). X: panel of the same element
// type with ellp columns (padding columns zero), ld ldx. FP32 accumulation;
// C is written with element type tcout (FP64 or FP32). `part` holds split
// partials, `tile_cnt` the per-tile counters (tc_counter_elems). With
// `pieces` non-null the split tiles are left as pieces in `part` (described in
// *pieces) for the consumer to add; the counters are not used.
cudaError_t launch_sketch_tc(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, int trans,
                             const void* x, int64_t ldx, int64_t ell, int64_t ellp, void* part, int* tile_cnt,
                             void* c,
                             ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel,
                             cudaStream_t st, TcPieces* pieces = nullptr);

// Tiled bf16 copy of A (m x n, row stride lda, FP32 or FP64): tile (I, J) =
// rows 128 I.., columns 64 J.. (zero beyond m, n), 16 KB at byte
// ((I * tiled_ntp(n) + J) << 14) of each part, in the layout a 128-byte-swizzled
// TMA box of it takes in shared memory. nparts = 1: bf16(A) (round to nearest
// even); nparts = 3 (FP32 A): the exact splits A_h, A_m, A_l, one part each,
// tiled_part_bytes(m, n) apart. `out` 16-byte aligned.
int64_t tiled_ntp(int64_t n);
int64_t tiled_part_bytes(int64_t m, int64_t n);
cudaError_t launch_cast_tiled(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* out, int nparts,
                              const int* cancel, cudaStream_t st);
// The same for the 128-row blocks [rb0, rb1) and a choice of parts: 1 (A_h),
// 2 (A_m and A_l only, FP32 A), 3 (all three, FP32 A).
cudaError_t launch_cast_tiled_rows(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* out,
                                   int parts, int64_t rb0, int64_t rb1, const int* cancel, cudaStream_t st);
// launch_sketch_tc with A given as its tiled bf16 copy (launch_cast_tiled):
// every stage of A is one contiguous bulk copy. nsegs > 1 multiplies by the
// sum of the copy's first nsegs parts (A_h + A_m: A to about 16 significant
// bits instead of 8), each part a K segment of the same accumulation.
cudaError_t launch_sketch_tc_tiled(const void* a_tiles, int64_t m, int64_t n, int trans, const void* x, int64_t ldx,
                                   int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* c, ElemType tcout,
                                   int64_t ldc, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                                   TcPieces* pieces = nullptr, int nsegs = 1);
// FP32-accurate W = A Q on the tensor cores by exact three-way bf16 splits:
// a3 is the tiled copy of A with its three parts A_h, A_m, A_l
// (launch_cast_tiled with nparts = 3), q3 a bf16 panel of 3 * ellp columns
// [Q_h | Q_m | Q_l] (ld ldq). Products of bf16 parts are exact and accumulate
// in FP32, so W = the sum of the nine part products carries the rounding of an
// FP32 dot product. W: panel (ell columns, type tw, ld ldw).
cudaError_t launch_project_split_tc_tiled(const void* a3, int64_t m, int64_t n, const void* q3, int64_t ldq,
                                          int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* w, ElemType tw,
                                          int64_t ldw, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                                          TcPieces* pieces = nullptr);

// One warp holds tensor memory while it waits on an mbarrier nothing arrives
// on; after about limit_ns it sets flags[FLAG_TIMEOUT], frees the tensor
// memory and returns (a test of the bounded-wait path).
cudaError_t launch_wait_probe(int* flags, unsigned long long limit_ns, cudaStream_t st);

// True when a row-major matrix can be a TMA source as is: 16-byte aligned
// base and row stride.
bool tma_rows_aligned(const void* a, int64_t lda, int elem_bytes);

// out[i * ldb + j] = A[i * lda + j] for j < n, 0 for n <= j < ldb.
cudaError_t launch_copy_f32_padded(const float* a, int64_t m, int64_t n, int64_t lda, float* out, int64_t ldb,
                                   cudaStream_t st);

// One pass over FP32 A (m x n, row stride lda) writing any non-null of: at =
// A^T (n rows of stride ldt, ldt a multiple of 64 and >= m; columns
// [m, round_up(m, 64)) zero), a3 (as launch_cast_tiled with three parts) and a
// row-major copy acopy (row stride ldc, a multiple of 4 in [n, round_up(n, 64)],
// zero beyond n).
cudaError_t launch_prep_f32(const float* a, int64_t m, int64_t n, int64_t lda, float* at, int64_t ldt, void* a3,
                            float* acopy, int64_t ldc, const int* cancel, cudaStream_t st);
// Writes q3 = [Q_h | Q_m | Q_l] from an FP32 panel (ell valid columns of ellp).
cudaError_t launch_split_panel(const float* q, int64_t ldq, int64_t rows, int64_t ell, int64_t ellp, void* q3,
                               int64_t ldq3, const int* cancel, cudaStream_t st);

// Grouped products: one launch over the problems of a batch. Each problem is
// a record of tc_group_item_bytes() bytes (any host address; 128-byte
// aligned in device memory when launched) filled on the host by one of the
// two calls below, with the arguments of launch_sketch_tc_tiled (a product on the tiled bf16 copy) or
// of launch_project_split_tc_tiled (the split projection). A problem's grid
// is its own (about 64 stream-K units per CTA), so its sums do not depend on
// the other problems; its split tiles are added by the product itself (the
// counters must be zero). Out: the problem's grid, the dynamic shared memory
// it needs and the partial floats it may use.
size_t tc_group_item_bytes();
// Partial floats the three grouped products of an m x n problem may use.
int64_t tc_group_partial_elems(int64_t m, int64_t n, int64_t ellp, int num_sms);
cudaError_t tc_group_sketch_item(void* item, const void* a_tiles, int64_t m, int64_t n, int trans, const void* x,
                                 int64_t ldx, int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* c,
                                 ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel, int* grid,
                                 size_t* smem, int64_t* part_floats);
cudaError_t tc_group_project_item(void* item, const void* a3, int64_t m, int64_t n, const void* q3, int64_t ldq,
                                  int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* w, ElemType tw,
                                  int64_t ldw, int num_sms, int* flags, const int* cancel, int* grid, size_t* smem,
                                  int64_t* part_floats);
// count records from `items` (device); max_grid / max_smem: the largest grid
// and shared memory of those records.
cudaError_t launch_sketch_tc_grouped(const void* items, int count, int max_grid, size_t max_smem, cudaStream_t st);

// Stage-shape autotuner of the tensor-core products (process-wide).
void tc_set_autotune(bool on);
// Number of tuned shapes; for 0 <= index < that number, its extents and choice.
int tc_autotune_entry(int index, long long* mtot, long long* ktot, int* nb, int* trans, int* kgroup, int* stages,
                      float* us);

}  // namespace corutv
