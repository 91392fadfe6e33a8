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

// abf[i * ldb + j] = bf16(A[i * lda + j]) (round to nearest even); columns
// [n, ldb) are zero.
cudaError_t launch_cast_bf16(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* abf,
                             int64_t ldb, const int* cancel, cudaStream_t st);

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

// FP32-accurate W = A Q on the tensor cores by exact three-way bf16 splits:
// a3 holds rows [A_h | A_m | A_l] (each segment `seg` elements, seg a multiple
// of 64, zero beyond n), q3 is a bf16 panel of 3 * ellp columns
// [Q_h | Q_m | Q_l] (ld ldq). Products of bf16 parts are exact and
// accumulate in FP32, so W = sum of the nine part products carries the
// rounding of an FP32 dot product. W: panel (ell columns, type tw, ld ldw).
cudaError_t launch_project_split_tc(const void* a3, int64_t m, int64_t n, int64_t seg, const void* q3, int64_t ldq,
                                    int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* w, ElemType tw,
                                    int64_t ldw,
                                    int num_sms, int* flags, const int* cancel, cudaStream_t st,
                                    TcPieces* pieces = nullptr);
// Writes a3 (rows of [A_h | A_m | A_l]) from FP32 A.
cudaError_t launch_cast_bf16_split(const float* a, int64_t m, int64_t n, int64_t lda, void* a3, int64_t seg,
                                   const int* cancel, cudaStream_t st);
// One pass over FP32 A (m x n, row stride lda) writing any non-null of: at =
// A^T (n rows of stride ldt, ldt a multiple of 64 and >= m; columns
// [m, round_up(m, 64)) zero), a3 (as launch_cast_bf16_split) and a row-major
// copy acopy (row stride ldc, a multiple of 4 in [n, round_up(n, 64)], zero
// beyond n).
cudaError_t launch_prep_f32(const float* a, int64_t m, int64_t n, int64_t lda, float* at, int64_t ldt, void* a3,
                            int64_t seg, float* acopy, int64_t ldc, const int* cancel, cudaStream_t st);
// Writes q3 = [Q_h | Q_m | Q_l] from an FP32 panel (ell valid columns of ellp).
cudaError_t launch_split_panel(const float* q, int64_t ldq, int64_t rows, int64_t ell, int64_t ellp, void* q3,
                               int64_t ldq3, const int* cancel, cudaStream_t st);

}  // namespace corutv
