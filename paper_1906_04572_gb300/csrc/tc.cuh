// Tensor-core (tcgen05 + TMA) sketch products of libcorutv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace corutv {

// Elements of split-K partial storage the tensor-core products may use
// (FP32 elements; the caller provides at least this many).
int64_t tc_partial_elems(int64_t m, int64_t n, int64_t ellp, int64_t ldm, int64_t ldn, int num_sms);

// C = A X (trans = 0; C: m x ell panel with ld ldc = ldm) or C = A^T X
// (trans = 1; C: n x ell panel, ldc = ldn). A: m x n row-major of type ta
// (T_BF16 -> kind::f16 with bf16 operands; T_F32 -> kind::tf32), row stride
// lda (lda * elem_size a multiple of 16 bytes). X: panel of the same element
// type with ellp columns (padding columns zero), ld ldx. FP32 accumulation;
// C is written as FP64. `part` holds split partials.
cudaError_t launch_sketch_tc(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, int trans,
                             const void* x, int64_t ldx, int64_t ell, int64_t ellp, void* part, double* c,
                             int64_t ldc, int num_sms, int* flags, const int* cancel, cudaStream_t st);

// abf[i * ldb + j] = bf16(A[i * lda + j]) (round to nearest even); columns
// [n, ldb) are zero.
cudaError_t launch_cast_bf16(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* abf,
                             int64_t ldb, const int* cancel, cudaStream_t st);

// True when a row-major matrix can be a TMA source as is: 16-byte aligned
// base and row stride.
bool tma_rows_aligned(const void* a, int64_t lda, int elem_bytes);

// out[i * ldb + j] = A[i * lda + j] for j < n, 0 for n <= j < ldb.
cudaError_t launch_copy_f32_padded(const float* a, int64_t m, int64_t n, int64_t lda, float* out, int64_t ldb,
                                   cudaStream_t st);

}  // namespace corutv
