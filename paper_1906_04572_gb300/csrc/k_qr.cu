// Small dense factorisations of libcorutv:
//  * Cholesky of an ell x ell Gram matrix (CholeskyQR, the thin QR of
//    Sec. 3.1 "C1 = Q1 R1, C2 = Q2 R2"), FP64, with the shift of shifted
//    CholeskyQR (Fukaya et al., SIAM J. Sci. Comput. 2020) when the Gram is
//    not numerically positive definite;
//  * Q = C R^{-1} by forward substitution, one thread per row;
//  * the column-pivoted QR of D (eq. 8), one block, FP64, Householder
//    reflections with Businger-Golub pivoting on recomputed column norms;
//  * the gathers of eq. 9 (V = Q2 P, T = Rt).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace corutv {

namespace {

constexpr int kCholThreads = 256;

// rows = number of rows of the matrix whose Gram is factorised (for the shift).
__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* g, int ell, int64_t rows, double* r, int* flags, int* skip_out,
                const int* cancel) {
    const int tid = threadIdx.x;
    if (cancel && *cancel) {
        if (skip_out && tid == 0) *skip_out = 1;
        return;
    }
    extern __shared__ double S[];  // ell x (ell + 1)
    const int ld = ell + 1;
    __shared__ int fail;
    __shared__ double trace;
    if (tid == 0) {
        double t = 0.0;
        for (int a = 0; a < ell; ++a) t += g[a * ell + a];
        trace = t;
    }
    __syncthreads();
    // shift s = 11 (rows ell + ell (ell + 1)) u ||C||_F^2 (u = 2^-53), then x100
    const double u = 1.1102230246251565e-16;
    const double base_shift = 11.0 * ((double)rows * ell + (double)ell * (ell + 1)) * u * trace;
    int attempt = 0;
    for (; attempt < 3; ++attempt) {
        const double shift = attempt == 0 ? 0.0 : base_shift * (attempt == 1 ? 1.0 : 100.0);
        for (int e = tid; e < ell * ell; e += kCholThreads) {
            const int a = e / ell, b = e % ell;
            S[a * ld + b] = g[a * ell + b] + (a == b ? shift : 0.0);
        }
        if (tid == 0) fail = 0;
        __syncthreads();
        for (int j = 0; j < ell; ++j) {
            if (tid == 0) {
                const double d = S[j * ld + j];
                if (!(d > 0.0) || !isfinite(d)) fail = 1;
                else S[j * ld + j] = sqrt(d);
            }
            __syncthreads();
            if (fail) break;
            const double rjj = S[j * ld + j];
            for (int c = j + 1 + tid; c < ell; c += kCholThreads) S[j * ld + c] /= rjj;
            __syncthreads();
            const int nt = ell - j - 1;
            for (int e = tid; e < nt * nt; e += kCholThreads) {
                const int a = j + 1 + e / nt, b = j + 1 + e % nt;
                if (b >= a) S[a * ld + b] -= S[j * ld + a] * S[j * ld + b];
            }
            __syncthreads();
        }
        if (!fail) break;
        __syncthreads();
    }
    const bool broke = attempt == 3;
    for (int e = tid; e < ell * ell; e += kCholThreads) {
        const int a = e / ell, b = e % ell;
        double v = (b >= a) ? S[a * ld + b] : 0.0;
        if (broke) v = (a == b) ? 1.0 : 0.0;
        r[e] = v;
    }
    if (tid == 0) {
        if (broke) atomicExch(&flags[FLAG_BREAKDOWN], 1);
        if (attempt > 0) atomicAdd(&flags[FLAG_SHIFTED], 1);
        if (skip_out) *skip_out = (attempt > 0 && !broke) ? 0 : 1;
    }
}

// Row i of Q solves q_i R = c_i (R upper): q_i[j] = (c_i[j] - sum_{t<j} q_i[t] R[t][j]) / R[j][j].
template <typename TC, typename TQC>
__global__ void trsm_rows_kernel(const double* c, int64_t ldc, int64_t rows, int ell, const double* r,
                                 double* q, int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel) {
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* Rs = reinterpret_cast<TC*>(smem_raw);   // ell x ell row-major
    const int nthr = blockDim.x;
    TC* Ts = Rs + ell * ell;                      // [ell][nthr]
    const int tid = threadIdx.x;
    for (int e = tid; e < ell * ell; e += nthr) Rs[e] = (TC)r[e];
    const int64_t i = (int64_t)blockIdx.x * nthr + tid;
    if (i < rows)
        for (int j = 0; j < ell; ++j) Ts[j * nthr + tid] = (TC)c[j * ldc + i];
    __syncthreads();
    if (i >= rows) return;
    for (int j = 0; j < ell; ++j) {
        TC s0 = Ts[j * nthr + tid], s1 = 0;
        int t = 0;
        for (; t + 1 < j; t += 2) {
            s0 -= Ts[t * nthr + tid] * Rs[t * ell + j];
            s1 -= Ts[(t + 1) * nthr + tid] * Rs[(t + 1) * ell + j];
        }
        if (t < j) s0 -= Ts[t * nthr + tid] * Rs[t * ell + j];
        Ts[j * nthr + tid] = (s0 + s1) / Rs[j * ell + j];
    }
    for (int j = 0; j < ell; ++j) {
        const TC v = Ts[j * nthr + tid];
        q[j * ldq + i] = (double)v;
        if (qc) qc[j * ldqc + i] = (TQC)v;
    }
}

template <typename TC>
int trsm_threads(int ell) {
    const long budget = 200 * 1024;
    long per = (budget - (long)ell * ell * (long)sizeof(TC)) / ((long)ell * (long)sizeof(TC));
    per = per / 32 * 32;
    if (per > 256) per = 256;
    if (per < 32) per = 32;
    return (int)per;
}

template <typename TC, typename TQC>
cudaError_t trsm_launch(const double* c, int64_t ldc, int64_t rows, int ell, const double* r,
                        double* q, int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel,
                        cudaStream_t st) {
    const int nthr = trsm_threads<TC>(ell);
    const size_t smem = sizeof(TC) * ((size_t)ell * ell + (size_t)ell * nthr);
    cudaError_t e = cudaFuncSetAttribute(trsm_rows_kernel<TC, TQC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((rows + nthr - 1) / nthr);
    count_launch();
    trsm_rows_kernel<TC, TQC><<<blocks, nthr, smem, st>>>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// QRCP of the small D (eq. 8). 256 threads = 8 warps.
// ---------------------------------------------------------------------------
constexpr int kQrcpThreads = 256;
constexpr int kQrcpWarps = kQrcpThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Apply H = I - tau v v^T (v = [1; W[j+1:, j]]) to column c of W, rows j..ell-1.
__device__ __forceinline__ void house_apply_col(double* W, int ld, int ell, int j, int c, double tau,
                                                int lane) {
    double dot = 0.0;
    for (int i = j + 1 + lane; i < ell; i += 32) dot += W[i * ld + j] * W[i * ld + c];
    dot = warp_sum(dot);
    dot += W[j * ld + c];
    const double f = tau * dot;
    if (lane == 0) W[j * ld + c] -= f;
    for (int i = j + 1 + lane; i < ell; i += 32) W[i * ld + c] -= f * W[i * ld + j];
}

__global__ void __launch_bounds__(kQrcpThreads)
qrcp_kernel(const double* d, int ell, double* qt, double* rt, int* perm, const int* cancel) {
    if (cancel && *cancel) return;
    extern __shared__ double W[];  // ell x (ell + 1) row-major, then nrm[ell], tau[ell], sgn[ell]
    const int ld = ell + 1;
    double* nrm = W + ell * ld;
    double* tau = nrm + ell;
    double* sgn = tau + ell;
    int* pv = reinterpret_cast<int*>(sgn + ell);
    __shared__ int piv_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < ell * ell; e += kQrcpThreads) W[(e / ell) * ld + (e % ell)] = d[e];
    for (int c = tid; c < ell; c += kQrcpThreads) pv[c] = c;
    __syncthreads();
    for (int j = 0; j < ell; ++j) {
        // 1. recomputed residual norms of the trailing columns
        for (int c = j + warp; c < ell; c += kQrcpWarps) {
            double s = 0.0;
            for (int i = j + lane; i < ell; i += 32) s += W[i * ld + c] * W[i * ld + c];
            s = warp_sum(s);
            if (lane == 0) nrm[c] = s;
        }
        __syncthreads();
        // 2. pivot = argmax, lowest index on ties
        if (warp == 0) {
            double best = -1.0;
            int bi = ell;
            for (int c = j + lane; c < ell; c += 32) {
                const double v = nrm[c];
                if (v > best) { best = v; bi = c; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) piv_s = bi;
        }
        __syncthreads();
        const int p = piv_s;
        // 3. swap columns j and p
        if (p != j) {
            for (int i = tid; i < ell; i += kQrcpThreads) {
                const double tmp = W[i * ld + j];
                W[i * ld + j] = W[i * ld + p];
                W[i * ld + p] = tmp;
            }
            if (tid == 0) {
                const int t = pv[j];
                pv[j] = pv[p];
                pv[p] = t;
            }
        }
        __syncthreads();
        // 4. Householder reflector of column j (warp 0)
        if (warp == 0) {
            const double alpha = W[j * ld + j];
            double x2 = 0.0;
            for (int i = j + 1 + lane; i < ell; i += 32) x2 += W[i * ld + j] * W[i * ld + j];
            x2 = warp_sum(x2);
            double t = 0.0;
            if (x2 > 0.0) {
                const double nr = sqrt(alpha * alpha + x2);
                const double beta = alpha >= 0.0 ? -nr : nr;
                t = (beta - alpha) / beta;
                const double scale = 1.0 / (alpha - beta);
                for (int i = j + 1 + lane; i < ell; i += 32) W[i * ld + j] *= scale;
                if (lane == 0) W[j * ld + j] = beta;
            }
            if (lane == 0) tau[j] = t;
        }
        __syncthreads();
        // 5. apply it to the trailing columns
        const double tj = tau[j];
        if (tj != 0.0)
            for (int c = j + 1 + warp; c < ell; c += kQrcpWarps) house_apply_col(W, ld, ell, j, c, tj, lane);
        __syncthreads();
    }
    // Rt = upper(W) with diag(Rt) >= 0
    for (int a = tid; a < ell; a += kQrcpThreads) sgn[a] = W[a * ld + a] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;
        rt[e] = (b >= a) ? sgn[a] * W[a * ld + b] : 0.0;
    }
    for (int c = tid; c < ell; c += kQrcpThreads) perm[c] = pv[c];
    __syncthreads();
    // Qt = H_0 H_1 ... H_{ell-1} formed in place (backward accumulation)
    for (int j = ell - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (j < ell - 1 && tj != 0.0)
            for (int c = j + 1 + warp; c < ell; c += kQrcpWarps) house_apply_col(W, ld, ell, j, c, tj, lane);
        __syncthreads();
        for (int i = tid; i < ell; i += kQrcpThreads) {
            if (i > j) W[i * ld + j] *= -tj;
            else if (i == j) W[j * ld + j] = 1.0 - tj;
            else W[i * ld + j] = 0.0;
        }
        __syncthreads();
    }
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;
        qt[e] = W[a * ld + b] * sgn[b];
    }
}

template <typename TV>
__global__ void gather_v_kernel(const double* q2, int64_t ldq2, int64_t n, int ell, const int* perm,
                                TV* v, int64_t ldv, const int* cancel) {
    if (cancel && *cancel) return;
    __shared__ double tile[128][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int tid = threadIdx.x;  // 256
    for (int e = tid; e < ell * 32; e += blockDim.x) {
        const int j = e / 32, ii = e % 32;
        const int64_t i = i0 + ii;
        tile[j][ii] = (i < n) ? q2[(int64_t)perm[j] * ldq2 + i] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < ell * 32; e += blockDim.x) {
        const int ii = e / ell, j = e % ell;
        const int64_t i = i0 + ii;
        if (i < n) v[i * ldv + j] = (TV)tile[j][ii];
    }
}

template <typename TD>
__global__ void copy_small_kernel(const double* src, int n, TD* dst, const int* cancel) {
    if (cancel && *cancel) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        dst[e] = (TD)src[e];
}

}  // namespace

cudaError_t launch_cholesky(const double* g, int64_t ell, int64_t rows, double* r, int* flags,
                               int* skip_out, const int* cancel, cudaStream_t st) {
    const size_t smem = sizeof(double) * (size_t)ell * (ell + 1);
    cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    cholesky_kernel<<<1, kCholThreads, smem, st>>>(g, (int)ell, rows, r, flags, skip_out, cancel);
    return cudaGetLastError();
}

cudaError_t launch_trsm_rows(const double* c, int64_t ldc, int64_t rows, int64_t ell,
                             const double* r, ElemType tc, double* q, int64_t ldq, void* qc,
                             ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st) {
    if (tc == T_F64) {
        if (!qc || tqc == T_F64)
            return trsm_launch<double, double>(c, ldc, rows, (int)ell, r, q, ldq, static_cast<double*>(qc),
                                               ldqc, cancel, st);
        if (tqc == T_F32)
            return trsm_launch<double, float>(c, ldc, rows, (int)ell, r, q, ldq, static_cast<float*>(qc),
                                              ldqc, cancel, st);
        return trsm_launch<double, __nv_bfloat16>(c, ldc, rows, (int)ell, r, q, ldq,
                                                  static_cast<__nv_bfloat16*>(qc), ldqc, cancel, st);
    }
    if (!qc || tqc == T_F32)
        return trsm_launch<float, float>(c, ldc, rows, (int)ell, r, q, ldq, static_cast<float*>(qc), ldqc,
                                         cancel, st);
    if (tqc == T_F64)
        return trsm_launch<float, double>(c, ldc, rows, (int)ell, r, q, ldq, static_cast<double*>(qc),
                                          ldqc, cancel, st);
    return trsm_launch<float, __nv_bfloat16>(c, ldc, rows, (int)ell, r, q, ldq,
                                             static_cast<__nv_bfloat16*>(qc), ldqc, cancel, st);
}

cudaError_t launch_qrcp(const double* d, int64_t ell, double* qt, double* rt, int* perm,
                        const int* cancel, cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)ell * (ell + 1) + 3 * (size_t)ell) + sizeof(int) * ell;
    cudaError_t e = cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    qrcp_kernel<<<1, kQrcpThreads, smem, st>>>(d, (int)ell, qt, rt, perm, cancel);
    return cudaGetLastError();
}

cudaError_t launch_gather_v(const double* q2, int64_t ldq2, int64_t n, int64_t ell, const int* perm,
                            void* v, ElemType tv, int64_t ldv, const int* cancel, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 31) / 32);
    if (tv == T_F64) {
        count_launch();
        gather_v_kernel<double><<<blocks, 256, 0, st>>>(q2, ldq2, n, (int)ell, perm, static_cast<double*>(v),
                                                        ldv, cancel);
    } else {
        count_launch();
        gather_v_kernel<float><<<blocks, 256, 0, st>>>(q2, ldq2, n, (int)ell, perm, static_cast<float*>(v),
                                                       ldv, cancel);
    }
    return cudaGetLastError();
}

cudaError_t launch_copy_small(const double* src, int64_t ell, void* dst, ElemType tdst,
                              const int* cancel, cudaStream_t st) {
    const int n = (int)(ell * ell);
    if (tdst == T_F64) {
        count_launch();
        copy_small_kernel<double><<<(n + 255) / 256, 256, 0, st>>>(src, n, static_cast<double*>(dst), cancel);
    } else {
        count_launch();
        copy_small_kernel<float><<<(n + 255) / 256, 256, 0, st>>>(src, n, static_cast<float*>(dst), cancel);
    }
    return cudaGetLastError();
}

}  // namespace corutv
