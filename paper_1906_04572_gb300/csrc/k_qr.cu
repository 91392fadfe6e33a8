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

// ---------------------------------------------------------------------------
// FP64 reciprocal and reciprocal square root without the FP64 divide / sqrt
// sequences (each several hundred cycles on this part): an FP32 estimate on
// the operand scaled into FP32 range by a power of two, then two
// Newton-Raphson steps in FP64, each squaring the relative error
// (about 2^-23 -> 2^-46 -> 2^-92, so the result is within a few ulp).
//   1/sqrt(x): y <- y (3/2 - (x/2) y^2)
//   1/x      : y <- y + y (1 - x y)
// For normal, finite, nonzero operands (1/sqrt: positive); others fall back
// to the library operations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double scale_pow2(double x, int k) {  // x * 2^k, k within the exponent range
    return __hiloint2double(__double2hiint(x) + (k << 20), __double2loint(x));
}

__device__ __forceinline__ double rsqrt_nr(double x) {
    const int ef = (__double2hiint(x) >> 20) & 0x7ff;
    if (ef == 0 || ef == 0x7ff || x < 0.0) return 1.0 / sqrt(x);
    const int k = (ef - 1023) >> 1;            // x = xs 2^(2k), xs in [1, 4)
    const double xs = scale_pow2(x, -2 * k);
    double y = (double)rsqrtf((float)xs);
    const double hx = 0.5 * xs;
    y = y * fma(-hx, y * y, 1.5);
    y = y * fma(-hx, y * y, 1.5);
    return scale_pow2(y, -k);
}

__device__ __forceinline__ double rcp_nr(double x) {
    const int ef = (__double2hiint(x) >> 20) & 0x7ff;
    if (ef == 0 || ef == 0x7ff) return 1.0 / x;
    const int k = ef - 1023;                   // x = xs 2^k, |xs| in [1, 2)
    const double xs = scale_pow2(x, -k);
    double y = (double)__frcp_rn((float)xs);
    y = fma(y, fma(-xs, y, 1.0), y);
    y = fma(y, fma(-xs, y, 1.0), y);
    return scale_pow2(y, -k);
}

constexpr int kCholThreads = 128;  // one warp per SM sub-partition (each has its own FP64 unit)

// Right-looking Cholesky, upper factor, R^T R = G (+ shift I), one column at
// a time: every warp derives 1/r_jj itself (no extra barrier), row j is
// scaled, then the trailing upper triangle takes the rank-1 update with
// rows spread over the four warps and columns over the lanes.
// rows = number of rows of the matrix whose Gram is factorised (for the shift).
__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* g, int ell, int64_t rows, double* r, int* flags, int* skip_out,
                const int* cancel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kCholThreads / 32;
    if (cancel && *cancel) {
        if (skip_out && tid == 0) *skip_out = 1;
        return;
    }
    extern __shared__ double S[];  // ell x (ell + 1), upper triangle used
    const int ld = ell + 1;
    __shared__ double trace;
    int attempt = 0;
    bool fail = false;
    for (; attempt < 3; ++attempt) {
        double shift = 0.0;
        if (attempt > 0) {
            // shift s = 11 (rows ell + ell (ell + 1)) u ||C||_F^2 (u = 2^-53), then x100;
            // ||C||_F^2 = trace(G), summed only when a shift is needed
            if (tid == 0) {
                double t = 0.0;
                for (int a = 0; a < ell; ++a) t += g[a * ell + a];
                trace = t;
            }
            __syncthreads();
            const double u = 1.1102230246251565e-16;
            shift = 11.0 * ((double)rows * ell + (double)ell * (ell + 1)) * u * trace * (attempt == 1 ? 1.0 : 100.0);
        }
        for (int e = tid; e < ell * ell; e += kCholThreads) {
            const int a = e / ell, b = e % ell;
            S[a * ld + b] = g[a * ell + b] + (a == b ? shift : 0.0);
        }
        __syncthreads();
        fail = false;
        for (int j = 0; j < ell; ++j) {
            const double d = S[j * ld + j];  // same value in every thread
            if (!(d > 0.0) || !isfinite(d)) {
                fail = true;
                break;
            }
            const double y = rsqrt_nr(d);  // 1 / r_jj
            for (int c = j + 1 + tid; c < ell; c += kCholThreads) S[j * ld + c] *= y;
            __syncthreads();
            if (tid == 0) S[j * ld + j] = d * y;
            for (int a = j + 1 + warp; a < ell; a += nwarps) {
                const double sja = S[j * ld + a];
                for (int c = a + lane; c < ell; c += 32) S[a * ld + c] -= sja * S[j * ld + c];
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
    TC* Rd = Ts + (size_t)ell * nthr;             // 1 / R[j][j]
    const int tid = threadIdx.x;
    for (int e = tid; e < ell * ell; e += nthr) Rs[e] = (TC)r[e];
    for (int j = tid; j < ell; j += nthr) Rd[j] = (TC)(1.0 / r[j * ell + j]);
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
        Ts[j * nthr + tid] = (s0 + s1) * Rd[j];
    }
    for (int j = 0; j < ell; ++j) {
        const TC v = Ts[j * nthr + tid];
        q[j * ldq + i] = (double)v;
        if (qc) qc[j * ldqc + i] = (TQC)v;
    }
}

// Threads (= rows) per block: up to 256, bounded by shared memory. A row's
// solve is a dependent chain, so larger blocks mainly serve to load R once
// per 256 rows.
template <typename TC>
int trsm_threads(int ell, int64_t rows) {
    const long budget = 200 * 1024;
    long per = (budget - (long)ell * (ell + 1) * (long)sizeof(TC)) / ((long)ell * (long)sizeof(TC));
    per = per / 32 * 32;
    if (per > 256) per = 256;
    if (per < 32) per = 32;
    (void)rows;
    return (int)per;
}

template <typename TC, typename TQC>
cudaError_t trsm_launch(const double* c, int64_t ldc, int64_t rows, int ell, const double* r,
                        double* q, int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel,
                        cudaStream_t st) {
    const int nthr = trsm_threads<TC>(ell, rows);
    const size_t smem = sizeof(TC) * ((size_t)ell * ell + (size_t)ell * nthr + (size_t)ell);
    cudaError_t e = cudaFuncSetAttribute(trsm_rows_kernel<TC, TQC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((rows + nthr - 1) / nthr);
    count_launch();
    trsm_rows_kernel<TC, TQC><<<blocks, nthr, smem, st>>>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// QRCP of the small D (eq. 8), one block of four warps (one per SM
// sub-partition, each with its own FP64 unit). W is column-major in shared
// memory (column c at W + c * ldw, ldw odd so that lanes owning consecutive
// columns hit distinct banks). Column-wise work (squared norms, reflector
// dot products and updates) is split as lanes = columns, warps = quarters of
// the active rows; partial sums meet in shared memory in warp order.
// Pivot choice compares the non-negative squared norms through their bit
// patterns (same order as the values), lowest index on ties.
// ---------------------------------------------------------------------------
constexpr int kQrcpThreads = 128;
constexpr int kQrcpWarps = kQrcpThreads / 32;

// rows [lo, hi) of the active range [j, ell) owned by warp w
__device__ __forceinline__ void quarter(int j, int ell, int w, int& lo, int& hi) {
    const int n = ell - j;
    const int qn = (n + kQrcpWarps - 1) / kQrcpWarps;
    lo = j + w * qn;
    hi = min(ell, lo + qn);
    if (lo > ell) lo = ell;
}

// Apply H_j = I - tau v v^T (v = [1; W[j][j+1:]]) to columns c0..ell-1, rows j..ell-1.
__device__ void apply_reflector(double* W, int ldw, double* part, int j, int c0, int ell, double tau, int lane,
                                int warp) {
    const double* v = W + j * ldw;
    int lo, hi;
    quarter(j, ell, warp, lo, hi);
    for (int cb = c0; cb < ell; cb += 32) {
        const int c = cb + lane;
        if (c < ell) {
            const double* x = W + c * ldw;
            double s0 = 0.0, s1 = 0.0;
            int i = lo;
            if (i == j && i < hi) { s0 = x[j]; ++i; }  // v[j] = 1
            for (; i + 1 < hi; i += 2) {
                s0 += v[i] * x[i];
                s1 += v[i + 1] * x[i + 1];
            }
            if (i < hi) s0 += v[i] * x[i];
            part[warp * 128 + (c - cb)] = s0 + s1;
        }
        __syncthreads();
        if (c < ell) {
            double dot = part[c - cb];
            for (int w = 1; w < kQrcpWarps; ++w) dot += part[w * 128 + (c - cb)];
            const double f = tau * dot;
            double* x = W + c * ldw;
            int i = lo;
            if (i == j && i < hi) { x[j] -= f; ++i; }
            for (; i < hi; ++i) x[i] -= f * v[i];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kQrcpThreads)
qrcp_kernel(const double* d, int ell, double* qt, double* rt, int* perm, const int* cancel) {
    if (cancel && *cancel) return;
    extern __shared__ double W[];  // ell columns of ldw doubles, then part, nrm, tau, sgn, perm
    const int ldw = ell | 1;
    double* part = W + ell * ldw;           // kQrcpWarps x 128
    double* nrm = part + kQrcpWarps * 128;  // ell
    double* tau = nrm + ell;
    double* sgn = tau + ell;
    int* pv = reinterpret_cast<int*>(sgn + ell);
    __shared__ int piv_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;  // d row-major: entry (a, b) -> column b, row a
        W[b * ldw + a] = d[e];
    }
    for (int c = tid; c < ell; c += kQrcpThreads) pv[c] = c;
    __syncthreads();
    for (int j = 0; j < ell; ++j) {
        int lo, hi;
        quarter(j, ell, warp, lo, hi);
        // 1. recomputed squared residual norms of columns j..ell-1
        for (int cb = j; cb < ell; cb += 32) {
            const int c = cb + lane;
            if (c < ell) {
                const double* x = W + c * ldw;
                double s0 = 0.0, s1 = 0.0;
                int i = lo;
                for (; i + 1 < hi; i += 2) {
                    s0 += x[i] * x[i];
                    s1 += x[i + 1] * x[i + 1];
                }
                if (i < hi) s0 += x[i] * x[i];
                part[warp * 128 + (c - j)] = s0 + s1;
            }
        }
        __syncthreads();
        // 2. pivot: warp 0 adds the quarters (warp order) and takes the argmax
        if (warp == 0) {
            long long best = -1;
            int bi = ell;
            for (int c = j + lane; c < ell; c += 32) {
                double s = part[c - j];
                for (int w = 1; w < kQrcpWarps; ++w) s += part[w * 128 + (c - j)];
                nrm[c] = s;
                const long long key = __double_as_longlong(s);
                if (key > best) { best = key; bi = c; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) piv_s = bi;
        }
        __syncthreads();
        const int p = piv_s;
        // 3. swap columns j and p (whole columns)
        if (p != j) {
            for (int i = tid; i < ell; i += kQrcpThreads) {
                const double t = W[j * ldw + i];
                W[j * ldw + i] = W[p * ldw + i];
                W[p * ldw + i] = t;
            }
            if (tid == 0) {
                const int t = pv[j];
                pv[j] = pv[p];
                pv[p] = t;
                const double tn = nrm[j];
                nrm[j] = nrm[p];
                nrm[p] = tn;
            }
            __syncthreads();
        }
        // 4. reflector of column j from its squared norm s = alpha^2 + |x|^2:
        //    beta = -sign(alpha) sqrt(s), tau = 1 - alpha / beta,
        //    v[i] = x[i] / (alpha - beta); H = I when x is exactly zero.
        {
            double* x = W + j * ldw;
            const double alpha = x[j];
            const double s = nrm[j];
            double t = 0.0;
            if (s != alpha * alpha) {
                const double y = rsqrt_nr(s);            // 1 / |column|
                const double nr = s * y;
                const double beta = alpha >= 0.0 ? -nr : nr;
                const double inv_beta = alpha >= 0.0 ? -y : y;
                t = fma(-alpha, inv_beta, 1.0);
                const double scale = rcp_nr(alpha - beta);
                for (int i = j + 1 + tid; i < ell; i += kQrcpThreads) x[i] *= scale;
                __syncthreads();
                if (tid == 0) x[j] = beta;
            }
            if (tid == 0) tau[j] = t;
            __syncthreads();
        }
        // 5. apply it to the trailing columns
        const double tj = tau[j];
        if (tj != 0.0 && j + 1 < ell) apply_reflector(W, ldw, part, j, j + 1, ell, tj, lane, warp);
    }
    // Rt = upper(W) with diag(Rt) >= 0
    for (int a = tid; a < ell; a += kQrcpThreads) sgn[a] = W[a * ldw + a] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;
        rt[e] = (b >= a) ? sgn[a] * W[b * ldw + a] : 0.0;
    }
    for (int c = tid; c < ell; c += kQrcpThreads) perm[c] = pv[c];
    __syncthreads();
    // Qt = H_0 H_1 ... H_{ell-1}, accumulated backwards in place
    for (int j = ell - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (j < ell - 1 && tj != 0.0) apply_reflector(W, ldw, part, j, j + 1, ell, tj, lane, warp);
        double* x = W + j * ldw;
        for (int i = tid; i < ell; i += kQrcpThreads) {
            if (i > j) x[i] *= -tj;
            else if (i == j) x[j] = 1.0 - tj;
            else x[i] = 0.0;
        }
        __syncthreads();
    }
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;
        qt[e] = W[b * ldw + a] * sgn[b];
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
    const size_t smem = sizeof(double) * ((size_t)ell * (ell | 1) + 4 * 128 + 3 * (size_t)ell) + sizeof(int) * ell;
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
