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
// a time, with a one-step lookahead. The upper triangle is enumerated row by
// row from the bottom row up, columns right to left (table `tri`), so the
// trailing triangle of step j (rows > j) is a contiguous prefix of length
// (ell-j-1)(ell-j)/2 whose last entry is the next pivot (j+1, j+1). Step j:
// all threads scale row j by 1/r_jj (computed one step earlier); then warp 0
// forms the next pivot d = G'(j+1,j+1) - r(j,j+1)^2, checks it and computes
// 1/sqrt(d), while warps 1-3 apply the rank-1 update to the rest of the
// prefix with every lane busy.
// rows = number of rows of the matrix whose Gram is factorised (for the shift).
__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* g, int ell, int64_t rows, double* r, int* flags, int* skip_out,
                const int* cancel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (cancel && *cancel) {
        if (skip_out && tid == 0) *skip_out = 1;
        return;
    }
    extern __shared__ double S[];  // ell x (ell + 1) doubles, then the uint16 table
    const int ld = ell + 1;
    unsigned short* tri = reinterpret_cast<unsigned short*>(S + (size_t)ell * ld);
    __shared__ double trace, ynext;
    __shared__ int fail_s;
    // table: bottom-up rows; row a holds columns ell-1 .. a
    for (int a = ell - 1 - tid; a >= 0; a -= kCholThreads) {
        const int rb = ell - 1 - a;            // rows below the top of the enumeration
        int e = rb * (rb + 1) / 2;
        for (int c = ell - 1; c >= a; --c) tri[e++] = (unsigned short)((a << 8) | c);
    }
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
        if (tid == 0) {
            const double d0 = g[0] + shift;
            fail_s = !(d0 > 0.0) || !isfinite(d0);
            ynext = fail_s ? 0.0 : rsqrt_nr(d0);
        }
        __syncthreads();
        fail = fail_s != 0;
        for (int j = 0; j < ell && !fail; ++j) {
            const double y = ynext;  // 1 / r_jj
            for (int c = j + 1 + tid; c < ell; c += kCholThreads) S[j * ld + c] *= y;
            if (tid == 0) S[j * ld + j] *= y;  // d_jj / sqrt(d_jj) = r_jj
            __syncthreads();
            if (j + 1 < ell) {
                if (warp == 0) {
                    if (lane == 0) {
                        const double s = S[j * ld + j + 1];
                        const double d = fma(-s, s, S[(j + 1) * ld + j + 1]);
                        S[(j + 1) * ld + j + 1] = d;
                        const bool bad = !(d > 0.0) || !isfinite(d);
                        if (bad) fail_s = 1;
                        else ynext = rsqrt_nr(d);
                    }
                } else {
                    const int len = (ell - j - 1) * (ell - j) / 2 - 1;  // prefix without (j+1, j+1)
                    for (int e = tid - 32; e < len; e += kCholThreads - 32) {
                        const int ac = tri[e];
                        const int a = ac >> 8, c = ac & 0xff;
                        S[a * ld + c] = fma(-S[j * ld + a], S[j * ld + c], S[a * ld + c]);
                    }
                }
            }
            __syncthreads();
            fail = fail_s != 0;
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
// Columns are solved in blocks of kTrsmB: the contributions of the columns
// already solved go into kTrsmB independent accumulators (one shared load of
// q_i[t] feeds all of them), then the small triangle inside the block is
// finished in order. Row i is held in shared memory (one thread per row).
constexpr int kTrsmB = 8;
template <typename TI, typename TC, typename TQC>
__global__ void trsm_rows_kernel(const TI* c, int64_t ldc, int64_t rows, int ell, const double* r,
                                 TI* q, int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel) {
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* Rs = reinterpret_cast<TC*>(smem_raw);   // ell x ell row-major
    const int nthr = blockDim.x;
    TC* Ts = Rs + ell * ell;                      // [ell][nthr]
    TC* Rd = Ts + (size_t)ell * nthr;             // 1 / R[j][j]
    const int tid = threadIdx.x;
    for (int e = tid; e < ell * ell; e += nthr) Rs[e] = (TC)r[e];
    for (int j = tid; j < ell; j += nthr) Rd[j] = (TC)1 / (TC)r[j * ell + j];
    const int64_t i = (int64_t)blockIdx.x * nthr + tid;
    if (i < rows)
        for (int j = 0; j < ell; ++j) Ts[j * nthr + tid] = (TC)c[j * ldc + i];
    __syncthreads();
    if (i >= rows) return;
    for (int j0 = 0; j0 < ell; j0 += kTrsmB) {
        const int nb = min(kTrsmB, ell - j0);
        TC acc[kTrsmB];
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k) acc[k] = (k < nb) ? Ts[(j0 + k) * nthr + tid] : (TC)0;
        for (int t = 0; t < j0; ++t) {
            const TC qt = Ts[t * nthr + tid];
            const TC* rrow = Rs + t * ell + j0;
#pragma unroll
            for (int k = 0; k < kTrsmB; ++k)
                if (k < nb) acc[k] -= qt * rrow[k];
        }
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k) {
            if (k >= nb) break;
            TC s = acc[k];
#pragma unroll
            for (int kk = 0; kk < k; ++kk) s -= acc[kk] * Rs[(j0 + kk) * ell + j0 + k];
            acc[k] = s * Rd[j0 + k];
        }
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k)
            if (k < nb) Ts[(j0 + k) * nthr + tid] = acc[k];
    }
    for (int j = 0; j < ell; ++j) {
        const TC v = Ts[j * nthr + tid];
        q[j * ldq + i] = (TI)v;
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

template <typename TI, typename TC, typename TQC>
cudaError_t trsm_launch(const void* c, int64_t ldc, int64_t rows, int ell, const double* r, void* q, int64_t ldq,
                        void* qc, int64_t ldqc, const int* cancel, cudaStream_t st) {
    const int nthr = trsm_threads<TC>(ell, rows);
    const size_t smem = sizeof(TC) * ((size_t)ell * ell + (size_t)ell * nthr + (size_t)ell);
    cudaError_t e = cudaFuncSetAttribute(trsm_rows_kernel<TI, TC, TQC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((rows + nthr - 1) / nthr);
    count_launch();
    trsm_rows_kernel<TI, TC, TQC><<<blocks, nthr, smem, st>>>(static_cast<const TI*>(c), ldc, rows, ell, r,
                                                              static_cast<TI*>(q), ldq, static_cast<TQC*>(qc),
                                                              ldqc, cancel);
    return cudaGetLastError();
}

template <typename TI, typename TC>
cudaError_t trsm_dispatch(const void* c, int64_t ldc, int64_t rows, int ell, const double* r, void* q,
                          int64_t ldq, void* qc, ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st) {
    if (!qc) return trsm_launch<TI, TC, TI>(c, ldc, rows, ell, r, q, ldq, nullptr, 0, cancel, st);
    switch (tqc) {
        case T_F64: return trsm_launch<TI, TC, double>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st);
        case T_F32: return trsm_launch<TI, TC, float>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st);
        case T_BF16: return trsm_launch<TI, TC, __nv_bfloat16>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// QRCP of the small D (eq. 8), one block of four warps (one per SM
// sub-partition, each sub-partition with its own FP64 unit). W is column-major in shared
// memory (column c at W + c * ldw, ldw odd so that lanes owning consecutive
// columns hit distinct banks). Column-wise work (squared norms, reflector
// dot products and updates) is split as lanes = columns, warps = quarters of
// the active rows; partial sums meet in shared memory in warp order.
// Pivot choice compares the non-negative squared norms through their bit
// patterns (same order as the values), lowest index on ties.
// ---------------------------------------------------------------------------
constexpr int kQrcpThreads = 128;  // one warp per sub-partition (a second one per sub-partition measured slower)
constexpr int kQrcpWarps = kQrcpThreads / 32;

// rows [lo, hi) of the active range [j, ell) owned by warp w (one of kQrcpWarps shares)
__device__ __forceinline__ void row_share(int j, int ell, int w, int& lo, int& hi) {
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
    row_share(j, ell, warp, lo, hi);
    for (int cb = c0; cb < ell; cb += 32) {
        const int c = cb + lane;
        if (c < ell) {
            const double* x = W + c * ldw;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int i = lo;
            if (i == j && i < hi) { s0 = x[j]; ++i; }  // v[j] = 1
            for (; i + 3 < hi; i += 4) {
                s0 += v[i] * x[i];
                s1 += v[i + 1] * x[i + 1];
                s2 += v[i + 2] * x[i + 2];
                s3 += v[i + 3] * x[i + 3];
            }
            for (; i < hi; ++i) s0 += v[i] * x[i];
            part[warp * 128 + (c - cb)] = (s0 + s1) + (s2 + s3);
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
        row_share(j, ell, warp, lo, hi);
        // 1. recomputed squared residual norms of columns j..ell-1
        for (int cb = j; cb < ell; cb += 32) {
            const int c = cb + lane;
            if (c < ell) {
                const double* x = W + c * ldw;
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int i = lo;
                for (; i + 3 < hi; i += 4) {
                    s0 += x[i] * x[i];
                    s1 += x[i + 1] * x[i + 1];
                    s2 += x[i + 2] * x[i + 2];
                    s3 += x[i + 3] * x[i + 3];
                }
                for (; i < hi; ++i) s0 += x[i] * x[i];
                part[warp * 128 + (c - j)] = (s0 + s1) + (s2 + s3);
            }
        }
        __syncthreads();
        // 2. pivot: warp 0 adds the shares (warp order) and takes the argmax
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

template <typename TQ, typename TV>
__global__ void gather_v_kernel(const TQ* q2, int64_t ldq2, int64_t n, int ell, const int* perm,
                                TV* v, int64_t ldv, const int* cancel) {
    if (cancel && *cancel) return;
    __shared__ double tile[128][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int tid = threadIdx.x;  // 256
    for (int e = tid; e < ell * 32; e += blockDim.x) {
        const int j = e / 32, ii = e % 32;
        const int64_t i = i0 + ii;
        tile[j][ii] = (i < n) ? (double)q2[(int64_t)perm[j] * ldq2 + i] : 0.0;
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
    const size_t smem = sizeof(double) * (size_t)ell * (ell + 1) + sizeof(unsigned short) * (size_t)ell * (ell + 1) / 2;
    cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    cholesky_kernel<<<1, kCholThreads, smem, st>>>(g, (int)ell, rows, r, flags, skip_out, cancel);
    return cudaGetLastError();
}

cudaError_t launch_trsm_rows(const void* c, ElemType tp, int64_t ldc, int64_t rows, int64_t ell,
                             const double* r, ElemType tc, void* q, int64_t ldq, void* qc,
                             ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st) {
    const int l = (int)ell;
    if (tp == T_F64 && tc == T_F64) return trsm_dispatch<double, double>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st);
    if (tp == T_F64 && tc == T_F32) return trsm_dispatch<double, float>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st);
    if (tp == T_F32 && tc == T_F32) return trsm_dispatch<float, float>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_qrcp(const double* d, int64_t ell, double* qt, double* rt, int* perm,
                        const int* cancel, cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)ell * (ell | 1) + kQrcpWarps * 128 + 3 * (size_t)ell) + sizeof(int) * ell;
    cudaError_t e = cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    qrcp_kernel<<<1, kQrcpThreads, smem, st>>>(d, (int)ell, qt, rt, perm, cancel);
    return cudaGetLastError();
}

cudaError_t launch_gather_v(const void* q2, ElemType tq2, int64_t ldq2, int64_t n, int64_t ell, const int* perm,
                            void* v, ElemType tv, int64_t ldv, const int* cancel, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 31) / 32);
    count_launch();
    if (tq2 == T_F64 && tv == T_F64)
        gather_v_kernel<double, double><<<blocks, 256, 0, st>>>(static_cast<const double*>(q2), ldq2, n, (int)ell,
                                                                perm, static_cast<double*>(v), ldv, cancel);
    else if (tq2 == T_F64)
        gather_v_kernel<double, float><<<blocks, 256, 0, st>>>(static_cast<const double*>(q2), ldq2, n, (int)ell,
                                                               perm, static_cast<float*>(v), ldv, cancel);
    else if (tv == T_F64)
        gather_v_kernel<float, double><<<blocks, 256, 0, st>>>(static_cast<const float*>(q2), ldq2, n, (int)ell,
                                                               perm, static_cast<double*>(v), ldv, cancel);
    else
        gather_v_kernel<float, float><<<blocks, 256, 0, st>>>(static_cast<const float*>(q2), ldq2, n, (int)ell,
                                                              perm, static_cast<float*>(v), ldv, cancel);
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
