// SIMT kernels of libcorutv:
//  * the generic skinny product out = Aop^T Bop (FP64 or FP32 FMA) used for
//    the FP64 / FP32 passes over A (eqs. 4, 5, 7), the Gram matrices of
//    CholeskyQR, D = Q1^T W and U = Q1 Qt (eq. 9);
//  * the fixed-order reduction of split-K partial products;
//  * step 1 of Algorithm 1: the Philox-4x32-10 Gaussian test matrix;
//  * layout / precision conversions of the tall-skinny panels.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace corutv {

namespace {

constexpr int kThreads = 256;
constexpr int kBM = 64;
constexpr int kBK = 32;
constexpr int kTM = 4;

template <typename T>
__device__ __forceinline__ T zero_of() { return T(0); }

template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI v) { return static_cast<TO>(v); }
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}
// double -> bf16 rounded to nearest even in one step: round toward zero to
// float, mark an inexact result in the last float bit (round to odd), then
// round to bf16. The float keeps 16 more bits than bf16, so the odd bit only
// breaks ties the way exact rounding would.
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, double>(double v) {
    float f = __double2float_rz(v);
    if ((double)f != v && isfinite(v)) f = __uint_as_float(__float_as_uint(f) | 1u);
    return __float2bfloat16_rn(f);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16, float>(float v) { return __float2bfloat16(v); }

// out[r][j] = sum_k Aop[k][r] Bop[k][j] over the split's k range.
// Tiles of kBM output rows x (16 TN) columns, kBK k per stage; 256 threads,
// each owns kTM rows x TN columns (columns tx, tx+16, ... to avoid bank
// conflicts on the B tile).
template <typename TA, typename TB, typename TC, int TN>
__global__ void __launch_bounds__(kThreads) gemm_simt_kernel(GemmArgs g) {
    pdl_trigger();
    pdl_wait();
    if (g.cancel && *g.cancel) return;
    constexpr int LP = 16 * TN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* As = reinterpret_cast<TC*>(smem_raw);                 // [kBK][kBM + 1]
    TC* Bs = As + kBK * (kBM + 1);                            // [kBK][LP + 1]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * kBM;
    const int split = blockIdx.y;
    const int64_t kper = ((g.K + g.splits - 1) / g.splits + kBK - 1) / kBK * kBK;
    const int64_t kbeg = (int64_t)split * kper;
    const int64_t kend = (g.K < kbeg + kper) ? g.K : kbeg + kper;
    const TA* A = static_cast<const TA*>(g.a);
    const TB* B = static_cast<const TB*>(g.b);
    const bool a_kfast = (g.amode == A_ROWS || g.amode == A_PANEL_T);

    TC acc[kTM][TN];
#pragma unroll
    for (int i = 0; i < kTM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = zero_of<TC>();

    for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
        for (int idx = tid; idx < kBM * kBK; idx += kThreads) {
            int r, k;
            if (a_kfast) { r = idx / kBK; k = idx % kBK; } else { k = idx / kBM; r = idx % kBM; }
            const int64_t gr = r0 + r, gk = k0 + k;
            TC v = zero_of<TC>();
            if (gr < g.R && gk < kend) {
                const int64_t off = a_kfast ? gr * g.lda + gk : gk * g.lda + gr;
                v = cvt<TC>(A[off]);
            }
            As[k * (kBM + 1) + r] = v;
        }
        for (int idx = tid; idx < kBK * LP; idx += kThreads) {
            int j, k;
            if (g.bmode == B_PANEL) { j = idx / kBK; k = idx % kBK; } else { k = idx / LP; j = idx % LP; }
            const int64_t gk = k0 + k;
            TC v = zero_of<TC>();
            if (j < g.L && gk < kend) v = cvt<TC>((g.bmode == B_PANEL) ? B[j * g.ldb + gk] : B[gk * g.ldb + j]);
            Bs[k * (LP + 1) + j] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kBK; ++k) {
            TC av[kTM], bv[TN];
#pragma unroll
            for (int i = 0; i < kTM; ++i) av[i] = As[k * (kBM + 1) + ty * kTM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[k * (LP + 1) + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < kTM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    TC* out = static_cast<TC*>(g.out) + (int64_t)split * g.split_stride;
#pragma unroll
    for (int i = 0; i < kTM; ++i) {
        const int64_t r = r0 + ty * kTM + i;
        if (r >= g.R) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t c = tx + 16 * j;
            if (c >= g.L) continue;
            out[g.omode == O_PANEL ? c * g.ldo + r : r * g.ldo + c] = acc[i][j];
        }
    }
}

template <typename TA, typename TB, typename TC, int TN>
cudaError_t launch_tn(const GemmArgs& g, cudaStream_t st) {
    const size_t smem = sizeof(TC) * (size_t)(kBK * (kBM + 1) + kBK * (16 * TN + 1));
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(gemm_simt_kernel<TA, TB, TC, TN>));
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.R + kBM - 1) / kBM), (unsigned)g.splits);
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(gemm_simt_kernel<TA, TB, TC, TN>, dim3(grid), dim3(kThreads), (size_t)(smem), st, g);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

template <typename TA, typename TB, typename TC>
cudaError_t launch_types(const GemmArgs& g, cudaStream_t st) {
    if (g.L <= 16) return launch_tn<TA, TB, TC, 1>(g, st);
    if (g.L <= 32) return launch_tn<TA, TB, TC, 2>(g, st);
    if (g.L <= 64) return launch_tn<TA, TB, TC, 4>(g, st);
    return launch_tn<TA, TB, TC, 8>(g, st);
}

}  // namespace

int gemm_simt_splits(int64_t R, int64_t K, int num_sms) {
    const int64_t tiles = (R + kBM - 1) / kBM;
    int64_t want = (2LL * num_sms + tiles - 1) / tiles;
    const int64_t maxs = K / kBK > 1 ? K / kBK : 1;  // at least one k-stage per split
    if (want > maxs) want = maxs;
    if (want < 1) want = 1;
    if (want > 1024) want = 1024;
    return (int)want;
}

cudaError_t launch_gemm_simt(const GemmArgs& g, cudaStream_t st) {
    if (g.R <= 0 || g.L <= 0 || g.L > kMaxEllSimt || g.splits < 1) return cudaErrorInvalidValue;
    const ElemType tb = g.tb == T_SAME ? g.tc : g.tb;
    if (g.L > 128) {
        // column groups of at most 128 output columns: the B operand and the
        // output (each split's partial alike) start j0 columns further on
        for (int64_t j0 = 0; j0 < g.L; j0 += 128) {
            GemmArgs h = g;
            h.L = std::min<int64_t>(128, g.L - j0);
            h.b = static_cast<const char*>(g.b) + (g.bmode == B_PANEL ? j0 * g.ldb : j0) * elem_size(tb);
            h.out = static_cast<char*>(g.out) + (g.omode == O_PANEL ? j0 * g.ldo : j0) * elem_size(g.tc);
            const cudaError_t e = launch_gemm_simt(h, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (g.ta == T_F64 && tb == T_F64 && g.tc == T_F64) return launch_types<double, double, double>(g, st);
    if (g.ta == T_F32 && tb == T_F32 && g.tc == T_F32) return launch_types<float, float, float>(g, st);
    if (g.ta == T_F32 && tb == T_F64 && g.tc == T_F64) return launch_types<float, double, double>(g, st);
    if (g.ta == T_F64 && tb == T_F32 && g.tc == T_F32) return launch_types<double, float, float>(g, st);
    if (g.ta == T_F64 && tb == T_F64 && g.tc == T_F32) return launch_types<double, double, float>(g, st);
    return cudaErrorInvalidValue;
}

int device_sms() {
    static std::atomic<int> cached[64];  // zero until first asked
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of split partials: out = sum_s part[s], s ascending.
// Element (x, y) of the region is at y * ld + x.
// ---------------------------------------------------------------------------
namespace {
// Block = 32 output elements x 8 split groups. Thread (x, g) adds the
// partials g, g + 8, g + 16, ... of element x with four accumulators; the
// eight group sums are then added in group order. The summation order depends
// only on the split count, so results are reproducible.
constexpr int kRedGroups = 8;
template <typename TP, typename TO>
__global__ void __launch_bounds__(32 * kRedGroups)
reduce_splits_kernel(const TP* part, int splits, int64_t stride, TO* out, int64_t ld, int64_t rows,
                     int64_t cols, int64_t ld_out, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ double red[kRedGroups][33];
    const int tx = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t total = rows * cols;
    const int64_t e = (int64_t)blockIdx.x * 32 + tx;
    double s = 0.0;
    if (e < total) {
        const int64_t y = e / rows, x = e % rows;
        const TP* p = part + y * ld + x;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int q = g;
        for (; q + 3 * kRedGroups < splits; q += 4 * kRedGroups) {
            a0 += (double)p[(int64_t)q * stride];
            a1 += (double)p[(int64_t)(q + kRedGroups) * stride];
            a2 += (double)p[(int64_t)(q + 2 * kRedGroups) * stride];
            a3 += (double)p[(int64_t)(q + 3 * kRedGroups) * stride];
        }
        for (; q < splits; q += kRedGroups) a0 += (double)p[(int64_t)q * stride];
        s = (a0 + a1) + (a2 + a3);
    }
    red[g][tx] = s;
    __syncthreads();
    if (g == 0 && e < total) {
        double t = red[0][tx];
        for (int k = 1; k < kRedGroups; ++k) t += red[k][tx];
        const int64_t y = e / rows, x = e % rows;
        out[y * ld_out + x] = (TO)t;
    }
}

template <typename TP, typename TO>
cudaError_t reduce_launch(const void* part, int splits, int64_t stride, void* out, int64_t ld, int64_t rows,
                          int64_t cols, int64_t ld_out, const int* cancel, cudaStream_t st) {
    const unsigned blocks = (unsigned)((rows * cols + 31) / 32);
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(reduce_splits_kernel<TP, TO>, dim3(blocks), dim3(32 * kRedGroups), (size_t)(0), st, static_cast<const TP*>(part), splits, stride,
                                                                     static_cast<TO*>(out), ld, rows, cols, ld_out,
                                                                     cancel);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_reduce_splits(const void* part, ElemType tpart, int splits, int64_t stride, void* out,
                                 ElemType tout, int64_t ld, int64_t rows, int64_t cols, int64_t ld_out,
                                 const int* cancel, cudaStream_t st) {
    if (rows * cols <= 0) return cudaSuccess;
    if (tpart == T_F64 && tout == T_F64) return reduce_launch<double, double>(part, splits, stride, out, ld, rows, cols, ld_out, cancel, st);
    if (tpart == T_F32 && tout == T_F64) return reduce_launch<float, double>(part, splits, stride, out, ld, rows, cols, ld_out, cancel, st);
    if (tpart == T_F32 && tout == T_F32) return reduce_launch<float, float>(part, splits, stride, out, ld, rows, cols, ld_out, cancel, st);
    if (tpart == T_F64 && tout == T_F32) return reduce_launch<double, float>(part, splits, stride, out, ld, rows, cols, ld_out, cancel, st);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Step 1 of Algorithm 1: Gaussian test matrix from Philox-4x32-10
// (Salmon et al., SC'11) and the Box-Muller transform (cosine branch).
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ void philox_4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double gauss_at(uint64_t seed, uint32_t sid, uint32_t i, uint32_t j) {
    uint32_t c[4] = {i, j, sid, 0u};
    philox_4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t a = ((((uint64_t)c[0]) << 32) | c[1]) >> 11;
    const uint64_t b = ((((uint64_t)c[2]) << 32) | c[3]) >> 11;
    const double scale = 1.0 / 9007199254740992.0;  // 2^-53
    const double u1 = ((double)a + 1.0) * scale;
    const double u2 = (double)b * scale;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// The same draw with the Box-Muller transform in FP32 (the 53-bit uniforms
// rounded to float): within ~1e-6 relative of gauss_at, for FP32 panels, where
// the FP64 log / cos would run on the FP64 pipe (about 64 cycles per warp
// instruction on this GPU) for no accuracy the FP32 panel keeps.
__device__ __forceinline__ float gauss_at_f32(uint64_t seed, uint32_t sid, uint32_t i, uint32_t j) {
    uint32_t c[4] = {i, j, sid, 0u};
    philox_4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t a = ((((uint64_t)c[0]) << 32) | c[1]) >> 11;
    const uint64_t b = ((((uint64_t)c[2]) << 32) | c[3]) >> 11;
    const float u1 = __ull2float_rn(a + 1) * 0x1p-53f;
    const float u2 = __ull2float_rn(b) * 0x1p-53f;
    return sqrtf(-2.0f * logf(u1)) * cosf(6.2831853071795865f * u2);
}

template <typename TX>
__device__ __forceinline__ TX gauss_elem(uint64_t seed, uint32_t sid, uint32_t i, uint32_t j);
template <>
__device__ __forceinline__ double gauss_elem<double>(uint64_t seed, uint32_t sid, uint32_t i, uint32_t j) {
    return gauss_at(seed, sid, i, j);
}
template <>
__device__ __forceinline__ float gauss_elem<float>(uint64_t seed, uint32_t sid, uint32_t i, uint32_t j) {
    return gauss_at_f32(seed, sid, i, j);
}

template <typename TX>
__global__ void gaussian_panel_kernel(uint64_t seed, uint32_t sid, int64_t n, int64_t ell,
                                      int64_t ellp, TX* x, int64_t ldx, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const int64_t total = n * ellp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / n, i = e % n;
        x[j * ldx + i] = (j < ell) ? gauss_elem<TX>(seed, sid, (uint32_t)i, (uint32_t)j) : (TX)0;
    }
}

__global__ void gaussian_rowmajor_kernel(uint64_t seed, uint32_t sid, int64_t n, int64_t ell,
                                         double* psi, int64_t ld) {
    pdl_trigger();
    pdl_wait();
    const int64_t total = n * ell;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ell, j = e % ell;
        psi[i * ld + j] = gauss_at(seed, sid, (uint32_t)i, (uint32_t)j);
    }
}

int grid_for(int64_t total) {
    int64_t b = (total + 255) / 256;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    return (int)b;
}
}  // namespace

cudaError_t launch_gaussian_panel(uint64_t seed, uint32_t stream_id, int64_t n, int64_t ell,
                                  int64_t ellp, void* x, ElemType tx, int64_t ldx, const int* cancel,
                                  cudaStream_t st) {
    count_launch();
    if (tx == T_F64)
        {
            cudaError_t pe_ = launch_pdl(gaussian_panel_kernel<double>, dim3(grid_for(n * ellp)), dim3(256), (size_t)(0), st, seed, stream_id, n, ell, ellp,
                                                                          static_cast<double*>(x), ldx, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    else
        {
            cudaError_t pe_ = launch_pdl(gaussian_panel_kernel<float>, dim3(grid_for(n * ellp)), dim3(256), (size_t)(0), st, seed, stream_id, n, ell, ellp,
                                                                         static_cast<float*>(x), ldx, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    return cudaGetLastError();
}

cudaError_t launch_gaussian_rowmajor(uint64_t seed, uint32_t stream_id, int64_t n, int64_t ell,
                                     double* psi, int64_t ld, cudaStream_t st) {
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(gaussian_rowmajor_kernel, dim3(grid_for(n * ell)), dim3(256), (size_t)(0), st, seed, stream_id, n, ell, psi, ld);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout conversions through 32 x 32 shared-memory tiles (both sides
// coalesced).
// ---------------------------------------------------------------------------
namespace {
// dst(row-major rows x cols) <- src(panel) or the reverse; `to_panel`
// selects the direction. Padding columns [cols, colsp) of a panel output
// are written as zero.
template <typename TD>
__global__ void transpose_kernel(const double* src, int64_t lds, int64_t rows, int64_t cols,
                                 int64_t colsp, TD* dst, int64_t ldd, bool to_panel,
                                 const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int s = ty; s < 32; s += 8) {
        double v = 0.0;
        if (to_panel) {  // src row-major: (i0+s, j0+tx)
            const int64_t i = i0 + s, j = j0 + tx;
            if (i < rows && j < cols) v = src[i * lds + j];
        } else {         // src panel: (i0+tx, j0+s)
            const int64_t i = i0 + tx, j = j0 + s;
            if (i < rows && j < cols) v = src[j * lds + i];
        }
        tile[s][tx] = v;
    }
    __syncthreads();
    for (int s = ty; s < 32; s += 8) {
        if (to_panel) {  // dst panel: (i0+tx, j0+s) = tile[tx][s]
            const int64_t i = i0 + tx, j = j0 + s;
            if (i < rows && j < colsp) dst[j * ldd + i] = cvt<TD>(tile[tx][s]);
        } else {         // dst row-major: (i0+s, j0+tx) = tile[tx][s]
            const int64_t i = i0 + s, j = j0 + tx;
            if (i < rows && j < cols) dst[i * ldd + j] = cvt<TD>(tile[tx][s]);
        }
    }
}

template <typename TS, typename TD>
__global__ void panel_convert_kernel(const TS* src, int64_t lds, int64_t rows, int64_t cols,
                                     TD* dst, int64_t ldd, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, i = e % rows;
        dst[j * ldd + i] = cvt<TD>(src[j * lds + i]);
    }
}
}  // namespace

cudaError_t launch_rowmajor_to_panel(const double* src, int64_t lds, int64_t rows, int64_t cols,
                                     int64_t colsp, void* dst, ElemType tdst, int64_t ldd, cudaStream_t st) {
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((colsp + 31) / 32));
    count_launch();
    if (tdst == T_F64)
        {
            cudaError_t pe_ = launch_pdl(transpose_kernel<double>, dim3(grid), dim3(dim3(32, 8)), (size_t)(0), st, src, lds, rows, cols, colsp, static_cast<double*>(dst),
                                                               ldd, true, nullptr);
            if (pe_ != cudaSuccess) return pe_;
        }
    else
        {
            cudaError_t pe_ = launch_pdl(transpose_kernel<float>, dim3(grid), dim3(dim3(32, 8)), (size_t)(0), st, src, lds, rows, cols, colsp, static_cast<float*>(dst),
                                                              ldd, true, nullptr);
            if (pe_ != cudaSuccess) return pe_;
        }
    return cudaGetLastError();
}

cudaError_t launch_panel_to_rowmajor(const double* src, int64_t lds, int64_t rows, int64_t cols,
                                     void* dst, ElemType tdst, int64_t ldd, const int* cancel,
                                     cudaStream_t st) {
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    if (tdst == T_F64) {
        count_launch();
        {
            cudaError_t pe_ = launch_pdl(transpose_kernel<double>, dim3(grid), dim3(dim3(32, 8)), (size_t)(0), st, src, lds, rows, cols, cols,
                                                               static_cast<double*>(dst), ldd, false,
                                                               cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    } else {
        count_launch();
        {
            cudaError_t pe_ = launch_pdl(transpose_kernel<float>, dim3(grid), dim3(dim3(32, 8)), (size_t)(0), st, src, lds, rows, cols, cols,
                                                              static_cast<float*>(dst), ldd, false,
                                                              cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    }
    return cudaGetLastError();
}

template <typename TS>
cudaError_t panel_convert_from(const TS* src, int64_t lds, int64_t rows, int64_t cols, void* dst, ElemType tdst,
                               int64_t ldd, const int* cancel, cudaStream_t st) {
    const int blocks = grid_for(rows * cols);
    count_launch();
    switch (tdst) {
        case T_F64:
            {
                cudaError_t pe_ = launch_pdl(panel_convert_kernel<TS, double>, dim3(blocks), dim3(256), (size_t)(0), st, src, lds, rows, cols, static_cast<double*>(dst),
                                                                     ldd, cancel);
                if (pe_ != cudaSuccess) return pe_;
            }
            break;
        case T_F32:
            {
                cudaError_t pe_ = launch_pdl(panel_convert_kernel<TS, float>, dim3(blocks), dim3(256), (size_t)(0), st, src, lds, rows, cols, static_cast<float*>(dst),
                                                                    ldd, cancel);
                if (pe_ != cudaSuccess) return pe_;
            }
            break;
        case T_BF16:
            {
                cudaError_t pe_ = launch_pdl(panel_convert_kernel<TS, __nv_bfloat16>, dim3(blocks), dim3(256), (size_t)(0), st, 
                src, lds, rows, cols, static_cast<__nv_bfloat16*>(dst), ldd, cancel);
                if (pe_ != cudaSuccess) return pe_;
            }
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_panel_convert(const void* src, ElemType tsrc, int64_t lds, int64_t rows, int64_t cols,
                                 void* dst, ElemType tdst, int64_t ldd, const int* cancel, cudaStream_t st) {
    if (tsrc == T_F64)
        return panel_convert_from(static_cast<const double*>(src), lds, rows, cols, dst, tdst, ldd, cancel, st);
    if (tsrc == T_F32)
        return panel_convert_from(static_cast<const float*>(src), lds, rows, cols, dst, tdst, ldd, cancel, st);
    return cudaErrorInvalidValue;
}


// ---------------------------------------------------------------------------
// Grouped forms (one launch over the problems of a batch).
// ---------------------------------------------------------------------------
namespace {
// zero fill of a byte range (16-byte aligned start, length a multiple of 4)
__device__ __forceinline__ void zero_body(const ZeroArgs& a) {
    pdl_trigger();
    pdl_wait();
    const int64_t n4 = a.bytes >> 4;
    uint4* p = static_cast<uint4*>(a.p);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = make_uint4(0u, 0u, 0u, 0u);
    uint32_t* q = reinterpret_cast<uint32_t*>(static_cast<char*>(a.p) + (n4 << 4));
    const int64_t r4 = (a.bytes - (n4 << 4)) >> 2;
    if (blockIdx.x == 0)
        for (int64_t e = threadIdx.x; e < r4; e += blockDim.x) q[e] = 0u;
}

// The Gaussian panel of launch_gaussian_panel's FP32 draw, stored as bf16
// (the rounding panel_convert applies to that FP32 panel)
__device__ __forceinline__ void gaussian_bf16_body(const GaussArgs& a) {
    pdl_trigger();
    pdl_wait();
    if (a.cancel && *a.cancel) return;
    const int64_t total = a.n * a.ellp;
    __nv_bfloat16* x = static_cast<__nv_bfloat16*>(a.x);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / a.n, i = e % a.n;
        const float v = (j < a.ell) ? gauss_elem<float>(a.seed, a.sid, (uint32_t)i, (uint32_t)j) : 0.f;
        x[j * a.ldx + i] = cvt<__nv_bfloat16>(v);
    }
}
}  // namespace

GroupItem<ZeroArgs> zero_item(void* p, int64_t bytes) {
    GroupItem<ZeroArgs> it;
    it.a = ZeroArgs{p, bytes};
    it.gx = kAnyGrid;
    it.gy = 1;
    return it;
}

GroupItem<GaussArgs> gaussian_item(const GaussArgs& a) {
    GroupItem<GaussArgs> it;
    it.a = a;
    it.gx = kAnyGrid;
    it.gy = 1;
    return it;
}

cudaError_t launch_zero_grouped(const GroupItem<ZeroArgs>* it, int count, unsigned gx, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    count_launch();
    cudaError_t e = launch_pdl(grouped_kernel<ZeroArgs, zero_body, 256>, dim3(gx, 1, (unsigned)count), dim3(256),
                               (size_t)0, st, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_gaussian_grouped(const GroupItem<GaussArgs>* it, int count, unsigned gx, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    count_launch();
    cudaError_t e = launch_pdl(grouped_kernel<GaussArgs, gaussian_bf16_body, 256>, dim3(gx, 1, (unsigned)count),
                               dim3(256), (size_t)0, st, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace corutv
