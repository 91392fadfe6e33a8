// ALM-CoRUTV iteration kernels (Algorithm 2, Sec. 4).
//
// One iteration j, given the CoR-UTV factors of B_j = M - S_j + Y_j / mu_j:
//   r       = #{i : T_ii > 1/mu_j}                      (operator C_delta)
//   Z       = V T(1:r,:)^T            (cols x ell, columns >= r zero)
//   L_{j+1} = U Z^T  = U(:,1:r) T(1:r,:) V^T            (never stored per iteration)
//   S_{j+1} = shrink(M - L_{j+1} + Y_j / mu_j, lambda / mu_j)
//   Y_{j+1} = Y_j + mu_j (M - L_{j+1} - S_{j+1})
//   B_{j+1} = M - S_{j+1} + Y_{j+1} / mu_{j+1}          (input of the next CoR-UTV)
//   zeta_j  = ||M - L_{j+1} - S_{j+1}||_F / ||M||_F
// The update is one fused pass over the m x n state (reads M, Y; writes S, Y, B)
// that forms L_{j+1} on the fly from the rank-r factors.
#include <algorithm>

#include "internal.cuh"

namespace corutv {

namespace {

constexpr int kUpdCols = 128;   // threads per block = columns per tile
constexpr int kUpdRows = 16;    // rows per tile
constexpr int kMaxEll = kMaxEllSimt;  // ell = 2k; kernels are instantiated for ell <= 64, <= 128 and <= 320
constexpr int kFinalThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;  // valid in thread 0
}

template <typename TM>
__device__ __forceinline__ double ld_m(const void* m, int64_t off) {
    return (double)static_cast<const TM*>(m)[off];
}

// S = 0, Y = 0, B = M; per-block sum of M^2.
template <typename TM, typename TS>
__global__ void rpca_init_kernel(const TM* m, int64_t ldm, int64_t rows, int64_t cols, TS* s, TS* y,
                                 TS* b, double* fro_part) {
    pdl_trigger();
    pdl_wait();
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, c = e % cols;
        const double mv = (double)m[i * ldm + c];
        s[e] = (TS)0;
        y[e] = (TS)0;
        b[e] = (TS)mv;
        acc += mv * mv;
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) fro_part[blockIdx.x] = t;
}

// r = #{i : Rt_ii > inv_mu}; Z[i][s] = sum_h Q2[i][perm[h]] Rt[s][h] for s < r.
// Rt is staged in shared memory up to ell = 128 and read from global memory
// (the same entries for every thread of a warp) beyond.
template <typename TQ, int kE>
__global__ void rank_z_kernel(const double* rt, const TQ* q2, int64_t ldq2, const int* perm,
                              int64_t cols, int ell, double inv_mu, int* rank, double* z, int64_t ldz,
                              const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ double Rsm[];  // ell x ell (kE <= 128)
    const double* Rs = kE <= 128 ? Rsm : rt;
    __shared__ int ps[kE];
    __shared__ int r_s;
    if (kE <= 128)
        for (int e = threadIdx.x; e < ell * ell; e += blockDim.x) Rsm[e] = rt[e];
    for (int e = threadIdx.x; e < ell; e += blockDim.x) ps[e] = perm[e];
    if (threadIdx.x == 0) {
        int r = 0;
        for (int i = 0; i < ell; ++i)
            if (rt[i * ell + i] > inv_mu) ++r;
        r_s = r;
        if (blockIdx.x == 0) *rank = r;
    }
    __syncthreads();
    const int r = r_s;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cols) return;
    double v[kE];
#pragma unroll 4
    for (int h = 0; h < ell; ++h) v[h] = (double)q2[(int64_t)ps[h] * ldq2 + i];
    for (int s = 0; s < ell; ++s) {
        double acc = 0.0;
        if (s < r)
            for (int h = s; h < ell; ++h) acc += v[h] * Rs[s * ell + h];  // Rt upper triangular
        z[(int64_t)s * ldz + i] = acc;
    }
}

// Fused S / Y / B update over a tile of kUpdRows x kUpdCols elements, in the
// arithmetic of the state (TS): FP32 for FP32 data (on this GPU the FP64
// pipe runs at a sixtieth of the FP32 rate), FP64 for FP64 data. The squared
// residual is summed per thread in TS and across the block in FP64.
template <typename TM, typename TS, int kE>
__global__ void __launch_bounds__(kUpdCols)
rpca_update_kernel(const TM* m, int64_t ldm, int64_t rows, int64_t cols, TS* s, TS* y, TS* b,
                   const double* u, int64_t ldu, const double* z, int64_t ldz, int ell, const int* rank,
                   double mu, double mu_next, double lambda, double* res_part, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ double red[32];
    __shared__ TS Us[kUpdRows][kE];
    const int r = *rank;
    const int64_t i0 = (int64_t)blockIdx.y * kUpdRows;
    const int64_t c = (int64_t)blockIdx.x * kUpdCols + threadIdx.x;
    for (int e = threadIdx.x; e < kUpdRows * kE; e += blockDim.x) {
        const int ii = e / kE, sidx = e % kE;
        const int64_t i = i0 + ii;
        Us[ii][sidx] = (i < rows && sidx < r) ? (TS)u[(int64_t)sidx * ldu + i] : (TS)0;
    }
    TS zc[kE];
    if (c < cols) {
#pragma unroll 4
        for (int sidx = 0; sidx < ell; ++sidx) zc[sidx] = (sidx < r) ? (TS)z[(int64_t)sidx * ldz + c] : (TS)0;
    }
    __syncthreads();
    const TS inv_mu = (TS)(1.0 / mu), inv_mu_next = (TS)(1.0 / mu_next), delta = (TS)(lambda / mu), muc = (TS)mu;
    TS acc = 0;
    if (c < cols) {
        for (int ii = 0; ii < kUpdRows; ++ii) {
            const int64_t i = i0 + ii;
            if (i >= rows) break;
            TS l = 0;
            for (int sidx = 0; sidx < r; ++sidx) l = fma(Us[ii][sidx], zc[sidx], l);
            const int64_t e = i * cols + c;
            const TS mv = (TS)m[i * ldm + c];
            const TS yv = y[e];
            const TS x = mv - l + yv * inv_mu;
            const TS mag = fabs(x) - delta;
            const TS sv = mag > (TS)0 ? copysign(mag, x) : (TS)0;
            const TS res = mv - l - sv;
            const TS yn = yv + muc * res;
            s[e] = sv;
            y[e] = yn;
            b[e] = mv - sv + yn * inv_mu_next;
            acc = fma(res, res, acc);
        }
    }
    const double t = block_sum(f2d_exact(acc), red);
    if (threadIdx.x == 0) res_part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Power-iteration products for the default mu0 (||M||_2). y = M x: one warp
// per row, lanes along the row (coalesced), FP64 accumulation.
template <typename TM>
__global__ void gemv_rows_kernel(const TM* mat, int64_t ldm, int64_t m, int64_t n, const double* x, double* y) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < m; i += nw) {
        const TM* row = mat + i * ldm;
        double a = 0.0;
        for (int64_t c = lane; c < n; c += 32) a = fma(f2d_exact(row[c]), x[c], a);
#pragma unroll
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) y[i] = a;
    }
}

// Column partials of M^T u over row chunks: thread = column (coalesced), block
// row = chunk; FP64 accumulation in row order.
template <typename TM>
__global__ void gemv_cols_kernel(const TM* mat, int64_t ldm, int64_t m, int64_t n, const double* u, double* part,
                                 int64_t ldp, int64_t chunk_rows) {
    pdl_trigger();
    pdl_wait();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
    const int64_t r1 = r0 + chunk_rows < m ? r0 + chunk_rows : m;
    if (c >= n) return;
    double a = 0.0;
    for (int64_t i = r0; i < r1; ++i) a = fma(f2d_exact(mat[i * ldm + c]), u[i], a);
    part[(int64_t)blockIdx.y * ldp + c] = a;
}

// zeta_j and the convergence flag; one block, fixed summation order.
__global__ void finish_iter_kernel(const double* res_part, int nparts, const double* fro_part, int nfro,
                                   double tol, int iter, double* zeta_hist, int* flags, const int* rank) {
    pdl_trigger();
    pdl_wait();
    if (flags[FLAG_RPCA_DONE]) return;
    __shared__ double red[32];
    double a = 0.0, f = 0.0;
    for (int e = threadIdx.x; e < nparts; e += blockDim.x) a += res_part[e];
    for (int e = threadIdx.x; e < nfro; e += blockDim.x) f += fro_part[e];
    const double ra = block_sum(a, red);
    const double rf = block_sum(f, red);
    if (threadIdx.x == 0) {
        const double zeta = sqrt(ra) / sqrt(rf);
        zeta_hist[iter] = zeta;
        flags[FLAG_RPCA_ITERS] = iter + 1;
        flags[FLAG_RPCA_RANK] = *rank;
        if (zeta < tol) flags[FLAG_RPCA_DONE] = 1;
    }
}

template <typename TL, int kE>
__global__ void __launch_bounds__(kUpdCols)
reconstruct_kernel(const double* u, int64_t ldu, const double* z, int64_t ldz, const int* rank, int ell,
                   int64_t rows, int64_t cols, TL* lout, int64_t ldl) {
    pdl_trigger();
    pdl_wait();
    __shared__ TL Us[kUpdRows][kE];
    const int r = *rank;
    const int64_t i0 = (int64_t)blockIdx.y * kUpdRows;
    const int64_t c = (int64_t)blockIdx.x * kUpdCols + threadIdx.x;
    for (int e = threadIdx.x; e < kUpdRows * kE; e += blockDim.x) {
        const int ii = e / kE, sidx = e % kE;
        const int64_t i = i0 + ii;
        Us[ii][sidx] = (i < rows && sidx < r) ? (TL)u[(int64_t)sidx * ldu + i] : (TL)0;
    }
    TL zc[kE];
    if (c < cols)
        for (int sidx = 0; sidx < ell; ++sidx) zc[sidx] = (sidx < r) ? (TL)z[(int64_t)sidx * ldz + c] : (TL)0;
    __syncthreads();
    if (c >= cols) return;
    for (int ii = 0; ii < kUpdRows; ++ii) {
        const int64_t i = i0 + ii;
        if (i >= rows) break;
        TL l = 0;
        for (int sidx = 0; sidx < r; ++sidx) l = fma(Us[ii][sidx], zc[sidx], l);
        lout[i * ldl + c] = l;
    }
}

int init_blocks(int64_t total) {
    int64_t b = (total + 255) / 256;
    if (b > 1184) b = 1184;
    if (b < 1) b = 1;
    return (int)b;
}

__global__ void vec_fill_kernel(double* v, int64_t n, double value) {
    pdl_trigger();
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = value;
}

__global__ void vec_normalize_kernel(const double* w, double* v, int64_t n, double* lam) {
    pdl_trigger();
    pdl_wait();
    __shared__ double red[32];
    __shared__ double nrm;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += w[i] * w[i];
    const double t = block_sum(a, red);
    if (threadIdx.x == 0) {
        nrm = sqrt(t);
        *lam = nrm;
    }
    __syncthreads();
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = w[i] * inv;
}

}  // namespace

cudaError_t launch_vec_fill(double* v, int64_t n, double value, cudaStream_t st) {
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(vec_fill_kernel, dim3((unsigned)std::min<int64_t>((n + 255) / 256, 1024)), dim3(256), (size_t)(0), st, v, n, value);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

cudaError_t launch_vec_normalize(const double* w, double* v, int64_t n, double* lam, cudaStream_t st) {
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(vec_normalize_kernel, dim3(1), dim3(1024), (size_t)(0), st, w, v, n, lam);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

cudaError_t launch_gemv_rows(const void* mat, ElemType tm, int64_t ldm, int64_t m, int64_t n, const double* x,
                             double* y, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<int64_t>((m + 7) / 8, 1216);  // 8 rows (warps) per block
    count_launch();
    cudaError_t e = tm == T_F32
        ? launch_pdl(gemv_rows_kernel<float>, dim3(blocks), dim3(256), (size_t)0, st, static_cast<const float*>(mat),
                     ldm, m, n, x, y)
        : launch_pdl(gemv_rows_kernel<double>, dim3(blocks), dim3(256), (size_t)0, st,
                     static_cast<const double*>(mat), ldm, m, n, x, y);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_gemv_cols_partial(const void* mat, ElemType tm, int64_t ldm, int64_t m, int64_t n,
                                     const double* u, double* part, int64_t ldp, int chunks, cudaStream_t st) {
    if (chunks < 1 || ldp < n) return cudaErrorInvalidValue;
    const int64_t chunk_rows = (m + chunks - 1) / chunks;
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)chunks);
    count_launch();
    cudaError_t e = tm == T_F32
        ? launch_pdl(gemv_cols_kernel<float>, grid, dim3(256), (size_t)0, st, static_cast<const float*>(mat), ldm, m,
                     n, u, part, ldp, chunk_rows)
        : launch_pdl(gemv_cols_kernel<double>, grid, dim3(256), (size_t)0, st, static_cast<const double*>(mat), ldm,
                     m, n, u, part, ldp, chunk_rows);
    return e != cudaSuccess ? e : cudaGetLastError();
}

int rpca_update_blocks(int64_t rows, int64_t cols) {
    return (int)(((cols + kUpdCols - 1) / kUpdCols) * ((rows + kUpdRows - 1) / kUpdRows));
}

cudaError_t launch_rpca_init(const void* m, ElemType tm, int64_t ldm, int64_t rows, int64_t cols,
                             float* s, float* y, float* b, double* s64, double* y64, double* b64,
                             double* fro_part, int* nparts, cudaStream_t st) {
    const int blocks = init_blocks(rows * cols);
    *nparts = blocks;
    if (tm == T_F32) {
        count_launch();
        {
            cudaError_t pe_ = launch_pdl(rpca_init_kernel<float, float>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const float*>(m), ldm, rows, cols,
                                                               s, y, b, fro_part);
            if (pe_ != cudaSuccess) return pe_;
        }
    } else {
        count_launch();
        {
            cudaError_t pe_ = launch_pdl(rpca_init_kernel<double, double>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const double*>(m), ldm, rows,
                                                                 cols, s64, y64, b64, fro_part);
            if (pe_ != cudaSuccess) return pe_;
        }
    }
    return cudaGetLastError();
}

template <typename TQ, int kE>
cudaError_t rank_z_launch(const double* rt, const void* vq2, int64_t ldv, const int* perm, int64_t cols, int64_t ell,
                          double inv_mu, int* rank, double* z, int64_t ldz, const int* cancel, cudaStream_t st) {
    const size_t smem = kE <= 128 ? sizeof(double) * (size_t)ell * ell : 0;
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(rank_z_kernel<TQ, kE>));
    if (e != cudaSuccess) return e;
    count_launch();
    e = launch_pdl(rank_z_kernel<TQ, kE>, dim3((unsigned)((cols + 127) / 128)), dim3(128), smem, st, rt,
                   static_cast<const TQ*>(vq2), ldv, perm, cols, (int)ell, inv_mu, rank, z, ldz, cancel);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_rpca_rank_z(const double* rt, const void* vq2, ElemType tq2, int64_t ldv, const int* perm,
                               int64_t cols, int64_t ell, double inv_mu, int* rank, double* z,
                               int64_t ldz, const int* cancel, cudaStream_t st) {
    if (ell > kMaxEll) return cudaErrorInvalidValue;
    if (tq2 == T_F64)
        return ell <= 64    ? rank_z_launch<double, 64>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st)
               : ell <= 128 ? rank_z_launch<double, 128>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st)
                            : rank_z_launch<double, kMaxEll>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st);
    return ell <= 64    ? rank_z_launch<float, 64>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st)
           : ell <= 128 ? rank_z_launch<float, 128>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st)
                        : rank_z_launch<float, kMaxEll>(rt, vq2, ldv, perm, cols, ell, inv_mu, rank, z, ldz, cancel, st);
}

template <typename TM, typename TS, int kE>
cudaError_t update_launch(const RpcaIterArgs& a, const TM* m, TS* s, TS* y, TS* b, dim3 grid, cudaStream_t st) {
    count_launch();
    cudaError_t e = launch_pdl(rpca_update_kernel<TM, TS, kE>, grid, dim3(kUpdCols), (size_t)0, st, m, a.ldm, a.rows,
                               a.cols, s, y, b, a.u, a.ldu, a.z, a.ldz, (int)a.ell, a.rank, a.mu, a.mu_next,
                               a.lambda, a.res_part, a.cancel);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_rpca_update(const RpcaIterArgs& a, int* nparts, cudaStream_t st) {
    if (a.ell > kMaxEll) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((a.cols + kUpdCols - 1) / kUpdCols), (unsigned)((a.rows + kUpdRows - 1) / kUpdRows));
    *nparts = (int)(grid.x * grid.y);
    if (a.tm == T_F32) {
        const float* m = static_cast<const float*>(a.m);
        return a.ell <= 64    ? update_launch<float, float, 64>(a, m, a.s, a.y, a.b, grid, st)
               : a.ell <= 128 ? update_launch<float, float, 128>(a, m, a.s, a.y, a.b, grid, st)
                              : update_launch<float, float, kMaxEll>(a, m, a.s, a.y, a.b, grid, st);
    }
    const double* m = static_cast<const double*>(a.m);
    return a.ell <= 64    ? update_launch<double, double, 64>(a, m, a.s64, a.y64, a.b64, grid, st)
           : a.ell <= 128 ? update_launch<double, double, 128>(a, m, a.s64, a.y64, a.b64, grid, st)
                          : update_launch<double, double, kMaxEll>(a, m, a.s64, a.y64, a.b64, grid, st);
}

cudaError_t launch_rpca_finish_iter(const double* res_part, int nparts, const double* fro_part,
                                    int nfro, double tol, int iter, double* zeta_hist,
                                    int* flags, const int* rank, cudaStream_t st) {
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(finish_iter_kernel, dim3(1), dim3(kFinalThreads), (size_t)(0), st, res_part, nparts, fro_part, nfro, tol, iter, zeta_hist,
                                                    flags, rank);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

template <typename TL, int kE>
cudaError_t reconstruct_launch(const double* u, int64_t ldu, const double* z, int64_t ldz, const int* rank,
                               int64_t ell, int64_t rows, int64_t cols, void* lout, int64_t ldl, cudaStream_t st) {
    dim3 grid((unsigned)((cols + kUpdCols - 1) / kUpdCols), (unsigned)((rows + kUpdRows - 1) / kUpdRows));
    count_launch();
    cudaError_t e = launch_pdl(reconstruct_kernel<TL, kE>, grid, dim3(kUpdCols), (size_t)0, st, u, ldu, z, ldz, rank,
                               (int)ell, rows, cols, static_cast<TL*>(lout), ldl);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_rpca_reconstruct(const double* u, int64_t ldu, const double* z, int64_t ldz,
                                    const int* rank, int64_t ell, int64_t rows, int64_t cols,
                                    void* lout, ElemType tl, int64_t ldl, cudaStream_t st) {
    if (ell > kMaxEll) return cudaErrorInvalidValue;
    if (tl == T_F32)
        return ell <= 64    ? reconstruct_launch<float, 64>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st)
               : ell <= 128 ? reconstruct_launch<float, 128>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st)
                            : reconstruct_launch<float, kMaxEll>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st);
    return ell <= 64    ? reconstruct_launch<double, 64>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st)
           : ell <= 128 ? reconstruct_launch<double, 128>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st)
                        : reconstruct_launch<double, kMaxEll>(u, ldu, z, ldz, rank, ell, rows, cols, lout, ldl, st);
}

}  // namespace corutv
