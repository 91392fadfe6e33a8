// Small dense factorisations of libcorutv:
//  * Cholesky of an ell x ell Gram matrix (CholeskyQR, the thin QR of
//    Sec. 3.1 "C1 = Q1 R1, C2 = Q2 R2"), FP64, with the shift of shifted
//    CholeskyQR (Fukaya et al., SIAM J. Sci. Comput. 2020) when the Gram is
//    not numerically positive definite;
//  * Q = C R^{-1} by forward substitution, one thread per row;
//  * the column-pivoted QR of D (eq. 8), one block, FP64, Householder
//    reflections with Businger-Golub pivoting on recomputed column norms;
//  * the gathers of eq. 9 (V = Q2 P, T = Rt).
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include <type_traits>

#include "internal.cuh"

namespace corutv {

namespace {

// ---------------------------------------------------------------------------
// FP64 reciprocal and reciprocal square root without the FP64 divide / sqrt
// sequences (each several hundred cycles on this part, where every FP64
// warp instruction holds its sub-partition's FP64 pipe for about 64 cycles):
// the hardware's FP64 estimate (PTX rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64,
// relative error below 2^-19.9 measured over 2^26 inputs spread across the
// exponent range, about 40 cycles) followed by ONE third-order Householder
// step, i.e. the Taylor series of the exact correction factor to second order:
//   1/sqrt(x): e = 1 - x y^2,  y (1 - e)^-1/2 = y (1 + e/2 + 3e^2/8 + O(e^3))
//   1/x      : e = 1 - x y,    y (1 - e)^-1   = y (1 + e + e^2 + O(e^3))
// The truncation error is O(e^3) (about 2^-60), so the result is within a
// few ulp (1 ulp of the library operation over the same 2^26 inputs); the
// dependent chain is 4 (resp. 3) FP64 operations after the estimate. For
// operands of magnitude in [2^-999, 2^1001) (1/sqrt: positive), tested on the
// bit pattern with integer operations; others fall back to the library
// operations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rsqrt_nr(double x) {
    const int hi = __double2hiint(x);
    const int ef = (hi >> 20) & 0x7ff;
    // integer tests (an FP64 compare costs ~2 FMAs of latency): positive and
    // 2^-999 <= x < 2^1001, so that y^2 and the estimate stay normal
    if (hi < 0 || (unsigned)(ef - 24) >= 2000u) return 1.0 / sqrt(x);
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y * y, 1.0);
    const double c = fma(0.375, e, 0.5);       // 1/2 + 3e/8
    return fma(y * e, c, y);
}

__device__ __forceinline__ double rcp_nr(double x) {
    const int ef = (__double2hiint(x) >> 20) & 0x7ff;
    if ((unsigned)(ef - 24) >= 2000u) return 1.0 / x;  // 2^-999 <= |x| < 2^1001: 1/x stays normal
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// Right-looking Cholesky, upper factor, R^T R = G (+ shift I), in the
// square-root-free form: S holds the Schur complement rows, p_t = S_tt is the
// t-th pivot and the step-t update is S_ac -= (S_ta / p_t) S_tc (a, c > t);
// R_tc = S_tc / sqrt(p_t) once all the rows are final, for all rows at once.
// The pivots form the only sequential chain: p_{t+1} = S'_{t+1,t+1} -
// (S_{t,t+1} / p_t) S_{t,t+1}, one reciprocal (estimate + 3 FP64 operations)
// and two FP64 operations per column. On this GPU every FP64 warp instruction
// holds its sub-partition's FP64 pipe for about 64 cycles whatever the number
// of active lanes (a predicated-off one too), so the chain runs alone on one
// sub-partition and every FP64 instruction sits in a loop whose trip count is
// the same on all lanes of its warp:
//  * warp 0 (the chain): at step t it takes row t (final), forms r_t = 1/p_t
//    and the scaled row L_t = r_t S_t, hands both to the update warps, then
//    applies step t to row t+1 itself (lanes = columns) once the update warps
//    have applied steps < t to that row -- which gives p_{t+1};
//  * warps 1-3 and 5-7 (on the other three sub-partitions) apply step s to
//    rows >= s+2: row s+2 first, then a signal to warp 0, then the rest of
//    the trailing triangle (bottom-up enumeration `tri`), 32 entries per warp
//    instruction;
//  * warp 4 (sub-partition 0, shared with the chain) stays out of the loop.
// The two hand-offs are producer/consumer named barriers (update warps
// arrive, warp 0 waits: ids 1, 2 by the parity of the step; warp 0 arrives,
// update warps wait: ids 3, 4), so no step waits for the whole trailing update
// of the step before it. Each side runs at most one step ahead of the other
// on a hand-off, so two ids per direction keep consecutive steps' arrivals
// apart; the update warps' waits on the second hand-off also keep them in
// step with each other.
// rows = number of rows of the matrix whose Gram is factorised (for the shift).
constexpr int kCholThreads = 256;
constexpr int kCholUpdThreads = 192;
constexpr int kCholMaxEll = 128;

// d > 0 and finite, by integer tests on the bit pattern
__device__ __forceinline__ bool pos_finite(double d) {
    const long long b = __double_as_longlong(d);
    return b > 0 && ((b >> 52) & 0x7ff) != 0x7ff;
}

// d > m for m >= 0 finite, with the IEEE result (false for NaN), by integer tests
__device__ __forceinline__ bool gt_nonneg(double d, double m) {
    const long long b = __double_as_longlong(d);
    return b > __double_as_longlong(m) && (b & 0x7fffffffffffffffLL) <= 0x7ff0000000000000LL;
}

__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <bool kDefic>
__device__ __forceinline__ void cholesky_body(const double* g, int ell, int64_t rows, double* r, int* flags,
                                              int* skip_out, const int* cancel, double unit_roundoff, int* defic,
                                              double tau_rel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ double S[];  // ell x (ell + 1) doubles, then the uint16 table
    const int ld = ell + 1;
    unsigned short* tri = reinterpret_cast<unsigned short*>(S + (size_t)ell * ld);
    __shared__ double Lr[3][kCholMaxEll];  // L_t in slot t % 3 (read by step t of the update warps)
    __shared__ double ys[kCholMaxEll];
    __shared__ int rowdep[kCholMaxEll];
    __shared__ double trace, dmin_s;
    __shared__ int fail_at;  // step whose pivot failed (kNoFail: none)
    constexpr int kNoFail = 1 << 30;
    constexpr int kSync = 32 + kCholUpdThreads;  // warp 0 + update warps
    // table (independent of the predecessor's output, built before waiting on
    // it): bottom-up rows; row a holds columns ell-1 .. a
    for (int a = ell - 1 - tid; a >= 0; a -= kCholThreads) {
        const int rb = ell - 1 - a;            // rows below the top of the enumeration
        int e = rb * (rb + 1) / 2;
        for (int c = ell - 1; c >= a; --c) tri[e++] = (unsigned short)((a << 8) | c);
    }
    pdl_wait();
    if (cancel && *cancel) {
        if (skip_out && tid == 0) *skip_out = 1;
        return;
    }
    if (kDefic) {
        // dependence threshold: tau_rel times the largest diagonal entry
        if (warp == 0) {
            double mx = 0.0;
            for (int a = lane; a < ell; a += 32) mx = fmax(mx, g[a * ell + a]);
#pragma unroll
            for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) dmin_s = tau_rel * mx;
        }
    }
    const int wu = warp - (warp > 4 ? 2 : 1);  // update warp 0 .. 5 (warps 1-3, 5-7)
    int attempt = 0;
    bool fail = false;
    for (; attempt < 3; ++attempt) {
        double shift = 0.0;
        if (attempt > 0) {
            // shift s = 11 (rows ell + ell (ell + 1)) u ||C||_F^2, u the unit roundoff of the
            // arithmetic that formed G (Fukaya et al.), then x100;
            // ||C||_F^2 = trace(G), summed only when a shift is needed
            if (warp == 0) {
                double t = 0.0;
                for (int a = lane; a < ell; a += 32) t += g[a * ell + a];
#pragma unroll
                for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) trace = t;
            }
            __syncthreads();
            const double u = unit_roundoff;
            shift = 11.0 * ((double)rows * ell + (double)ell * (ell + 1)) * u * trace * (attempt == 1 ? 1.0 : 100.0);
        }
        // eight loads in flight per thread before their stores; the row index
        // from an FP32 product ((e + 1/2) / ell is at least 1/(2 ell) away from an
        // integer, far above the product's rounding for e < 2^14), and no FP64
        // operation on the way (the shift is added to the diagonal afterwards)
        const float inv_ell = 1.0f / (float)ell;
        for (int e0 = 0; e0 < ell * ell; e0 += 8 * kCholThreads) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + tid + k * kCholThreads;
                v[k] = e < ell * ell ? g[e] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + tid + k * kCholThreads;
                if (e < ell * ell) {
                    const int a = __float2int_rz(((float)e + 0.5f) * inv_ell), b = e - a * ell;
                    S[a * ld + b] = v[k];
                }
            }
        }
        if (attempt > 0) {
            __syncthreads();
            for (int a = tid; a < ell; a += kCholThreads) S[a * ld + a] += shift;
        }
        for (int a = tid; a < ell; a += kCholThreads) {
            rowdep[a] = 0;
            if (kDefic) defic[a] = 0;
        }
        if (tid == 0) fail_at = kNoFail;
        __syncthreads();
        // FP64 operations of the update warps sit in loops whose trip counts are
        // the same on all lanes of a warp (a branch, not a predicate): a
        // predicated-off FP64 instruction would still hold the pipe.
        if (warp == 0) {
            double p = S[0];
            const double dmin = kDefic ? dmin_s : 0.0;
            for (int t = 0;; ++t) {
                // kDefic: a pivot <= dmin marks column t numerically dependent (r_t = 0: row t updates nothing)
                const bool dep = kDefic && !gt_nonneg(p, dmin);
                const bool ok = dep || pos_finite(p);
                double rt = rcp_nr(p);
                if (kDefic) rt = dep ? 0.0 : rt;
                // L_t = r_t S_t (row t is final in S): strip 0 inline, the rest in a loop
                double* Lt = Lr[t % 3];
                const double* St = S + t * ld;
                double l0;
                {
                    const int c = t + lane;
                    l0 = St[c < ell ? c : ell - 1] * rt;
                    if (c < ell) Lt[c] = l0;
                }
#pragma unroll 1
                for (int c0 = t + 32; c0 < ell; c0 += 32) {
                    const int c = c0 + lane;
                    const double x = St[c < ell ? c : ell - 1] * rt;
                    if (c < ell) Lt[c] = x;
                }
                if (!ok) {
                    if (lane == 0) fail_at = t;
                } else if (kDefic && dep) {
                    if (lane == 0) {
                        rowdep[t] = 1;
                        defic[t] = 1;
                    }
                }
                if (t <= ell - 3) bar_arrive(3 + (t & 1), kSync);  // L_t, fail_at -> update step t
                if (!ok) {
                    // update step t-1 still signals (it saw fail_at = t > t-1): take it so the barrier stays balanced
                    if (t >= 1 && t - 1 <= ell - 3) bar_sync(1 + ((t - 1) & 1), kSync);
                    break;
                }
                if (t == ell - 1) break;
                const double w = __shfl_sync(0xffffffffu, l0, 1);  // L_{t,t+1}
                if (t >= 1) bar_sync(1 + ((t - 1) & 1), kSync);    // update step t-1 has finished row t+1
                // step t on row t+1 (columns t+1 ..): S_{t+1,c} -= L_{t,t+1} S_{t,c}
                double* Sn = S + (t + 1) * ld;
                double p_next;
                {
                    const int c = t + 1 + lane;
                    const int cc = c < ell ? c : ell - 1;
                    p_next = fma(-w, St[cc], Sn[cc]);
                    if (c < ell) Sn[c] = p_next;
                }
                p = __shfl_sync(0xffffffffu, p_next, 0);
#pragma unroll 1
                for (int c0 = t + 33; c0 < ell; c0 += 32) {
                    const int c = c0 + lane;
                    const int cc = c < ell ? c : ell - 1;
                    const double x = fma(-w, St[cc], Sn[cc]);
                    if (c < ell) Sn[c] = x;
                }
                __syncwarp();
            }
        } else if (warp != 4) {
            for (int s = 0; s <= ell - 3; ++s) {
                bar_sync(3 + (s & 1), kSync);  // row s and L_s are final
                if (fail_at <= s) break;       // a later step's failure does not stop this one
                const double* rs = S + s * ld;
                const double* Ls = Lr[s % 3];
                // row s+2 first (columns s+2 .. ell-1), then the signal
                const int n1 = ell - s - 2;
                {
                    const double l = Ls[s + 2];
                    double* Sa = S + (s + 2) * ld;
                    for (int i0 = 32 * wu; i0 < n1; i0 += kCholUpdThreads) {
                        const int c = s + 2 + i0 + lane;
                        const int cc = c < ell ? c : ell - 1;
                        const double x = fma(-l, rs[cc], Sa[cc]);
                        if (c < ell) Sa[c] = x;
                    }
                }
                bar_arrive(1 + (s & 1), kSync);
                // rows >= s+3: the prefix tri[0 .. len3) of the bottom-up enumeration
                const int len3 = (n1 - 1) * n1 / 2;
#pragma unroll 4
                for (int e0 = 32 * wu; e0 < len3; e0 += kCholUpdThreads) {
                    const int e = e0 + lane;
                    const int ac = tri[e < len3 ? e : len3 - 1];
                    const int a = ac >> 8, c = ac & 0xff;
                    const double x = fma(-Ls[a], rs[c], S[a * ld + c]);
                    if (e < len3) S[a * ld + c] = x;
                }
            }
        }
        __syncthreads();
        fail = fail_at != kNoFail;
        if (!fail) break;
    }
    pdl_trigger();  // the successor may launch while R is written
    const bool broke = attempt == 3;
    // R_tc = S_tc / sqrt(p_t) for c >= t (the diagonal p_t / sqrt(p_t)); dependent rows -> e_t
    for (int t = tid; t < ell; t += kCholThreads) ys[t] = (broke || rowdep[t]) ? 0.0 : rsqrt_nr(S[t * ld + t]);
    __syncthreads();
    // the upper triangle through the packed enumeration `tri` (every lane of an
    // FP64 multiply busy), the lower one as zeros; dependent rows (and all rows
    // after a breakdown) are e_a
    const int ntri = ell * (ell + 1) / 2;
    for (int e = tid; e < ntri; e += kCholThreads) {
        const int ac = tri[e];
        const int a = ac >> 8, c = ac & 0xff;
        const bool unit = broke || rowdep[a];
        const double x = S[a * ld + c] * ys[a];
        r[(size_t)a * ell + c] = unit ? (a == c ? 1.0 : 0.0) : x;
    }
    const float inv_ell = 1.0f / (float)ell;
    for (int e = tid; e < ell * ell; e += kCholThreads) {
        const int a = __float2int_rz(((float)e + 0.5f) * inv_ell), c = e - a * ell;
        if (c < a) r[e] = 0.0;
    }
    if (tid == 0) {
        if (broke) atomicExch(&flags[FLAG_BREAKDOWN], 1);
        if (attempt > 0) atomicAdd(&flags[FLAG_SHIFTED], 1);
        if (skip_out) *skip_out = (attempt > 0 && !broke) ? 0 : 1;
    }
}

template <bool kDefic>
__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* g, int ell, int64_t rows, double* r, int* flags, int* skip_out,
                const int* cancel, double unit_roundoff, int* defic, double tau_rel) {
    cholesky_body<kDefic>(g, ell, rows, r, flags, skip_out, cancel, unit_roundoff, defic, tau_rel);
}

// Product of the upper triangular factors of successive CholeskyQR passes:
// out = Rn Ra (the thin QR C = Q R of the passes together has R = R_last ...
// R_first), or out = Rn when Ra is null, or out = Ra when *skip is set (a pass
// that did not run); with `transpose` out receives the transpose. One block
// per row a, thread c forms sum_{a <= t <= c} Rn[a][t] Ra[t][c] in FP64.
__global__ void trimul_kernel(const double* rn, const double* ra, double* out, int ell, int transpose,
                              const int* skip, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const int a = blockIdx.x, c = threadIdx.x;
    if (c >= ell) return;
    double v;
    if (skip && *skip) {
        v = ra[a * ell + c];
    } else if (!ra) {
        v = c >= a ? rn[a * ell + c] : 0.0;
    } else {
        v = 0.0;
        for (int t = a; t <= c; ++t) v = fma(rn[a * ell + t], ra[t * ell + c], v);
    }
    if (transpose) out[c * ell + a] = v;
    else out[a * ell + c] = v;
}

// Entry (i, j) of a random completion column: N(0, 1) / sqrt(rows) from
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) of the counter (i, j), two
// 53-bit uniforms and the cosine branch of Box-Muller. Only columns the
// Cholesky found numerically dependent use it; any orthonormal completion is
// a valid thin QR there, and the next CholeskyQR pass orthonormalises it.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float completion_entry(int64_t i, int j, int64_t rows) {
    // (i, j) with j < 256 keeps its original key; wider columns add their high bits at the top
    const unsigned long long key =
        (((unsigned long long)i << 8) | (unsigned long long)(j & 0xff)) + ((unsigned long long)(j >> 8) << 56);
    const unsigned long long h1 = splitmix64(2 * key), h2 = splitmix64(2 * key + 1);
    const float u1 = (float)((double)((h1 >> 11) + 1) * 0x1p-53);  // (0, 1]
    const float u2 = (float)((double)(h2 >> 11) * 0x1p-53);        // [0, 1)
    return sqrtf(-2.f * logf(u1)) * cosf(6.2831853f * u2) * rsqrtf((float)rows);
}

// Row i of Q solves q_i R = c_i (R upper): q_i[j] = (c_i[j] - sum_{t<j} q_i[t] R[t][j]) / R[j][j].
// Four adjacent lanes share a row. Columns are solved in blocks of kTrsmB:
// lane s adds the contributions of the solved columns t = s mod 4 into
// kTrsmB independent accumulators, two xor shuffles combine the four partial
// sums, and all four lanes finish the small triangle of the block in order
// (redundantly), each storing its quarter of the new values. A block of 128
// threads covers 32 rows, so a panel spreads over four times as many threads
// as with one thread per row, each with about a third of the instructions.
constexpr int kTrsmB = 8;
constexpr int kTrsmL = 4;                        // lanes per row
constexpr int kTrsmRows = 32;                    // rows per block
constexpr int kTrsmThreads = kTrsmL * kTrsmRows;
// Row-major per row in shared memory with a stride = 4 (mod 32) elements:
// the 32 lanes of a warp (8 rows x 4 consecutive columns) hit 32 distinct
// banks (a stride of 32 rows put a row's four lanes on one bank).
__host__ __device__ __forceinline__ int trsm_ld(int ell) { return ((ell + 31) & ~31) + 4; }
// Row stride of the staged R: every row starts 16-byte aligned, is padded
// with zeros to whole eight-column blocks, and the rows t .. t + 3 that the
// four lane groups of a warp read together land on distinct bank quadruples
// (stride = 4 (mod 8) floats, 2 (mod 8) doubles), so the eight R values of a
// step come in two 16-byte loads without bank conflicts.
template <typename TC>
__host__ __device__ __forceinline__ int trsm_ldr(int ell) {
    return ((ell + 7) & ~7) + (sizeof(TC) == 4 ? 4 : 2);
}
template <typename TC>
__host__ __device__ __forceinline__ size_t trsm_smem_elems(int ell, int rows) {
    return (size_t)ell * trsm_ldr<TC>(ell) + (size_t)rows * trsm_ld(ell) + (size_t)ell;
}
// Eight consecutive values from a 16-byte aligned shared-memory address.
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void ld8(const double* p, double (&v)[8]) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const double2 a = *reinterpret_cast<const double2*>(p + 2 * h);
        v[2 * h] = a.x;
        v[2 * h + 1] = a.y;
    }
}
template <typename TI, typename TC, typename TQC, int kRows>
__global__ void __launch_bounds__(kTrsmL * kRows)
trsm_rows_kernel(const TI* c, int64_t ldc, int64_t rows, int ell, const double* r, TI* q, int64_t ldq,
                 TQC* qc, int64_t ldqc, const int* cancel, const int* defic) {
    constexpr int kTrsmRows = kRows, kTrsmThreads = kTrsmL * kRows;
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldr = trsm_ldr<TC>(ell);
    TC* Rs = reinterpret_cast<TC*>(smem_raw);   // ell x ldr row-major, zero beyond column ell
    TC* Ts = Rs + ell * ldr;                    // [kTrsmRows][ld]: a row's c values, then its q values
    const int ld = trsm_ld(ell);
    TC* Rd = Ts + (size_t)kTrsmRows * trsm_ld(ell);  // 1 / R[j][j]
    const int tid = threadIdx.x;
    const int ln = tid & (kTrsmL - 1), rr = tid / kTrsmL;
    // loads in batches of 16 per thread, all in flight before their stores
    constexpr int kB = 16;
    for (int e0 = 0; e0 < ell * ldr; e0 += kB * kTrsmThreads) {
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kTrsmThreads + tid;
            const int row = e / ldr, col = e - row * ldr;
            v[u] = (e < ell * ldr && col < ell) ? r[row * ell + col] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kTrsmThreads + tid;
            if (e < ell * ldr) Rs[e] = (TC)v[u];
        }
    }
    for (int j = tid; j < ell; j += kTrsmThreads) Rd[j] = (TC)1 / (TC)r[j * ell + j];
    const int64_t i = (int64_t)blockIdx.x * kTrsmRows + rr;
    const bool live = i < rows;
    for (int j0 = ln; j0 < ell; j0 += kTrsmL * kB) {  // lane ln loads columns ln, ln + 4, ...
        TI v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = j0 + kTrsmL * u;
            v[u] = (live && j < ell) ? c[(int64_t)j * ldc + i] : (TI)0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = j0 + kTrsmL * u;
            if (j < ell) Ts[rr * ld + j] = (TC)v[u];
        }
    }
    __syncthreads();
    for (int j0 = 0; j0 < ell; j0 += kTrsmB) {
        const int nb = min(kTrsmB, ell - j0);
        TC acc[kTrsmB];
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k) acc[k] = (ln == 0 && k < nb) ? Ts[rr * ld + j0 + k] : (TC)0;
        // columns k >= nb of the last block meet R's zero padding; they are never stored
        for (int t = ln; t < j0; t += kTrsmL) {
            const TC qt = Ts[rr * ld + t];
            TC rv[kTrsmB];
            ld8(Rs + t * ldr + j0, rv);
#pragma unroll
            for (int k = 0; k < kTrsmB; ++k) acc[k] -= qt * rv[k];
        }
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k) {
            acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 1);
            acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 2);
        }
        // the block's triangle, column after column: q_kk is final once the
        // terms of the columns before it are subtracted (each q_k receives
        // them in increasing kk, as in row-wise substitution)
#pragma unroll
        for (int kk = 0; kk < kTrsmB; ++kk) {
            if (kk >= nb) break;
            acc[kk] *= Rd[j0 + kk];
            TC rv[kTrsmB];
            ld8(Rs + (j0 + kk) * ldr + j0, rv);
#pragma unroll
            for (int k = kk + 1; k < kTrsmB; ++k) acc[k] -= acc[kk] * rv[k];
        }
        __syncwarp();  // the row's lanes have read their c values before any is overwritten
#pragma unroll
        for (int k = 0; k < kTrsmB; ++k)
            if (k < nb && (k & (kTrsmL - 1)) == ln) Ts[rr * ld + j0 + k] = acc[k];
        __syncwarp();
    }
    pdl_trigger();  // the successor may launch while Q is written
    if (!live) return;
    for (int j = ln; j < ell; j += kTrsmL) {
        TC v = Ts[rr * ld + j];
        if (defic && defic[j]) v = (TC)completion_entry(i, j, rows);  // R row j is e_j: nothing else used q_j
        q[(int64_t)j * ldq + i] = (TI)v;
        if (qc) qc[(int64_t)j * ldqc + i] = (TQC)v;
    }
}

template <typename TI, typename TC, typename TQC, int kRows>
cudaError_t trsm_launch_rows(const void* c, int64_t ldc, int64_t rows, int ell, const double* r, void* q,
                             int64_t ldq, void* qc, int64_t ldqc, const int* cancel, cudaStream_t st,
                             const int* defic) {
    const size_t smem = sizeof(TC) * trsm_smem_elems<TC>(ell, kRows);
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(trsm_rows_kernel<TI, TC, TQC, kRows>));
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((rows + kRows - 1) / kRows);
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(trsm_rows_kernel<TI, TC, TQC, kRows>, dim3(blocks), dim3(kTrsmL * kRows), (size_t)(smem), st,
                                     static_cast<const TI*>(c), ldc, rows, ell, r, static_cast<TI*>(q), ldq,
                                     static_cast<TQC*>(qc), ldqc, cancel, defic);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

// Rows per block: every block stages R and runs the same substitution chain,
// so the kernel takes about one block's time per wave of blocks. 32 rows per
// block while all blocks fit in one wave; for longer panels 96 rows (three
// times the threads on the same staged R) when that takes fewer waves.
template <typename TC>
int trsm_rows_per_block(int64_t rows, int ell) {
    auto waves = [&](int per) {
        const size_t smem = sizeof(TC) * trsm_smem_elems<TC>(ell, per);
        if (smem > 227 * 1024) return (int64_t)1 << 40;  // does not fit one SM's shared memory
        int res = (int)std::min<size_t>(227 * 1024 / smem, 2048 / (size_t)(kTrsmL * per));
        if (res < 1) res = 1;
        const int64_t blocks = (rows + per - 1) / per;
        return (blocks + (int64_t)res * device_sms() - 1) / ((int64_t)res * device_sms());
    };
    return waves(96) < waves(32) ? 96 : 32;
}

template <typename TI, typename TC, typename TQC>
cudaError_t trsm_launch(const void* c, int64_t ldc, int64_t rows, int ell, const double* r, void* q, int64_t ldq,
                        void* qc, int64_t ldqc, const int* cancel, cudaStream_t st, const int* defic) {
    if (trsm_rows_per_block<TC>(rows, ell) == 96)
        return trsm_launch_rows<TI, TC, TQC, 96>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st, defic);
    return trsm_launch_rows<TI, TC, TQC, 32>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st, defic);
}

template <typename TI, typename TC>
cudaError_t trsm_dispatch(const void* c, int64_t ldc, int64_t rows, int ell, const double* r, void* q,
                          int64_t ldq, void* qc, ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st,
                          const int* defic) {
    if (!qc) return trsm_launch<TI, TC, TI>(c, ldc, rows, ell, r, q, ldq, nullptr, 0, cancel, st, defic);
    switch (tqc) {
        case T_F64: return trsm_launch<TI, TC, double>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st, defic);
        case T_F32: return trsm_launch<TI, TC, float>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st, defic);
        case T_BF16: return trsm_launch<TI, TC, __nv_bfloat16>(c, ldc, rows, ell, r, q, ldq, qc, ldqc, cancel, st, defic);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Q = C R^{-1} for FP32 panels as two short launches instead of a
// substitution chain per row: the FP32 inverse of R once, then a product in
// which every entry q_ij = sum_{k <= j} c_ik (R^{-1})_kj is an independent dot
// product. Each row's chain in the substitution kernel above is ell^2 / 2
// dependent steps long whatever the panel's length; here a warp's chain is at
// most ell multiply-adds.
//
// rinv_kernel: column j of R^{-1} solves R x = e_j by column-oriented back
// substitution, one warp per column: b = e_j; for k = j, j-1, ..., 0:
// x_k = b_k / R_kk, then b_i -= R_ik x_k for i < k. Lane l keeps b_i for
// i = l + 32 s; the steps run slot by slot (k = 32 S + kk) so that x_k's slot
// is known at compile time. R is read in FP32 (the precision the panel is
// solved in), stored transposed so that column k is contiguous.
// ri: ell x ldri row-major, zero below the diagonal and beyond column ell.
constexpr int kRiWarps = 8;
__host__ __device__ __forceinline__ int rinv_ldt(int ell) { return ((ell + 31) & ~31) + 1; }

template <int S>
__device__ __forceinline__ void rinv_slot(float (&b)[4], const float* Rt, int ldt, const float* rd, int lane,
                                          int top) {
    for (int kk = top; kk >= 0; --kk) {
        const int k = 32 * S + kk;
        const float* col = Rt + k * ldt;  // col[i] = R_ik
        float rk[S + 1];
#pragma unroll
        for (int s = 0; s <= S; ++s) rk[s] = col[lane + 32 * s];
        const float xk = __shfl_sync(0xffffffffu, b[S], kk) * rd[k];
#pragma unroll
        for (int s = 0; s < S; ++s) b[s] = fmaf(-rk[s], xk, b[s]);
        b[S] = lane < kk ? fmaf(-rk[S], xk, b[S]) : (lane == kk ? xk : b[S]);
    }
}

__device__ __forceinline__ void rinv_body(const double* r, int ell, float* ri, int ldri, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldt = rinv_ldt(ell);                     // odd: the transposing stores hit 32 banks
    float* Rt = reinterpret_cast<float*>(smem_raw);    // ell x ldt: Rt[k][i] = R_ik, i <= k
    float* rd = Rt + (size_t)ell * ldt;                // 1 / R_kk
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the upper triangle, 16 loads per thread in flight before their stores
    constexpr int kB = 16, kT = kRiWarps * 32;
    for (int e0 = 0; e0 < ell * ell; e0 += kB * kT) {
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kT + tid, i = e / ell, k = e - i * ell;
            v[u] = (e < ell * ell && k >= i) ? r[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kT + tid, i = e / ell, k = e - i * ell;
            if (e < ell * ell && k >= i) Rt[k * ldt + i] = (float)v[u];
        }
    }
    __syncthreads();
    for (int k = tid; k < ell; k += kRiWarps * 32) rd[k] = 1.f / Rt[k * ldt + k];
    __syncthreads();
    pdl_trigger();
    const int j = blockIdx.x * kRiWarps + warp;
    if (j >= ell) return;
    float b[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) b[s] = (lane + 32 * s == j) ? 1.f : 0.f;
    switch (j >> 5) {  // the slots from x_j's down to slot 0
        case 3: rinv_slot<3>(b, Rt, ldt, rd, lane, j & 31); [[fallthrough]];
        case 2: rinv_slot<2>(b, Rt, ldt, rd, lane, (j >> 5) == 2 ? j & 31 : 31); [[fallthrough]];
        case 1: rinv_slot<1>(b, Rt, ldt, rd, lane, (j >> 5) == 1 ? j & 31 : 31); [[fallthrough]];
        default: rinv_slot<0>(b, Rt, ldt, rd, lane, (j >> 5) == 0 ? j & 31 : 31);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        if (i < ell) ri[(int64_t)i * ldri + j] = i <= j ? b[s] : 0.f;
    }
    if (j == ell - 1)  // the padding columns
        for (int i = lane; i < ell; i += 32)
            for (int jj = ell; jj < ldri; ++jj) ri[(int64_t)i * ldri + jj] = 0.f;
}

__global__ void __launch_bounds__(kRiWarps * 32)
rinv_kernel(const double* r, int ell, float* ri, int ldri, const int* cancel) {
    rinv_body(r, ell, ri, ldri, cancel);
}

// trsm_gemm_kernel: 128 rows per block, staged column by column into shared
// memory (k-major: Cs[k][row]) together with R^{-1} (both with all of a
// thread's loads in flight before its stores); warp w computes columns
// 8w .. 8w + 7 for all 128 rows (4 adjacent rows per lane, 32 accumulators)
// over k <= 8w + 7 (R^{-1} is upper triangular), reading the R^{-1} row
// segment as two 16-byte loads that every lane shares. Writes Q (and its copy qc), replacing the columns
// the extra CholeskyQR pass marked dependent by their random completion.
// In place (q == c) is safe: a block reads all its rows before writing any.
constexpr int kTgRows = 128;
template <typename TQC>
__device__ __forceinline__ void trsm_gemm_body(const float* c, int64_t ldc, int64_t rows, int ell, const float* ri,
                                               int ldri, float* q, int64_t ldq, TQC* qc, int64_t ldqc,
                                               const int* cancel, const int* defic) {
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Cs = reinterpret_cast<float*>(smem_raw);  // [ell][kTgRows]
    float* Rs = Cs + (size_t)ell * kTgRows;         // R^{-1}: [ell][ldri]
    const int64_t r0 = (int64_t)blockIdx.x * kTgRows;
    const int nr = (int)(rows - r0 < kTgRows ? rows - r0 : kTgRows);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nt = blockDim.x;
    constexpr int kB = 8;
    const int nc4 = ell * (kTgRows / 4), nr4 = ell * ldri / 4;
    for (int e0 = 0; e0 < nc4 + nr4; e0 += kB * nt) {
        float4 v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * nt + tid;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < nc4) {
                const int k = e / (kTgRows / 4), i = 4 * (e % (kTgRows / 4));
                const float* src = c + (int64_t)k * ldc + r0 + i;
                if (i + 3 < nr) {
                    v[u] = __ldcs(reinterpret_cast<const float4*>(src));
                } else {
                    if (i < nr) v[u].x = src[0];
                    if (i + 1 < nr) v[u].y = src[1];
                    if (i + 2 < nr) v[u].z = src[2];
                }
            } else if (e < nc4 + nr4) {
                v[u] = __ldcg(reinterpret_cast<const float4*>(ri) + (e - nc4));
            }
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * nt + tid;
            if (e < nc4) {
                const int k = e / (kTgRows / 4), i = 4 * (e % (kTgRows / 4));
                *reinterpret_cast<float4*>(Cs + k * kTgRows + i) = v[u];
            } else if (e < nc4 + nr4) {
                reinterpret_cast<float4*>(Rs)[e - nc4] = v[u];
            }
        }
    }
    __syncthreads();
    const int j0 = 8 * w;
    if (j0 >= ell) return;  // warps beyond this problem's columns (a grouped launch sized for a wider one)
    const int kend = min(ell, j0 + 8);
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
    for (int k = 0; k < kend; ++k) {
        const float4 cv = *reinterpret_cast<const float4*>(Cs + k * kTgRows + 4 * lane);
        const float4 u0 = *reinterpret_cast<const float4*>(Rs + k * ldri + j0);
        const float4 u1 = *reinterpret_cast<const float4*>(Rs + k * ldri + j0 + 4);
        const float cr[4] = {cv.x, cv.y, cv.z, cv.w};
        const float rv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(cr[a], rv[b], acc[a][b]);
    }
    pdl_trigger();  // the successor may launch while Q is written
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int j = j0 + b;
        if (j >= ell) break;
        const bool dep = defic && defic[j];
        float v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = r0 + 4 * lane + a;
            v[a] = dep ? completion_entry(i, j, rows) : acc[a][b];
        }
        const int i0 = 4 * lane;
        if (i0 + 3 < nr) {
            *reinterpret_cast<float4*>(q + (int64_t)j * ldq + r0 + i0) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (i0 + a < nr) q[(int64_t)j * ldq + r0 + i0 + a] = v[a];
        }
        if (qc) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (i0 + a < nr) qc[(int64_t)j * ldqc + r0 + i0 + a] = (TQC)v[a];
        }
    }
}

template <typename TQC>
__global__ void __launch_bounds__(512)
trsm_gemm_kernel(const float* c, int64_t ldc, int64_t rows, int ell, const float* ri, int ldri, float* q,
                 int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel, const int* defic) {
    trsm_gemm_body<TQC>(c, ldc, rows, ell, ri, ldri, q, ldq, qc, ldqc, cancel, defic);
}

int trsm_inv_ldri(int ell) { return (ell + 7) & ~7; }

}  // namespace

int64_t trsm_rinv_floats(int64_t ell) { return ell * ((ell + 7) & ~7); }

namespace {

template <typename TQC>
cudaError_t trsm_inv_launch(const float* c, int64_t ldc, int64_t rows, int ell, const double* r, float* ri,
                            float* q, int64_t ldq, TQC* qc, int64_t ldqc, const int* cancel, cudaStream_t st,
                            const int* defic) {
    const int ldri = trsm_inv_ldri(ell);
    const size_t smem_ri = sizeof(float) * ((size_t)ell * rinv_ldt(ell) + ell);
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(rinv_kernel));
    if (e != cudaSuccess) return e;
    count_launch();
    e = launch_pdl(rinv_kernel, dim3((unsigned)((ell + kRiWarps - 1) / kRiWarps)), dim3(kRiWarps * 32), smem_ri, st,
                   r, ell, ri, ldri, cancel);
    if (e != cudaSuccess) return e;
    const size_t smem_g = sizeof(float) * (size_t)ell * (kTgRows + ldri);
    e = allow_max_dynamic_smem(reinterpret_cast<const void*>(trsm_gemm_kernel<TQC>));
    if (e != cudaSuccess) return e;
    count_launch();
    e = launch_pdl(trsm_gemm_kernel<TQC>, dim3((unsigned)((rows + kTgRows - 1) / kTgRows)),
                   dim3(32 * ((ell + 7) / 8)), smem_g, st, c, ldc, rows, ell, static_cast<const float*>(ri), ldri,
                   q, ldq, qc, ldqc, cancel, defic);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// QRCP of the small D (eq. 8): one block, FP64, Householder reflections with
// Businger-Golub pivoting on column norms recomputed exactly at every step.
//
// Every step is bound by the FP64 pipe (one warp instruction per sub-partition
// about every 65 cycles on this GPU) and by its dependent chain, so:
//  * the active columns are spread over 8 warps with a power-of-two group of
//    lanes per column (rows split inside the group, sums by xor shuffles), so
//    the lanes stay full as the active block shrinks;
//  * the next step's squared norms are recomputed exactly in the same pass
//    that applies the reflector (no separate norm pass). They are not
//    downdated: the pivot's norm also builds the next reflector, whose
//    orthogonality would inherit a downdated norm's error (up to ~1e-8);
//  * the dot products over the rows below the diagonal, t_c = x_j[j+1:]^T
//    x_c[j+1:], start before the reflector is known: with v = [1; x_{j+1:} /
//    (alpha - beta)], v^T x_c = x_c[j] + t_c / (alpha - beta). They run on
//    warps 1-3 and 5-7 (after the other warps swap the pivot column in),
//    while warp 0 swaps row j itself and computes beta, tau and 1 / (alpha -
//    beta) as soon as the pivot is known: its sub-partition's FP64 pipe then
//    serves that dependent chain alone; warps 4 and 8 stage column j;
//  * the pivot (argmax of the squared norms, compared through their bit
//    patterns, lowest index on ties) is taken by every warp redundantly, so it
//    needs no broadcast.
// W is column-major in shared memory (column c at W + c * ldw, ldw odd).
// ---------------------------------------------------------------------------
constexpr int kQrcpMapThreads = 256;                  // warps 0-7: column groups
constexpr int kQrcpThreads = kQrcpMapThreads + 32;    // warp 8: staging
constexpr int kQrcpDotThreads = 192;                  // warps 1-3, 5-7 during the reflector dots

// lanes per column for `ncols` active columns of `nrows` rows over `nthr`
// threads: a power of two <= 32, and at most a quarter of the rows (fewer
// shuffle levels once the block is small)
__device__ __forceinline__ int qr_group(int ncols, int nrows, int nthr = kQrcpMapThreads) {
    int g = 1;
    while (g < 32 && 2 * g * ncols <= nthr && 4 * g <= nrows) g <<= 1;
    return g;
}

__device__ __forceinline__ double group_sum(double v, int g) {
    for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// argmax of nrm[j..ell) (non-negative doubles, so their bit patterns order
// like their values) with one 64-bit max: the key is the bit pattern with its
// 7 lowest mantissa bits replaced by 127 - c, so equal norms go to the lowest
// index; norms within 2^-45 relative of each other count as equal.
__device__ __forceinline__ int qr_pivot(const double* nrm, int j, int ell, int lane) {
    long long best = -1;
    for (int c = j + lane; c < ell; c += 32) {
        const long long key = (__double_as_longlong(nrm[c]) & ~0x7fLL) | (127 - c);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        best = ob > best ? ob : best;
    }
    return 127 - (int)(best & 0x7f);
}

__device__ __forceinline__ void qrcp_body(const double* d, int ell, double* refl, double* rt, int* perm,
                                          const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ double W[];  // ell columns of ldw doubles, then nrm, xbuf, tau, sgn, tdot, perm
    const int ldw = ell | 1;
    double* nrm = W + ell * ldw;
    double* xbuf = nrm + ell;
    double* tau = xbuf + ell;
    double* sgn = tau + ell;
    double* tdot = sgn + ell;
    int* pv = reinterpret_cast<int*>(tdot + ell);
    __shared__ double sc_beta, sc_tau, sc_scale, sc_ts;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool mapped = tid < kQrcpMapThreads;
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int a = e / ell, b = e % ell;  // d row-major: entry (a, b) -> column b, row a
        W[b * ldw + a] = d[e];
    }
    for (int c = tid; c < ell; c += kQrcpThreads) pv[c] = c;
    __syncthreads();
    {   // squared norms of all columns
        const int g = qr_group(ell, ell);
        const int c = tid / g, ph = tid % g;
        double s = 0.0;
        if (mapped && c < ell)
            for (int i = ph; i < ell; i += g) s = fma(W[c * ldw + i], W[c * ldw + i], s);
        if (mapped) {
            s = group_sum(s, g);
            if (c < ell && ph == 0) nrm[c] = s;
        }
    }
    __syncthreads();
    for (int j = 0; j < ell; ++j) {
        // S1: pivot (every warp)
        const int p = qr_pivot(nrm, j, ell, lane);
        const int nc = ell - j - 1;
        if (warp == 0) {
            // row j of columns j and p, then the reflector of the pivot column
            if (lane == 0) {
                const double sj = nrm[p];  // squared norm of the pivot column, rows j..ell-1
                const double alpha = W[p * ldw + j];
                if (p != j) {
                    W[p * ldw + j] = W[j * ldw + j];
                    W[j * ldw + j] = alpha;
                    const int t = pv[j];
                    pv[j] = pv[p];
                    pv[p] = t;
                }
                // beta = -sign(alpha) |x| (sign(+-0) = +), tau = (beta - alpha) / beta,
                // scale = 1 / (alpha - beta); the sign taken by integer bit tests and the
                // zero-column test kept off the dependent chain
                const long long ab = __double_as_longlong(alpha);
                const bool neg = ab < 0 && (ab & 0x7fffffffffffffffLL) != 0;
                const double y = rsqrt_nr(sj);  // 1 / |column| (unused when the column is zero)
                const double nr = sj * y;
                const double beta_c = neg ? nr : -nr;
                const double inv_beta = neg ? y : -y;
                const double t_c = fma(-alpha, inv_beta, 1.0);
                const double scale_c = rcp_nr(alpha - beta_c);
                // H = I when the part below the diagonal is exactly zero
                const bool reflect = sj != alpha * alpha;
                const double beta = reflect ? beta_c : alpha;
                const double t = reflect ? t_c : 0.0;
                const double scale = reflect ? scale_c : 0.0;
                sc_beta = beta;
                sc_tau = t;
                sc_scale = scale;
                sc_ts = t * scale;
                tau[j] = t;
            }
        } else {
            // warps 1-8: the other rows of columns j and p
            if (p != j)
                for (int i = tid - 32; i < ell; i += kQrcpThreads - 32)
                    if (i != j) {
                        const double t = W[j * ldw + i];
                        W[j * ldw + i] = W[p * ldw + i];
                        W[p * ldw + i] = t;
                    }
            asm volatile("bar.sync 1, %0;" ::"n"(kQrcpThreads - 32) : "memory");
            // S2: t_c = x_j[j+1:]^T x_c[j+1:] (warps 1-3, 5-7) || staging of column j (warps 4, 8)
            if (warp != 4 && warp != 8) {
                const int t2 = (warp - (warp > 4 ? 2 : 1)) * 32 + lane;  // 0 .. 191
                const int g2 = qr_group(nc > 0 ? nc : 1, ell - j - 1 > 0 ? ell - j - 1 : 1, kQrcpDotThreads);
                const int c2 = j + 1 + t2 / g2, ph2 = t2 % g2;
                double tc = 0.0;
                if (c2 < ell) {
                    const double* x = W + j * ldw;
                    const double* y = W + c2 * ldw;
                    double s0 = 0.0, s1 = 0.0;
                    int i = j + 1 + ph2;
                    for (; i + g2 < ell; i += 2 * g2) {
                        s0 = fma(x[i], y[i], s0);
                        s1 = fma(x[i + g2], y[i + g2], s1);
                    }
                    if (i < ell) s0 = fma(x[i], y[i], s0);
                    tc = s0 + s1;
                }
                tc = group_sum(tc, g2);
                if (c2 < ell && ph2 == 0) tdot[c2] = tc;
            } else {
                for (int i = j + 1 + lane + (warp == 8 ? 32 : 0); i < ell; i += 64) xbuf[i] = W[j * ldw + i];
            }
        }
        __syncthreads();
        const int g = qr_group(nc > 0 ? nc : 1, ell - j);
        const int c = j + 1 + tid / g, ph = tid % g;
        const bool act = mapped && c < ell;
        // S3: apply H_j to columns c > j, accumulating their squared norms over rows > j
        //     (warps 0-7) || finish column j: v below the diagonal, beta on it (warp 8)
        if (mapped) {
            double acc = 0.0, xjc = 0.0, f = 0.0, fs = 0.0;
            double* y = W + (act ? c : j) * ldw;
            if (act) {
                xjc = y[j];
                const double w = fma(sc_scale, tdot[c], xjc);  // v^T x_c
                f = sc_tau * w;
                fs = sc_ts * w;
            }
            __syncwarp();  // every lane of the group has read x_c[j] before lane 0 rewrites it
            if (act) {
                int i = j + ph;
                if (i == j) {
                    y[j] = xjc - f;
                    i += g;
                }
                for (; i < ell; i += g) {
                    const double nv = fma(-xbuf[i], fs, y[i]);
                    y[i] = nv;
                    acc = fma(nv, nv, acc);
                }
            }
            acc = group_sum(acc, g);
            if (act && ph == 0) nrm[c] = acc;
        } else if (sc_tau != 0.0) {
            const double scale = sc_scale;
            for (int i = j + 1 + lane; i < ell; i += 32) W[j * ldw + i] = xbuf[i] * scale;
            if (lane == 0) W[j * ldw + j] = sc_beta;
        }
        __syncthreads();
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
    pdl_trigger();  // the Q formation may launch while the reflectors are written
    // reflectors for the Q formation: V column-major (v_j below the diagonal of
    // column j, zero elsewhere), then tau, then the column signs of Qt
    for (int e = tid; e < ell * ell; e += kQrcpThreads) {
        const int jj = e / ell, i = e % ell;
        refl[e] = i > jj ? W[jj * ldw + i] : 0.0;
    }
    for (int c = tid; c < ell; c += kQrcpThreads) {
        refl[ell * ell + c] = tau[c];
        refl[ell * ell + ell + c] = sgn[c];
    }
}

__global__ void __launch_bounds__(kQrcpThreads)
qrcp_kernel(const double* d, int ell, double* refl, double* rt, int* perm, const int* cancel) {
    qrcp_body(d, ell, refl, rt, perm, cancel);
}

// ---------------------------------------------------------------------------
// QRCP of D (eq. 8) on a cluster of kQcCtas CTAs (one per SM), for
// 64 < ell <= 128: the same Businger-Golub steps as qrcp_kernel -- recomputed
// norms, the pivot key of qr_pivot (norms within 2^-45 relative are ties,
// lowest position first), Householder reflections, diag(Rt) >= 0 -- with the
// FP64 trailing update spread over the cluster's SMs. Physical column c lives
// in CTA c mod kQcCtas; pivoting permutes positions in replicated tables
// instead of moving columns. One cluster barrier per step: after its update
// every CTA pushes to all CTAs (distributed shared memory, double-buffered by
// step parity) its best pivot key, that column's squared norm and its entries
// from the step's row down; after the barrier every CTA forms the winner's
// reflector itself (the same inputs, so bitwise the same v, tau, beta), the
// winner stores it in its column, and every CTA updates its other columns.
// Every CTA runs the same barriers in the same order (no data-dependent exit).
// ---------------------------------------------------------------------------
constexpr int kQcCtas = 8;
constexpr int kQcThreads = 256;
constexpr int kQcCols = 128 / kQcCtas;  // columns per CTA at most (two per warp)
constexpr int kQcLd = 129;              // odd column stride in shared memory
static_assert(kQcCols == 2 * (kQcThreads / 32), "one column per half-warp in one round");

__global__ void __cluster_dims__(kQcCtas, 1, 1) __launch_bounds__(kQcThreads)
qrcp_cluster_kernel(const double* d, int ell, double* refl, double* rt, int* perm, const int* cancel) {
    namespace cg = cooperative_groups;
    pdl_wait();
    if (cancel && *cancel) return;  // uniform over the cluster, before any barrier
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double W[kQcCols * kQcLd];       // own columns, local index lc = c / kQcCtas
    __shared__ double nrm[kQcCols];
    __shared__ double cand[2][kQcCtas][128];    // each CTA's candidate column (rows from the step down)
    __shared__ double cnrm[2][kQcCtas];         // its squared norm
    __shared__ long long keys[2][kQcCtas];      // its pivot key (-1: no column left)
    __shared__ double vbuf[128];                // v of the current step
    __shared__ double taus[128], betas[128];    // per step (replicated)
    __shared__ int pos_of[128], phys_at[128];   // replicated position tables
    __shared__ double sc_beta, sc_tau, sc_scale;
    __shared__ int sc_lc;                       // own local column of the next candidate (-1: none)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cluster.block_rank();
    const int nloc = ell > rank ? (ell - rank + kQcCtas - 1) / kQcCtas : 0;  // own columns
    for (int e = tid; e < nloc * ell; e += kQcThreads) {
        const int lc = e / ell, i = e - lc * ell;
        W[lc * kQcLd + i] = d[(size_t)i * ell + (lc * kQcCtas + rank)];  // d row-major: (i, c)
    }
    for (int c = tid; c < ell; c += kQcThreads) {
        pos_of[c] = c;
        phys_at[c] = c;
    }
    __syncthreads();
    for (int lc = warp; lc < nloc; lc += kQcThreads / 32) {
        double s = 0.0;
        for (int i = lane; i < ell; i += 32) s = fma(W[lc * kQcLd + i], W[lc * kQcLd + i], s);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm[lc] = s;
    }
    __syncthreads();
    // own best candidate for step j, pushed into buffer j & 1 of every CTA
    auto push_candidate = [&](int j) {
        const int b = j & 1;
        if (warp == 0) {
            long long best = -1;
            int blc = -1;
            for (int lc = lane; lc < nloc; lc += 32) {
                const int pc = pos_of[lc * kQcCtas + rank];
                if (pc >= j) {
                    const long long key = (__double_as_longlong(nrm[lc]) & ~0x7fLL) | (127 - pc);
                    if (key > best) {
                        best = key;
                        blc = lc;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int ol = __shfl_xor_sync(0xffffffffu, blc, o);
                if (ob > best) {
                    best = ob;
                    blc = ol;
                }
            }
            if (lane < kQcCtas) {
                cluster.map_shared_rank(&keys[b][0], lane)[rank] = best;
                cluster.map_shared_rank(&cnrm[b][0], lane)[rank] = blc >= 0 ? nrm[blc] : 0.0;
            }
            if (lane == 0) sc_lc = blc;
        }
        __syncthreads();
        const int blc = sc_lc;
        if (blc >= 0)
            for (int e = tid; e < kQcCtas * (ell - j); e += kQcThreads) {
                const int r = e / (ell - j), i = j + (e - r * (ell - j));
                cluster.map_shared_rank(&cand[b][0][0], r)[rank * 128 + i] = W[blc * kQcLd + i];
            }
    };
    push_candidate(0);
    for (int j = 0; j < ell; ++j) {
        const int b = j & 1;
        cluster.sync();  // every candidate of step j pushed (and every CTA done with step j-1)
        long long best = keys[b][0];
        int wr = 0;
#pragma unroll
        for (int r = 1; r < kQcCtas; ++r)
            if (keys[b][r] > best) {
                best = keys[b][r];
                wr = r;
            }
        const int pp = 127 - (int)(best & 0x7f);  // position of the pivot
        const int p = phys_at[pp];
        const double* x = &cand[b][wr][0];
        __syncthreads();  // every thread read the tables before thread 0 swaps
        if (tid == 0) {
            // positions j and pp swap (the same update in every CTA)
            if (pp != j) {
                const int pj = phys_at[j];
                phys_at[j] = p;
                phys_at[pp] = pj;
                pos_of[p] = j;
                pos_of[pj] = pp;
            }
            // beta = -sign(alpha) |x| (sign(+-0) = +), tau = (beta - alpha) / beta,
            // scale = 1 / (alpha - beta); H = I when the part below row j is exactly zero
            const double sj = cnrm[b][wr];
            const double alpha = x[j];
            const long long ab = __double_as_longlong(alpha);
            const bool neg = ab < 0 && (ab & 0x7fffffffffffffffLL) != 0;
            const double y = rsqrt_nr(sj);
            const double nr = sj * y;
            const double beta_c = neg ? nr : -nr;
            const double inv_beta = neg ? y : -y;
            const double t_c = fma(-alpha, inv_beta, 1.0);
            const double scale_c = rcp_nr(alpha - beta_c);
            const bool reflect = sj != alpha * alpha;
            sc_beta = reflect ? beta_c : alpha;
            sc_tau = reflect ? t_c : 0.0;
            sc_scale = reflect ? scale_c : 0.0;
            taus[j] = sc_tau;
            betas[j] = sc_beta;
        }
        __syncthreads();
        const double tj = sc_tau, scale = sc_scale;
        for (int i = j + 1 + tid; i < ell; i += kQcThreads) vbuf[i] = tj != 0.0 ? x[i] * scale : 0.0;
        __syncthreads();
        if (wr == rank) {  // the pivot column is own: it keeps v below the diagonal and beta on it
            double* xo = W + (p / kQcCtas) * kQcLd;
            for (int i = j + 1 + tid; i < ell; i += kQcThreads) xo[i] = vbuf[i];
            if (tid == 0) xo[j] = sc_beta;
        }
        // H_j on the own columns at positions > j, and their squared norms over
        // rows > j: two columns per warp, one per half-warp, so that each FP64
        // reduction instruction serves both
        {
            const int half = lane >> 4, hl = lane & 15;
            const int lc = 2 * warp + half;  // kQcCols = 16 = 2 x 8 warps: one round
            const bool act = lc < nloc && pos_of[lc * kQcCtas + rank] > j;
            double* xc = W + (act ? lc : 0) * kQcLd;
            double part = 0.0;
            if (act)
                for (int i = j + 1 + hl; i < ell; i += 16) part = fma(vbuf[i], xc[i], part);
#pragma unroll
            for (int o = 8; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const double f = act ? tj * (xc[j] + part) : 0.0;  // v^T x_c with v_j = 1
            double acc = 0.0;
            if (act)
                for (int i = j + 1 + hl; i < ell; i += 16) {
                    const double nv = fma(-f, vbuf[i], xc[i]);
                    xc[i] = nv;
                    acc = fma(nv, nv, acc);
                }
#pragma unroll
            for (int o = 8; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            __syncwarp();  // every lane read x_c[j] before its half's lane 0 rewrites it
            if (act && hl == 0) {
                xc[j] -= f;
                nrm[lc] = acc;
            }
        }
        __syncthreads();
        if (j + 1 < ell) push_candidate(j + 1);
    }
    cluster.sync();  // no CTA leaves while another may still write into its shared memory
    pdl_trigger();
    // Rt (row-major) column by column: rows <= position scaled by the sign of
    // their diagonal, zero below; V below the diagonal of each column
    for (int e = tid; e < nloc * ell; e += kQcThreads) {
        const int lc = e / ell, i = e - lc * ell;
        const int c = lc * kQcCtas + rank;
        const int pc = pos_of[c];
        const double w = W[lc * kQcLd + i];
        const double si = betas[i] < 0.0 ? -1.0 : 1.0;
        rt[(size_t)i * ell + pc] = i <= pc ? si * w : 0.0;
        refl[(size_t)pc * ell + i] = i > pc ? w : 0.0;
    }
    if (rank == 0)
        for (int c = tid; c < ell; c += kQcThreads) {
            perm[c] = phys_at[c];
            refl[(size_t)ell * ell + c] = taus[c];
            refl[(size_t)ell * ell + ell + c] = betas[c] < 0.0 ? -1.0 : 1.0;
        }
}

// Qt = H_0 H_1 ... H_{ell-1} diag(sgn). Column c of the product is
// H_0 H_1 ... H_c e_c (H_k leaves e_c alone for k > c), so the columns are
// independent: one warp per column (lanes own rows lane + 32 t, t < 4),
// applying H_c, H_{c-1}, ..., H_0 in turn with a warp-wide dot product each,
// two warps per block (ceil(ell / 2) blocks) so that each warp has a
// sub-partition's FP64 pipe to itself: a warp's steps are bound by that pipe
// (about 13 FP64 warp instructions per reflector), not by the other warps.
// V, tau and the signs are staged in shared memory.
constexpr int kQformWarps = 2;

__global__ void __launch_bounds__(kQformWarps * 32)
qform_kernel(const double* refl, int ell, double* qt, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ double Vs[];  // ell * ell + 2 * ell
    // the reflectors this block's columns use (k <= its last column), 16 loads
    // per thread in flight before their stores; then tau and the signs
    const int cmax = min(ell - 1, (int)blockIdx.x * kQformWarps + kQformWarps - 1);
    const int nv = (cmax + 1) * ell;
    constexpr int kB = 16;
    for (int e0 = 0; e0 < nv; e0 += kB * (int)blockDim.x) {
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * (int)blockDim.x + (int)threadIdx.x;
            v[u] = e < nv ? refl[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * (int)blockDim.x + (int)threadIdx.x;
            if (e < nv) Vs[e] = v[u];
        }
    }
    for (int e = threadIdx.x; e < 2 * ell; e += blockDim.x) Vs[ell * ell + e] = refl[ell * ell + e];
    __syncthreads();
    const double* tau = Vs + ell * ell;
    const double* sgn = tau + ell;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kQformWarps + (threadIdx.x >> 5);
    if (c >= ell) return;
    double q[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) q[t] = (lane + 32 * t == c) ? 1.0 : 0.0;
    for (int k = c; k >= 0; --k) {
        const double* v = Vs + k * ell;  // v[k] = 1 implied, v[i] = 0 for i < k
        double part = 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i < ell) part = fma(i == k ? 1.0 : v[i], q[t], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double f = tau[k] * part;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = lane + 32 * t;
            if (i >= k && i < ell) q[t] = fma(-f, i == k ? 1.0 : v[i], q[t]);
        }
    }
    pdl_trigger();
    const double sc = sgn[c];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int i = lane + 32 * t;
        if (i < ell) qt[(size_t)i * ell + c] = q[t] * sc;
    }
}

// U = Q1 Qt without forming Qt: each row x of Q1 is multiplied from the right
// by H_0, H_1, ..., H_{ell-1} (H_j = I - tau_j v_j v_j^T, v_j[j] = 1) and by
// diag(sgn), the reflectors and column signs the QRCP kernel wrote. Four
// adjacent lanes share a row (lane s owns the entries i = s mod 4); per
// reflector each lane forms its part of v_j^T x, two xor shuffles add the
// parts, and each lane updates its own entries. 32 rows per block.
template <typename TI, typename TC, typename TO>
__device__ __forceinline__ void apply_refl_body(const TI* x, int64_t ldx, int64_t rows, int ell, const double* refl,
                                                TO* out, int64_t ldo, int out_panel, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* Vs = reinterpret_cast<TC*>(smem_raw);   // ell x ell: column j = v_j (below the diagonal)
    TC* tau = Vs + ell * ell;
    TC* sgn = tau + ell;
    TC* Ts = sgn + ell;                         // [kTrsmRows][ld]
    const int ld = trsm_ld(ell);
    const int tid = threadIdx.x;
    const int ln = tid & (kTrsmL - 1), rr = tid / kTrsmL;
    constexpr int kB = 16;
    const int nv = ell * ell + 2 * ell;
    for (int e0 = 0; e0 < nv; e0 += kB * kTrsmThreads) {
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kTrsmThreads + tid;
            v[u] = e < nv ? refl[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int e = e0 + u * kTrsmThreads + tid;
            if (e < nv) Vs[e] = (TC)v[u];  // Vs, tau, sgn are contiguous like refl
        }
    }
    const int64_t i0 = (int64_t)blockIdx.x * kTrsmRows + rr;
    const bool live = i0 < rows;
    for (int j0 = ln; j0 < ell; j0 += kTrsmL * kB) {
        TI v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = j0 + kTrsmL * u;
            v[u] = (live && j < ell) ? x[(int64_t)j * ldx + i0] : (TI)0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = j0 + kTrsmL * u;
            if (j < ell) Ts[rr * ld + j] = (TC)v[u];
        }
    }
    __syncthreads();
    pdl_trigger();
    for (int j = 0; j < ell; ++j) {
        const TC* vj = Vs + j * ell;
        // first entry of this lane at or after j
        const int i_beg = j + ((ln - j) & (kTrsmL - 1));
        // four independent partial sums: the loads and FMAs of a lane overlap
        TC p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        int i = i_beg;
        if (i == j) {
            p0 = Ts[rr * ld + i];  // v_j[j] = 1
            i += kTrsmL;
        }
        for (; i + 3 * kTrsmL < ell; i += 4 * kTrsmL) {
            p0 += vj[i] * Ts[rr * ld + i];
            p1 += vj[i + kTrsmL] * Ts[rr * ld + i + kTrsmL];
            p2 += vj[i + 2 * kTrsmL] * Ts[rr * ld + i + 2 * kTrsmL];
            p3 += vj[i + 3 * kTrsmL] * Ts[rr * ld + i + 3 * kTrsmL];
        }
        for (; i < ell; i += kTrsmL) p0 += vj[i] * Ts[rr * ld + i];
        TC part = (p0 + p1) + (p2 + p3);
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        const TC f = tau[j] * part;
#pragma unroll 4
        for (int i2 = i_beg; i2 < ell; i2 += kTrsmL) Ts[rr * ld + i2] -= f * (i2 == j ? (TC)1 : vj[i2]);
    }
    if (!live) return;
    for (int i = ln; i < ell; i += kTrsmL) {
        const TC val = Ts[rr * ld + i] * sgn[i];
        if (out_panel) out[(int64_t)i * ldo + i0] = (TO)val;
        else out[i0 * ldo + i] = (TO)val;
    }
}

template <typename TI, typename TC, typename TO>
__global__ void __launch_bounds__(kTrsmThreads)
apply_refl_kernel(const TI* x, int64_t ldx, int64_t rows, int ell, const double* refl, TO* out, int64_t ldo,
                  int out_panel, const int* cancel) {
    apply_refl_body<TI, TC, TO>(x, ldx, rows, ell, refl, out, ldo, out_panel, cancel);
}

template <typename TQ, typename TV>
__device__ __forceinline__ void gather_v_body(const TQ* q2, int64_t ldq2, int64_t n, int ell, const int* perm,
                                              TV* v, int64_t ldv, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ double tile[128][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int tid = threadIdx.x;  // 256
    for (int j0 = 0; j0 < ell; j0 += 128) {  // column blocks of 128 (one for ell <= 128)
        const int nj = ell - j0 < 128 ? ell - j0 : 128;
        if (j0 > 0) __syncthreads();
        for (int e = tid; e < nj * 32; e += blockDim.x) {
            const int j = e / 32, ii = e % 32;
            const int64_t i = i0 + ii;
            tile[j][ii] = (i < n) ? (double)q2[(int64_t)perm[j0 + j] * ldq2 + i] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < nj * 32; e += blockDim.x) {
            const int ii = e / nj, j = e % nj;
            const int64_t i = i0 + ii;
            if (i < n) v[i * ldv + j0 + j] = (TV)tile[j][ii];
        }
    }
}

template <typename TQ, typename TV>
__global__ void gather_v_kernel(const TQ* q2, int64_t ldq2, int64_t n, int ell, const int* perm,
                                TV* v, int64_t ldv, const int* cancel) {
    gather_v_body<TQ, TV>(q2, ldq2, n, ell, perm, v, ldv, cancel);
}

// dst = src (ell x ell, row-major), or its transpose
template <typename TD>
__global__ void copy_small_kernel(const double* src, int ell, TD* dst, int transpose, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const int n = ell * ell;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int a = e / ell, c = e - a * ell;
        dst[e] = (TD)src[transpose ? c * ell + a : e];
    }
}


// ---------------------------------------------------------------------------
// The ell x ell steps for sketch widths 128 < ell <= 320 (SIMT paths only):
// one block each, the matrices in global memory (L2-resident: at most 800 KB)
// instead of one SM's shared memory. The same arithmetic as the one-SM
// kernels above, organised for correctness before speed: these widths serve
// the paper's larger RPCA problems (ell = 2k = 200, 300), not the throughput
// workloads.
// ---------------------------------------------------------------------------
constexpr int kBigThreads = 1024;
constexpr int kBigSlots = (kMaxEllSimt + 31) / 32;  // rows per lane of a one-warp column

// Cholesky with the contract of cholesky_kernel (shift passes, dependent
// columns, skip flag, status words), right-looking in the square-root-free
// form on R itself as the working matrix: p_t = S_tt, L_t = S_t / p_t,
// S_ac -= L_ta S_tc (t < a <= c), then R_tc = S_tc / sqrt(p_t).
template <bool kDefic>
__global__ void __launch_bounds__(kBigThreads)
cholesky_big_kernel(const double* g, int ell, int64_t rows, double* r, int* flags, int* skip_out,
                    const int* cancel, double unit_roundoff, int* defic, double tau_rel) {
    pdl_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (cancel && *cancel) {
        if (skip_out && tid == 0) *skip_out = 1;
        return;
    }
    __shared__ double L[kMaxEllSimt];
    __shared__ double ys[kMaxEllSimt];
    __shared__ int rowdep[kMaxEllSimt];
    __shared__ double rt_s, trace_s, dmin_s;
    __shared__ int fail_s;
    if (warp == 0) {
        double mx = 0.0, tr = 0.0;
        for (int a = lane; a < ell; a += 32) {
            mx = fmax(mx, g[(size_t)a * ell + a]);
            tr += g[(size_t)a * ell + a];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            tr += __shfl_xor_sync(0xffffffffu, tr, o);
        }
        if (lane == 0) {
            dmin_s = tau_rel * mx;
            trace_s = tr;
        }
    }
    __syncthreads();
    const double dmin = kDefic ? dmin_s : 0.0;
    int attempt = 0;
    for (; attempt < 3; ++attempt) {
        // shift s = 11 (rows ell + ell (ell + 1)) u ||C||_F^2 (Fukaya et al.), then x100
        const double shift = attempt == 0 ? 0.0
                                          : 11.0 * ((double)rows * ell + (double)ell * (ell + 1)) * unit_roundoff *
                                                trace_s * (attempt == 1 ? 1.0 : 100.0);
        for (int e = tid; e < ell * ell; e += kBigThreads) {
            const int a = e / ell, c = e - a * ell;
            r[e] = a == c ? g[e] + shift : g[e];
        }
        for (int a = tid; a < ell; a += kBigThreads) {
            rowdep[a] = 0;
            if (kDefic) defic[a] = 0;
        }
        if (tid == 0) fail_s = 0;
        __syncthreads();
        for (int t = 0; t < ell; ++t) {
            if (tid == 0) {
                const double p = r[(size_t)t * ell + t];
                const bool dep = kDefic && !gt_nonneg(p, dmin);
                if (!(dep || pos_finite(p))) fail_s = 1;
                if (dep) {
                    rowdep[t] = 1;
                    defic[t] = 1;
                }
                rt_s = dep ? 0.0 : rcp_nr(p);
            }
            __syncthreads();
            if (fail_s) break;
            const double rt = rt_s;
            for (int c = t + tid; c < ell; c += kBigThreads) L[c] = r[(size_t)t * ell + c] * rt;
            __syncthreads();
            for (int a = t + 1 + warp; a < ell; a += kBigThreads / 32) {
                const double la = L[a];
                double* ra = r + (size_t)a * ell;
                const double* rtt = r + (size_t)t * ell;
                for (int c = a + lane; c < ell; c += 32) ra[c] = fma(-la, rtt[c], ra[c]);
            }
            __syncthreads();
        }
        const bool failed = fail_s != 0;
        __syncthreads();
        if (!failed) break;
    }
    pdl_trigger();
    const bool broke = attempt == 3;
    for (int t = tid; t < ell; t += kBigThreads)
        ys[t] = (broke || rowdep[t]) ? 0.0 : rsqrt_nr(r[(size_t)t * ell + t]);
    __syncthreads();
    for (int e = tid; e < ell * ell; e += kBigThreads) {
        const int a = e / ell, c = e - a * ell;
        const bool unit = broke || rowdep[a];
        const double x = c >= a ? r[e] * ys[a] : 0.0;
        r[e] = c < a ? 0.0 : (unit ? (a == c ? 1.0 : 0.0) : x);
    }
    if (tid == 0) {
        if (broke) atomicExch(&flags[FLAG_BREAKDOWN], 1);
        if (attempt > 0) atomicAdd(&flags[FLAG_SHIFTED], 1);
        if (skip_out) *skip_out = (attempt > 0 && !broke) ? 0 : 1;
    }
}

// R^{-1} (type T, ell x ldri row-major, zero below the diagonal and beyond
// column ell) by column-oriented back substitution, one warp per column
// (lane l keeps rows l + 32 s), R read from global memory.
template <typename T>
__global__ void __launch_bounds__(256) rinv_big_kernel(const double* r, int ell, T* ri, int ldri, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    const int lane = threadIdx.x & 31, j = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= ell) return;
    T b[kBigSlots];
#pragma unroll
    for (int s = 0; s < kBigSlots; ++s) b[s] = (lane + 32 * s == j) ? (T)1 : (T)0;
    for (int k = j; k >= 0; --k) {
        const int sk = k >> 5;
        T bk = b[0];
#pragma unroll
        for (int s = 1; s < kBigSlots; ++s)
            if (s == sk) bk = b[s];
        const T xk = __shfl_sync(0xffffffffu, bk, k & 31) / (T)r[(size_t)k * ell + k];
#pragma unroll
        for (int s = 0; s < kBigSlots; ++s) {
            const int i = lane + 32 * s;
            if (i < k) b[s] = fma(-(T)r[(size_t)i * ell + k], xk, b[s]);
            else if (i == k) b[s] = xk;
        }
    }
#pragma unroll
    for (int s = 0; s < kBigSlots; ++s) {
        const int i = lane + 32 * s;
        if (i < ell) ri[(size_t)i * ldri + j] = i <= j ? b[s] : (T)0;
    }
    if (j == ell - 1)
        for (int i = lane; i < ell; i += 32)
            for (int jj = ell; jj < ldri; ++jj) ri[(size_t)i * ldri + jj] = (T)0;
}

// After Q = C R^{-1} (as a product): columns the extra CholeskyQR pass found
// dependent get their random completion, and qc receives Q's copy.
template <typename TI, typename TQC>
__global__ void trsm_post_kernel(TI* q, int64_t ldq, int64_t rows, int ell, TQC* qc, int64_t ldqc, const int* defic,
                                 const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    const int64_t total = rows * ell;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / rows);
        const int64_t i = e - (int64_t)j * rows;
        TI v = q[(int64_t)j * ldq + i];
        if (defic && defic[j]) {
            v = (TI)completion_entry(i, j, rows);
            q[(int64_t)j * ldq + i] = v;
        }
        if (qc) qc[(int64_t)j * ldqc + i] = (TQC)v;
    }
}

// QRCP (eq. 8) with the contract of qrcp_kernel: Businger-Golub pivoting on
// column norms recomputed at every step, Householder reflections, diag(Rt) >= 0;
// the pivot is the largest norm, the lowest index among equal ones (exact
// comparison). W (column-major, column c at W + c * ell) is the reflector
// buffer itself: V, tau and the signs end there in qrcp_kernel's layout.
__global__ void __launch_bounds__(kBigThreads)
qrcp_big_kernel(const double* d, int ell, double* refl, double* rt, int* perm, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ double nrm[kMaxEllSimt];
    __shared__ double tau[kMaxEllSimt];
    __shared__ int pv[kMaxEllSimt];
    __shared__ double wv[32];
    __shared__ int wi[32];
    __shared__ double sc_tau, sc_scale, sc_beta;
    __shared__ int sc_p, sc_reflect;
    double* W = refl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = kBigThreads / 32;
    for (int e = tid; e < ell * ell; e += kBigThreads) {
        const int a = e / ell, b = e - a * ell;  // d row-major: (a, b) -> column b, row a
        W[(size_t)b * ell + a] = d[e];
    }
    for (int c = tid; c < ell; c += kBigThreads) pv[c] = c;
    __syncthreads();
    for (int c = warp; c < ell; c += nw) {
        double s = 0.0;
        for (int i = lane; i < ell; i += 32) s = fma(W[(size_t)c * ell + i], W[(size_t)c * ell + i], s);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
    for (int j = 0; j < ell; ++j) {
        // pivot: the largest recomputed norm among columns j.., the lowest index on ties
        {
            double bv = -1.0;
            int bi = ell;
            for (int c = j + tid; c < ell; c += kBigThreads)
                if (nrm[c] > bv || (nrm[c] == bv && c < bi)) {
                    bv = nrm[c];
                    bi = c;
                }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                wv[warp] = bv;
                wi[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double v = wv[0];
                int i = wi[0];
                for (int w = 1; w < nw; ++w)
                    if (wv[w] > v || (wv[w] == v && wi[w] < i)) {
                        v = wv[w];
                        i = wi[w];
                    }
                sc_p = i;
            }
            __syncthreads();
        }
        const int p = sc_p;
        if (p != j) {
            for (int i = tid; i < ell; i += kBigThreads) {
                const double t = W[(size_t)j * ell + i];
                W[(size_t)j * ell + i] = W[(size_t)p * ell + i];
                W[(size_t)p * ell + i] = t;
            }
            if (tid == 0) {
                const int t = pv[j];
                pv[j] = pv[p];
                pv[p] = t;
                const double s = nrm[j];
                nrm[j] = nrm[p];
                nrm[p] = s;
            }
        }
        __syncthreads();
        if (tid == 0) {
            // beta = -sign(alpha) |x| (sign(+-0) = +), tau = (beta - alpha) / beta,
            // v = x / (alpha - beta) below the diagonal; H = I when that part is exactly zero
            const double sj = nrm[j];
            const double alpha = W[(size_t)j * ell + j];
            const bool neg = alpha < 0.0;
            const double nr = sqrt(sj);
            const bool reflect = sj != alpha * alpha;
            const double beta = neg ? nr : -nr;
            sc_reflect = reflect ? 1 : 0;
            sc_beta = reflect ? beta : alpha;
            sc_tau = reflect ? (beta - alpha) / beta : 0.0;
            sc_scale = reflect ? 1.0 / (alpha - beta) : 0.0;
            tau[j] = sc_tau;
        }
        __syncthreads();
        if (sc_reflect)
            for (int i = j + 1 + tid; i < ell; i += kBigThreads) W[(size_t)j * ell + i] *= sc_scale;
        __syncthreads();
        const double tj = sc_tau;
        const double* v = W + (size_t)j * ell;
        for (int c = j + 1 + warp; c < ell; c += nw) {
            double* x = W + (size_t)c * ell;
            double part = 0.0;
            for (int i = j + 1 + lane; i < ell; i += 32) part = fma(v[i], x[i], part);
#pragma unroll
            for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            const double f = tj * (x[j] + part);  // v^T x_c with v_j = 1
            double acc = 0.0;
            for (int i = j + 1 + lane; i < ell; i += 32) {
                const double nv = fma(-f, v[i], x[i]);
                x[i] = nv;
                acc = fma(nv, nv, acc);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                x[j] -= f;
                nrm[c] = acc;
            }
        }
        __syncthreads();
        if (tid == 0) W[(size_t)j * ell + j] = sc_beta;
        __syncthreads();
    }
    // Rt = upper(W) with diag(Rt) >= 0 (row a scaled by the sign of its diagonal)
    for (int e = tid; e < ell * ell; e += kBigThreads) {
        const int a = e / ell, b = e - a * ell;
        const double sa = W[(size_t)a * ell + a] < 0.0 ? -1.0 : 1.0;
        rt[e] = b >= a ? sa * W[(size_t)b * ell + a] : 0.0;
    }
    for (int c = tid; c < ell; c += kBigThreads) perm[c] = pv[c];
    __syncthreads();
    pdl_trigger();
    // tau and the signs after V; then V keeps only the part below the diagonal
    for (int c = tid; c < ell; c += kBigThreads) {
        refl[(size_t)ell * ell + c] = tau[c];
        refl[(size_t)ell * ell + ell + c] = W[(size_t)c * ell + c] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (int e = tid; e < ell * ell; e += kBigThreads) {
        const int jj = e / ell, i = e - jj * ell;
        if (i <= jj) W[e] = 0.0;
    }
}

// Qt = H_0 ... H_{ell-1} diag(sgn) column by column, one warp per column,
// the reflectors read from global memory.
__global__ void __launch_bounds__(256) qform_big_kernel(const double* refl, int ell, double* qt, const int* cancel) {
    pdl_wait();
    if (cancel && *cancel) return;
    const double* tau = refl + (size_t)ell * ell;
    const double* sgn = tau + ell;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= ell) return;
    double q[kBigSlots];
#pragma unroll
    for (int t = 0; t < kBigSlots; ++t) q[t] = (lane + 32 * t == c) ? 1.0 : 0.0;
    for (int k = c; k >= 0; --k) {
        const double* v = refl + (size_t)k * ell;  // v[k] = 1 implied, v[i] = 0 for i < k
        double part = 0.0;
#pragma unroll
        for (int t = 0; t < kBigSlots; ++t) {
            const int i = lane + 32 * t;
            if (i < ell) part = fma(i == k ? 1.0 : v[i], q[t], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double f = tau[k] * part;
#pragma unroll
        for (int t = 0; t < kBigSlots; ++t) {
            const int i = lane + 32 * t;
            if (i >= k && i < ell) q[t] = fma(-f, i == k ? 1.0 : v[i], q[t]);
        }
    }
    const double sc = sgn[c];
#pragma unroll
    for (int t = 0; t < kBigSlots; ++t) {
        const int i = lane + 32 * t;
        if (i < ell) qt[(size_t)i * ell + c] = q[t] * sc;
    }
}


}  // namespace

cudaError_t launch_trimul(const double* rn, const double* ra, double* out, int64_t ell, bool transpose,
                          const int* skip, const int* cancel, cudaStream_t st) {
    if (ell < 1 || ell > kMaxEllSimt || out == rn || out == ra) return cudaErrorInvalidValue;
    count_launch();
    cudaError_t e = launch_pdl(trimul_kernel, dim3((unsigned)ell), dim3(ell > 128 ? (unsigned)((ell + 31) / 32 * 32) : 128u),
                               (size_t)0, st, rn, ra, out, (int)ell,
                               transpose ? 1 : 0, skip, cancel);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_cholesky(const double* g, int64_t ell, int64_t rows, double* r, int* flags,
                               int* skip_out, const int* cancel, cudaStream_t st, double unit_roundoff,
                               int* defic, double tau_rel) {
    if (ell < 1 || ell > kMaxEllSimt) return cudaErrorInvalidValue;
    if (ell > kCholMaxEll) {
        count_launch();
        cudaError_t pe = defic ? launch_pdl(cholesky_big_kernel<true>, dim3(1), dim3(kBigThreads), (size_t)0, st, g, (int)ell,
                                            rows, r, flags, skip_out, cancel, unit_roundoff, defic, tau_rel)
                               : launch_pdl(cholesky_big_kernel<false>, dim3(1), dim3(kBigThreads), (size_t)0, st, g,
                                            (int)ell, rows, r, flags, skip_out, cancel, unit_roundoff, defic, tau_rel);
        return pe != cudaSuccess ? pe : cudaGetLastError();
    }
    const size_t smem = sizeof(double) * (size_t)ell * (ell + 1) + sizeof(unsigned short) * (size_t)ell * (ell + 1) / 2;
    auto kern = defic ? cholesky_kernel<true> : cholesky_kernel<false>;
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(kern, dim3(1), dim3(kCholThreads), smem, st, g, (int)ell, rows, r, flags,
                                     skip_out, cancel, unit_roundoff, defic, tau_rel);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

// Q = C R^{-1} for 128 < ell <= 320: R^{-1} (rinv_big_kernel, into rinv_work),
// then the product in column groups of at most 128, the last group first so
// that an in-place solve (q == c) reads only columns it has not overwritten
// (group J needs C's columns up to its own last one: R^{-1} is upper
// triangular), then the dependent columns' completion and the copy qc.
cudaError_t trsm_big(const void* c, ElemType tp, int64_t ldc, int64_t rows, int ell, const double* r, ElemType tc,
                     void* q, int64_t ldq, void* qc, ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st,
                     const int* defic, void* rinv_work) {
    if (!rinv_work || ell > kMaxEllSimt || tp != tc || (tp != T_F64 && tp != T_F32)) return cudaErrorInvalidValue;
    const int ldri = (ell + 7) & ~7;
    const unsigned rb = (unsigned)((ell + 7) / 8);
    count_launch();
    cudaError_t e = tc == T_F64 ? launch_pdl(rinv_big_kernel<double>, dim3(rb), dim3(256), (size_t)0, st, r, ell,
                                             static_cast<double*>(rinv_work), ldri, cancel)
                                : launch_pdl(rinv_big_kernel<float>, dim3(rb), dim3(256), (size_t)0, st, r, ell,
                                             static_cast<float*>(rinv_work), ldri, cancel);
    if (e != cudaSuccess) return e;
    const int64_t es = elem_size(tc);
    for (int64_t j0 = (int64_t)(ell - 1) / 128 * 128; j0 >= 0; j0 -= 128) {
        const int64_t L = std::min<int64_t>(128, ell - j0);
        GemmArgs g{A_PANEL, B_SMALL, O_PANEL, tp, tc, c, ldc,
                   static_cast<const char*>(rinv_work) + j0 * es, ldri,
                   static_cast<char*>(q) + j0 * ldq * es, ldq, 0, rows, j0 + L, L, 1, cancel};
        e = launch_gemm_simt(g, st);
        if (e != cudaSuccess) return e;
    }
    if (!defic && !qc) return cudaSuccess;
    const int64_t total = rows * ell;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    count_launch();
    auto post = [&](auto* qp, auto* qcp) {
        return launch_pdl(trsm_post_kernel<std::remove_pointer_t<decltype(qp)>, std::remove_pointer_t<decltype(qcp)>>,
                          dim3(blocks), dim3(256), (size_t)0, st, qp, ldq, rows, ell, qcp, ldqc, defic, cancel);
    };
    if (tp == T_F64) {
        double* qp = static_cast<double*>(q);
        if (!qc || tqc == T_F64) e = post(qp, static_cast<double*>(qc));
        else if (tqc == T_F32) e = post(qp, static_cast<float*>(qc));
        else return cudaErrorInvalidValue;
    } else {
        float* qp = static_cast<float*>(q);
        if (!qc || tqc == T_F32) e = post(qp, static_cast<float*>(qc));
        else if (tqc == T_F64) e = post(qp, static_cast<double*>(qc));
        else return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_trsm_rows(const void* c, ElemType tp, int64_t ldc, int64_t rows, int64_t ell,
                             const double* r, ElemType tc, void* q, int64_t ldq, void* qc,
                             ElemType tqc, int64_t ldqc, const int* cancel, cudaStream_t st,
                             const int* defic, float* rinv_work) {
    const int l = (int)ell;
    if (l > 128) return trsm_big(c, tp, ldc, rows, l, r, tc, q, ldq, qc, tqc, ldqc, cancel, st, defic, rinv_work);
    auto al16 = [](const void* p, int64_t ld) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0; };
    if (tp == T_F32 && tc == T_F32 && rinv_work && l >= 1 && l <= 128 && al16(c, ldc) && al16(q, ldq) &&
        (reinterpret_cast<uintptr_t>(rinv_work) & 15) == 0) {
        const float* cf = static_cast<const float*>(c);
        float* qf = static_cast<float*>(q);
        switch (qc ? tqc : T_F32) {
            case T_F32: return trsm_inv_launch<float>(cf, ldc, rows, l, r, rinv_work, qf, ldq, static_cast<float*>(qc), ldqc, cancel, st, defic);
            case T_F64: return trsm_inv_launch<double>(cf, ldc, rows, l, r, rinv_work, qf, ldq, static_cast<double*>(qc), ldqc, cancel, st, defic);
            case T_BF16: return trsm_inv_launch<__nv_bfloat16>(cf, ldc, rows, l, r, rinv_work, qf, ldq, static_cast<__nv_bfloat16*>(qc), ldqc, cancel, st, defic);
            default: return cudaErrorInvalidValue;
        }
    }
    if (tp == T_F64 && tc == T_F64) return trsm_dispatch<double, double>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st, defic);
    if (tp == T_F64 && tc == T_F32) return trsm_dispatch<double, float>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st, defic);
    if (tp == T_F32 && tc == T_F32) return trsm_dispatch<float, float>(c, ldc, rows, l, r, q, ldq, qc, tqc, ldqc, cancel, st, defic);
    return cudaErrorInvalidValue;
}

cudaError_t launch_qform(const double* refl, int64_t ell, double* qt, const int* cancel, cudaStream_t st) {
    if (ell < 1 || ell > kMaxEllSimt) return cudaErrorInvalidValue;
    count_launch();
    cudaError_t e;
    if (ell > 128) {
        e = launch_pdl(qform_big_kernel, dim3((unsigned)((ell + 7) / 8)), dim3(256), (size_t)0, st, refl, (int)ell, qt,
                       cancel);
    } else {
        const size_t smem_q = sizeof(double) * (size_t)(ell * ell + 2 * ell);
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(qform_kernel));
        if (e != cudaSuccess) return e;
        e = launch_pdl(qform_kernel, dim3((unsigned)((ell + kQformWarps - 1) / kQformWarps)), dim3(kQformWarps * 32),
                       smem_q, st, refl, (int)ell, qt, cancel);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_qrcp(const double* d, int64_t ell, double* qt, double* rt, int* perm, double* work,
                        const int* cancel, cudaStream_t st, bool form_q) {
    if (ell < 1 || ell > kMaxEllSimt || !work) return cudaErrorInvalidValue;
    if (ell > 128) {
        count_launch();
        cudaError_t pe = launch_pdl(qrcp_big_kernel, dim3(1), dim3(kBigThreads), (size_t)0, st, d, (int)ell, work, rt,
                                    perm, cancel);
        if (pe != cudaSuccess || !form_q) return pe != cudaSuccess ? pe : cudaGetLastError();
        return launch_qform(work, ell, qt, cancel, st);
    }
    cudaError_t e;
    count_launch();
    if (ell > 64) {
        // the trailing updates of the wider cores spread over a cluster of SMs
        // (617 -> 430 us at ell = 110, 872 -> 537 us at 128; 201 -> 197 us at 65)
        e = launch_pdl(qrcp_cluster_kernel, dim3(kQcCtas), dim3(kQcThreads), (size_t)0, st, d, (int)ell, work, rt, perm,
                       cancel);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem = sizeof(double) * ((size_t)ell * (ell | 1) + 5 * (size_t)ell) + sizeof(int) * ell;
        e = allow_max_dynamic_smem(reinterpret_cast<const void*>(qrcp_kernel));
        if (e != cudaSuccess) return e;
        e = launch_pdl(qrcp_kernel, dim3(1), dim3(kQrcpThreads), (size_t)(smem), st, d, (int)ell, work, rt, perm, cancel);
        if (e != cudaSuccess) return e;
    }
    if (!form_q) return cudaSuccess;
    return launch_qform(work, ell, qt, cancel, st);
}

// The same product for FP32 arithmetic and ell <= 64 with one thread per row
// of Q1, the row held in registers: each reflector is a dot product and an
// update of register values against v_j broadcast from shared memory (four
// v entries per 128-bit load), with no shuffle and no shared-memory round
// trip on the row's chain. The 64 columns are taken in four blocks of 16 so
// that reflector j touches only the blocks at or after j's own.
constexpr int kRrThreads = 128;   // rows per block
template <typename TI, typename TO>
__device__ __forceinline__ void apply_refl_rows_body(const TI* x, int64_t ldx, int64_t rows, int ell,
                                                     const double* refl, TO* out, int64_t ldo, int out_panel,
                                                     const int* cancel) {
    constexpr int kE = 64, kLdv = 64;  // v_j at Vs + j * kLdv (16-byte aligned columns)
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ __align__(16) float Vs[kE * kLdv];
    __shared__ float tau[kE], sgn[kE];
    __shared__ float Os[kRrThreads * 33];        // 32 columns of the rows, for coalesced row-major stores
    const int tid = threadIdx.x;
    // v_j below the diagonal, zero elsewhere (including the padding), as FP32
    for (int e = tid; e < kE * kLdv; e += kRrThreads) {
        const int j = e / kLdv, i = e - j * kLdv;
        Vs[e] = (j < ell && i > j && i < ell) ? (float)refl[(size_t)j * ell + i] : 0.f;
    }
    for (int j = tid; j < kE; j += kRrThreads) {
        tau[j] = j < ell ? (float)refl[(size_t)ell * ell + j] : 0.f;
        sgn[j] = j < ell ? (float)refl[(size_t)ell * ell + ell + j] : 0.f;
    }
    const int64_t i0 = (int64_t)blockIdx.x * kRrThreads + tid;
    const bool live = i0 < rows;
    float u[kE];
#pragma unroll
    for (int i = 0; i < kE; ++i) u[i] = (live && i < ell) ? (float)x[(int64_t)i * ldx + i0] : 0.f;
    __syncthreads();
    pdl_trigger();
#pragma unroll
    for (int jb = 0; jb < kE / 16; ++jb) {
        const int jend = min(ell, 16 * (jb + 1));
        for (int j = 16 * jb; j < jend; ++j) {
            const float4* v4 = reinterpret_cast<const float4*>(Vs + j * kLdv);
            // v_j^T u with v_j[j] = 1: u[j] plus the entries below (zero in Vs above j)
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
            for (int c = 4 * jb; c < kE / 4; ++c) {
                const float4 v = v4[c];
                d0 = fmaf(v.x, u[4 * c + 0], d0);
                d1 = fmaf(v.y, u[4 * c + 1], d1);
                d2 = fmaf(v.z, u[4 * c + 2], d2);
                d3 = fmaf(v.w, u[4 * c + 3], d3);
            }
            float uj = 0.f;  // u[j] (a register of this block of 16, picked by value)
#pragma unroll
            for (int i = 16 * jb; i < 16 * (jb + 1); ++i) uj = (i == j) ? u[i] : uj;
            const float f = tau[j] * (uj + ((d0 + d1) + (d2 + d3)));
#pragma unroll
            for (int i = 16 * jb; i < 16 * (jb + 1); ++i)
                if (i == j) u[i] -= f;
#pragma unroll
            for (int c = 4 * jb; c < kE / 4; ++c) {
                const float4 v = v4[c];
                u[4 * c + 0] = fmaf(-f, v.x, u[4 * c + 0]);
                u[4 * c + 1] = fmaf(-f, v.y, u[4 * c + 1]);
                u[4 * c + 2] = fmaf(-f, v.z, u[4 * c + 2]);
                u[4 * c + 3] = fmaf(-f, v.w, u[4 * c + 3]);
            }
        }
    }
    if (out_panel) {
        if (live)
#pragma unroll
            for (int i = 0; i < kE; ++i)
                if (i < ell) out[(int64_t)i * ldo + i0] = (TO)(u[i] * sgn[i]);
        return;
    }
    // row-major, 32 columns at a time: consecutive threads store consecutive
    // entries of one row
    const int64_t r0 = (int64_t)blockIdx.x * kRrThreads;
#pragma unroll
    for (int cb = 0; cb < kE; cb += 32) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 32; ++i) Os[tid * 33 + i] = u[cb + i] * sgn[cb + i];
        __syncthreads();
        const int nc = min(32, ell - cb);
        for (int e = tid; e < kRrThreads * nc; e += kRrThreads) {
            const int r = e / nc, i = e - r * nc;
            if (r0 + r < rows) out[(r0 + r) * ldo + cb + i] = (TO)Os[r * 33 + i];
        }
    }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kRrThreads)
apply_refl_rows_kernel(const TI* x, int64_t ldx, int64_t rows, int ell, const double* refl, TO* out, int64_t ldo,
                       int out_panel, const int* cancel) {
    apply_refl_rows_body<TI, TO>(x, ldx, rows, ell, refl, out, ldo, out_panel, cancel);
}

cudaError_t launch_apply_reflectors(const void* q1, ElemType tp, int64_t ldq, int64_t rows, int64_t ell,
                                    const double* refl, void* out, ElemType tout, int64_t ldo, bool out_panel,
                                    const int* cancel, cudaStream_t st) {
    if (ell < 1 || ell > 128) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((rows + kTrsmRows - 1) / kTrsmRows);
    const int l = (int)ell;
    auto go = [&](auto kern, size_t tc_bytes, auto xin, auto outp) -> cudaError_t {
        const size_t smem = tc_bytes * ((size_t)ell * ell + 2 * (size_t)ell + (size_t)kTrsmRows * trsm_ld(l));
        cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
        if (e != cudaSuccess) return e;
        count_launch();
        return launch_pdl(kern, dim3(blocks), dim3(kTrsmThreads), smem, st, xin, ldq, rows, l, refl, outp, ldo,
                          out_panel ? 1 : 0, cancel);
    };
    if (tp == T_F32 && tout == T_F32 && ell <= 64) {  // the register-row form
        count_launch();
        return launch_pdl(apply_refl_rows_kernel<float, float>, dim3((unsigned)((rows + kRrThreads - 1) / kRrThreads)),
                          dim3(kRrThreads), (size_t)0, st, static_cast<const float*>(q1), ldq, rows, l, refl,
                          static_cast<float*>(out), ldo, out_panel ? 1 : 0, cancel);
    }
    if (tp == T_F32 && tout == T_F32)
        return go(apply_refl_kernel<float, float, float>, sizeof(float), static_cast<const float*>(q1),
                  static_cast<float*>(out));
    if (tp == T_F32 && tout == T_F64)
        return go(apply_refl_kernel<float, double, double>, sizeof(double), static_cast<const float*>(q1),
                  static_cast<double*>(out));
    if (tp == T_F64 && tout == T_F64)
        return go(apply_refl_kernel<double, double, double>, sizeof(double), static_cast<const double*>(q1),
                  static_cast<double*>(out));
    if (tp == T_F64 && tout == T_F32)
        return go(apply_refl_kernel<double, double, float>, sizeof(double), static_cast<const double*>(q1),
                  static_cast<float*>(out));
    return cudaErrorInvalidValue;
}

cudaError_t launch_gather_v(const void* q2, ElemType tq2, int64_t ldq2, int64_t n, int64_t ell, const int* perm,
                            void* v, ElemType tv, int64_t ldv, const int* cancel, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 31) / 32);
    count_launch();
    if (tq2 == T_F64 && tv == T_F64)
        {
            cudaError_t pe_ = launch_pdl(gather_v_kernel<double, double>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const double*>(q2), ldq2, n, (int)ell,
                                                                perm, static_cast<double*>(v), ldv, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    else if (tq2 == T_F64)
        {
            cudaError_t pe_ = launch_pdl(gather_v_kernel<double, float>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const double*>(q2), ldq2, n, (int)ell,
                                                               perm, static_cast<float*>(v), ldv, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    else if (tv == T_F64)
        {
            cudaError_t pe_ = launch_pdl(gather_v_kernel<float, double>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const float*>(q2), ldq2, n, (int)ell,
                                                               perm, static_cast<double*>(v), ldv, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    else
        {
            cudaError_t pe_ = launch_pdl(gather_v_kernel<float, float>, dim3(blocks), dim3(256), (size_t)(0), st, static_cast<const float*>(q2), ldq2, n, (int)ell,
                                                              perm, static_cast<float*>(v), ldv, cancel);
            if (pe_ != cudaSuccess) return pe_;
        }
    return cudaGetLastError();
}

cudaError_t launch_copy_small(const double* src, int64_t ell, void* dst, ElemType tdst,
                              const int* cancel, cudaStream_t st, bool transpose) {
    const int l = (int)ell, n = l * l;
    count_launch();
    cudaError_t e = tdst == T_F64
                        ? launch_pdl(copy_small_kernel<double>, dim3((n + 255) / 256), dim3(256), (size_t)0, st, src, l,
                                     static_cast<double*>(dst), transpose ? 1 : 0, cancel)
                        : launch_pdl(copy_small_kernel<float>, dim3((n + 255) / 256), dim3(256), (size_t)0, st, src, l,
                                     static_cast<float*>(dst), transpose ? 1 : 0, cancel);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace corutv

// ---------------------------------------------------------------------------
// Grouped forms of the small steps (one launch over the problems of a batch):
// the one-problem kernels' bodies, blockIdx.z selecting the problem.
// ---------------------------------------------------------------------------
namespace corutv {
namespace {

template <bool kDefic>
__device__ __forceinline__ void chol_g(const CholArgs& a) {
    cholesky_body<kDefic>(a.g, a.ell, a.rows, a.r, a.flags, a.skip_out, a.cancel, a.unit_roundoff, a.defic,
                          a.tau_rel);
}
__device__ __forceinline__ void rinv_g(const RinvArgs& a) { rinv_body(a.r, a.ell, a.ri, a.ldri, a.cancel); }
template <typename TQC>
__device__ __forceinline__ void trsm_g(const TrsmArgs& a) {
    trsm_gemm_body<TQC>(a.c, a.ldc, a.rows, a.ell, a.ri, a.ldri, a.q, a.ldq, static_cast<TQC*>(a.qc), a.ldqc,
                        a.cancel, a.defic);
}
__device__ __forceinline__ void qrcp_g(const QrcpArgs& a) { qrcp_body(a.d, a.ell, a.refl, a.rt, a.perm, a.cancel); }
__device__ __forceinline__ void refl_g(const ReflArgs& a) {
    apply_refl_body<float, float, float>(a.x, a.ldx, a.rows, a.ell, a.refl, a.out, a.ldo, 0, a.cancel);
}
// ell <= 64: one row of Q1 per thread, in registers
__device__ __forceinline__ void refl_rows_g(const ReflArgs& a) {
    apply_refl_rows_body<float, float>(a.x, a.ldx, a.rows, a.ell, a.refl, a.out, a.ldo, 0, a.cancel);
}
__device__ __forceinline__ void gather_g(const GatherArgs& a) {
    gather_v_body<float, float>(a.q2, a.ldq2, a.n, a.ell, a.perm, a.v, a.ldv, a.cancel);
}
// T = Rt in FP32 (row-major) and the pivots copied out
__device__ __forceinline__ void emit_g(const EmitArgs& a) {
    pdl_trigger();
    pdl_wait();
    if (a.cancel && *a.cancel) return;
    const int n = a.ell * a.ell;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n + a.ell; e += gridDim.x * blockDim.x) {
        if (e < n) a.t[e] = (float)a.rt[e];
        else if (a.perm_dst) a.perm_dst[e - n] = a.perm_src[e - n];
    }
}

template <class A>
GroupItem<A> item_of(const A& a, unsigned gx, unsigned gy = 1) {
    GroupItem<A> it;
    it.a = a;
    it.gx = gx;
    it.gy = gy;
    return it;
}

template <class A, void (*F)(const A&), int kT>
cudaError_t launch_group(const GroupItem<A>* it, int count, dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    if (count > 65535) return cudaErrorInvalidValue;
    auto kern = grouped_kernel<A, F, kT>;
    if (smem > 0) {  // (the 48 KB default covers static and dynamic shared memory together)
        const cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
        if (e != cudaSuccess) return e;
    }
    count_launch();
    grid.z = (unsigned)count;
    const cudaError_t e = launch_pdl(kern, grid, block, smem, st, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

size_t chol_smem(int ell) {
    return sizeof(double) * (size_t)ell * (ell + 1) + sizeof(unsigned short) * (size_t)ell * (ell + 1) / 2;
}
size_t rinv_smem(int ell) { return sizeof(float) * ((size_t)ell * rinv_ldt(ell) + ell); }
size_t trsmg_smem(int ell) { return sizeof(float) * (size_t)ell * (kTgRows + trsm_inv_ldri(ell)); }
size_t qrcp_smem(int ell) {
    return sizeof(double) * ((size_t)ell * (ell | 1) + 5 * (size_t)ell) + sizeof(int) * ell;
}
size_t refl_smem(int ell) {
    return sizeof(float) * ((size_t)ell * ell + 2 * (size_t)ell + (size_t)kTrsmRows * trsm_ld(ell));
}

}  // namespace

GroupItem<CholArgs> cholesky_item(const CholArgs& a) { return item_of(a, 1); }
GroupItem<RinvArgs> rinv_item(const RinvArgs& a) { return item_of(a, (unsigned)((a.ell + kRiWarps - 1) / kRiWarps)); }
GroupItem<TrsmArgs> trsm_item(const TrsmArgs& a) {
    return item_of(a, (unsigned)((a.rows + kTgRows - 1) / kTgRows));
}
GroupItem<QrcpArgs> qrcp_item(const QrcpArgs& a) { return item_of(a, 1); }
GroupItem<ReflArgs> refl_item(const ReflArgs& a) {
    return item_of(a, (unsigned)((a.rows + kTrsmRows - 1) / kTrsmRows));
}
GroupItem<ReflArgs> refl_rows_item(const ReflArgs& a) {
    return item_of(a, a.ell <= 64 ? (unsigned)((a.rows + kRrThreads - 1) / kRrThreads) : 0u);
}
GroupItem<GatherArgs> gather_item(const GatherArgs& a) { return item_of(a, (unsigned)((a.n + 31) / 32)); }
GroupItem<EmitArgs> emit_item(const EmitArgs& a) { return item_of(a, kAnyGrid); }

cudaError_t launch_cholesky_grouped(const GroupItem<CholArgs>* it, int count, int max_ell, bool defic,
                                    cudaStream_t st) {
    if (max_ell < 1 || max_ell > kCholMaxEll) return cudaErrorInvalidValue;
    const size_t smem = chol_smem(max_ell);
    return defic ? launch_group<CholArgs, chol_g<true>, kCholThreads>(it, count, dim3(1), dim3(kCholThreads), smem, st)
                 : launch_group<CholArgs, chol_g<false>, kCholThreads>(it, count, dim3(1), dim3(kCholThreads), smem,
                                                                       st);
}

cudaError_t launch_rinv_grouped(const GroupItem<RinvArgs>* it, int count, unsigned gx, int max_ell, cudaStream_t st) {
    if (max_ell < 1 || max_ell > 128) return cudaErrorInvalidValue;
    return launch_group<RinvArgs, rinv_g, kRiWarps * 32>(it, count, dim3(gx), dim3(kRiWarps * 32), rinv_smem(max_ell),
                                                         st);
}

cudaError_t launch_trsm_grouped(const GroupItem<TrsmArgs>* it, int count, unsigned gx, int max_ell, bool qc_bf16,
                                cudaStream_t st) {
    if (max_ell < 1 || max_ell > 128) return cudaErrorInvalidValue;
    const dim3 block(32 * ((max_ell + 7) / 8));
    const size_t smem = trsmg_smem(max_ell);
    return qc_bf16 ? launch_group<TrsmArgs, trsm_g<__nv_bfloat16>, 512>(it, count, dim3(gx), block, smem, st)
                   : launch_group<TrsmArgs, trsm_g<float>, 512>(it, count, dim3(gx), block, smem, st);
}

cudaError_t launch_qrcp_grouped(const GroupItem<QrcpArgs>* it, int count, int max_ell, cudaStream_t st) {
    if (max_ell < 1 || max_ell > 128) return cudaErrorInvalidValue;
    return launch_group<QrcpArgs, qrcp_g, kQrcpThreads>(it, count, dim3(1), dim3(kQrcpThreads), qrcp_smem(max_ell),
                                                        st);
}

cudaError_t launch_refl_grouped(const GroupItem<ReflArgs>* it, int count, unsigned gx, int max_ell, cudaStream_t st) {
    if (max_ell < 1 || max_ell > 128) return cudaErrorInvalidValue;
    return launch_group<ReflArgs, refl_g, kTrsmThreads>(it, count, dim3(gx), dim3(kTrsmThreads), refl_smem(max_ell),
                                                        st);
}

cudaError_t launch_refl_rows_grouped(const GroupItem<ReflArgs>* it, int count, unsigned gx, cudaStream_t st) {
    return launch_group<ReflArgs, refl_rows_g, kRrThreads>(it, count, dim3(gx), dim3(kRrThreads), 0, st);
}

cudaError_t launch_gather_grouped(const GroupItem<GatherArgs>* it, int count, unsigned gx, cudaStream_t st) {
    return launch_group<GatherArgs, gather_g, 256>(it, count, dim3(gx), dim3(256), 0, st);
}

cudaError_t launch_emit_grouped(const GroupItem<EmitArgs>* it, int count, unsigned gx, cudaStream_t st) {
    return launch_group<EmitArgs, emit_g, 256>(it, count, dim3(gx), dim3(256), 0, st);
}

}  // namespace corutv
