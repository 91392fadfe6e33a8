// FP32 Gram products G = X^T Y (the Gram matrices of CholeskyQR, Sec. 3.1,
// and D = Q1^T (A Q2), eq. 7) in a single launch, with the split sums reduced
// inside the kernel in a fixed order.
//
// X, Y: FP32 panels (column j at X + j * ldx, `len` rows), ell <= 320
// columns. G: ell x ell FP64, row-major. The output is cut into 64 x 64
// tiles (only those on and above the diagonal when Y is X: the others are
// the mirror images, bitwise); each tile's rows of X / Y are split into S
// contiguous ranges, one CTA per (range, tile). A CTA accumulates its 64 x 64
// partial in FP32 (a 4 x 4 block of adjacent outputs per thread, its operands
// read as two 16-byte shared-memory loads per row; operands staged in shared
// memory 32 rows at a time). The ranges run as thread-block clusters of 8 CTAs: each CTA leaves
// its partial in its shared memory, and rank r of the cluster adds slice r
// (512 outputs) of the 8 partials in rank order over distributed shared
// memory and stores that slice of the cluster sum. A counter per (tile,
// slice) then tells which CTA stored the last cluster sum of its slice; that
// CTA adds the clusters' slices in cluster order and writes G. Nobody waits
// on another CTA outside its cluster, the counters return to zero, and the
// sums never depend on arrival order. A panel whose tensor-core product left
// its split tiles as pieces is completed here: the pieces of each row are
// added as it is staged (and, on request, written back into the panel).
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.cuh"

namespace corutv {

namespace {

constexpr int kGT = 64;      // output tile
constexpr int kGChunk = 32;  // rows staged per step
constexpr int kGThreads = 256;
constexpr int kGCluster = 8; // CTAs per cluster = output slices
constexpr int kGLd = kGT + 4;  // 16-byte aligned staging rows
constexpr int kGSlice = kGT * kGT / kGCluster;

struct GramPlan {
    int ntile, tiles, nc;  // clusters per tile; ranges per tile = 8 nc
    int sym;               // Y is X: the tiles ti <= tj only
};

GramPlan gram_plan(int64_t len, int ell, int num_sms, bool sym) {
    GramPlan p;
    p.ntile = (ell + kGT - 1) / kGT;
    p.sym = sym ? 1 : 0;
    p.tiles = sym ? p.ntile * (p.ntile + 1) / 2 : p.ntile * p.ntile;
    int64_t nc = 2 * num_sms / (kGCluster * p.tiles);               // about two CTAs per SM
    nc = std::min<int64_t>(nc, (len + 64 * kGCluster - 1) / (64 * kGCluster));  // >= 64 rows per range
    p.nc = (int)std::max<int64_t>(1, nc);
    return p;
}

constexpr int kPer = kGChunk * kGT / kGThreads;  // elements per thread and operand per chunk (8)

// Output tile `tile` -> block coordinates; with sym the tiles on and above
// the diagonal, row after row.
__device__ __forceinline__ void tile_coords(int tile, int ntile, bool sym, int& ti, int& tj) {
    if (!sym) {
        ti = tile / ntile;
        tj = tile % ntile;
        return;
    }
    ti = 0;
    while (tile >= ntile - ti) {
        tile -= ntile - ti;
        ++ti;
    }
    tj = ti + tile;
}

// Row `row`, columns col0 + 8 k (k < kPer), of an FP32 panel whose split
// product tiles may still be pieces (zero for rows outside the chunk and
// columns >= ell). A row of a tile covered by np > 1 CTAs is the sum of its
// np FP32 partials in piece order, the order the product's own fix-up adds
// them in, so the value is the one the product would have stored; with
// writeback it is stored into the panel. The loads of four pieces of all
// eight columns are issued before any add (one L2 round trip per four
// pieces).
// The piece count of the row's 128-row tile, kept per thread: a thread's rows
// advance by one chunk at a time, so the tile changes every few chunks.
struct TileNp {
    long long t = -1;
    int np = 1;
};

__device__ __forceinline__ void load_row(const float* panel, int64_t ld, const TcPieces& pc, bool writeback,
                                         int64_t row, bool row_ok, int col0, int ell, TileNp& tn,
                                         float (&v)[kPer]) {
    int np = 1;
    const float* src = nullptr;
    if (pc.part && row_ok) {
        const long long t = row >> 7;
        if (t != tn.t) {
            const long long first = unit_owner(t * pc.kc, pc.units, pc.grid);
            tn.np = (int)(unit_owner((t + 1) * pc.kc - 1, pc.units, pc.grid) - first) + 1;
            tn.t = t;
        }
        np = tn.np;
        src = pc.part + (t * pc.maxp * pc.ellp) * 128 + (row & 127);
    }
    if (np == 1) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int col = col0 + 8 * k;
            v[k] = (row_ok && col < ell) ? panel[(int64_t)col * ld + row] : 0.f;
        }
        return;
    }
    const long long ps = (long long)pc.ellp * 128;  // piece stride
#pragma unroll
    for (int k = 0; k < kPer; ++k) v[k] = 0.f;
    if (np == 2) {  // the common case: two pieces, no clamped duplicate loads
        float w0[kPer], w1[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int col = col0 + 8 * k;
            w0[k] = col < ell ? __ldcg(src + (long long)col * 128) : 0.f;
            w1[k] = col < ell ? __ldcg(src + ps + (long long)col * 128) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] += w0[k];
            v[k] += w1[k];
        }
    }
    for (int q0 = 0; q0 < np && np != 2; q0 += 4) {
        float w[4][kPer];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const float* sp = src + (long long)min(q0 + g, np - 1) * ps;  // clamped: loads stay unconditional
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int col = col0 + 8 * k;
                w[g][k] = col < ell ? __ldcg(sp + (long long)col * 128) : 0.f;
            }
        }
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (q0 + g < np) {
#pragma unroll
                for (int k = 0; k < kPer; ++k) v[k] += w[g][k];
            }
    }
    if (writeback) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int col = col0 + 8 * k;
            if (col < ell) const_cast<float*>(panel)[(int64_t)col * ld + row] = v[k];
        }
    }
}

__device__ __forceinline__ void gram_f32_body(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len,
                                              int ell, double* out, float* cpart, int* cnt, const GramPlan& pl,
                                              const int* cancel, const TcPieces& pieces_x, const TcPieces& pieces_y,
                                              int writeback) {
    pdl_wait();
    namespace cg = cooperative_groups;
    if (cancel && *cancel) return;  // uniform over the grid: no cluster barrier is left waiting
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ __align__(16) float sbuf[2 * kGChunk * kGLd];  // staging, then the 64 x 64 partial
    __shared__ int last_s;
    float* Xs = sbuf;
    float* Ys = sbuf + kGChunk * kGLd;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int S = pl.nc * kGCluster;
    const int s = blockIdx.x, tile = blockIdx.y;
    const int rank = (int)cluster.block_rank(), cid = s / kGCluster;
    int ti, tj;
    tile_coords(tile, pl.ntile, pl.sym != 0, ti, tj);
    const int64_t r_beg = (int64_t)s * len / S, r_end = (int64_t)(s + 1) * len / S;
    const bool same = x == y && ti == tj;
    const TcPieces& pcx = pieces_x;
    const TcPieces& pcy = pieces_y;
    const bool wb = writeback != 0;
    const bool wb_y = wb && x != y;  // with X = Y the X loads complete the panel
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
    // staging: each thread moves 8 elements per operand per chunk (one row,
    // the columns c0, c0 + 8, ...); a warp covers 8 consecutive rows of 4
    // columns per load (four 32-byte sectors), and its shared-memory stores
    // hit 32 distinct banks. The next chunk's loads are all issued (into
    // registers) before the current chunk is multiplied, so their latency
    // overlaps the arithmetic.
    static_assert(kGThreads == 256 && kGChunk == 32 && kGT == 64, "staging map");
    const int lane = tid & 31, warp = tid >> 5;
    const int sr = 8 * (warp & 3) + (lane & 7), sc = 4 * (warp >> 2) + (lane >> 3);
    float px[kPer], py[kPer];
    TileNp tnx, tny;
    auto load_chunk = [&](int64_t r0) {
        const int nr = (int)(r_end - r0 < kGChunk ? r_end - r0 : kGChunk);
        load_row(x, ldx, pcx, wb, r0 + sr, sr < nr, ti * kGT + sc, ell, tnx, px);
        if (!same) load_row(y, ldy, pcy, wb_y, r0 + sr, sr < nr, tj * kGT + sc, ell, tny, py);
    };
    if (r_beg < r_end) load_chunk(r_beg);
    for (int64_t r0 = r_beg; r0 < r_end; r0 += kGChunk) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            Xs[sr * kGLd + sc + 8 * k] = px[k];
            if (!same) Ys[sr * kGLd + sc + 8 * k] = py[k];
        }
        __syncthreads();
        if (r0 + kGChunk < r_end) load_chunk(r0 + kGChunk);
        const float* Yb = same ? Xs : Ys;
#pragma unroll 4
        for (int r = 0; r < kGChunk; ++r) {
            const float4 a4 = *reinterpret_cast<const float4*>(Xs + r * kGLd + 4 * ty);
            const float4 b4 = *reinterpret_cast<const float4*>(Yb + r * kGLd + 4 * tx);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(a[i], b[k], acc[i][k]);
        }
        __syncthreads();
    }
    pdl_trigger();  // the successor may launch during the reductions
    // the partial of this range stays in shared memory (row-major 64 x 64)
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(sbuf + (4 * ty + i) * kGT + 4 * tx) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    cluster.sync();
    // slice `rank` of the cluster sum: the 8 partials in rank order
    float* cp = cpart + ((size_t)tile * pl.nc + cid) * (kGT * kGT) + (size_t)rank * kGSlice;
    for (int e = tid; e < kGSlice; e += kGThreads) {
        float v[kGCluster];
#pragma unroll
        for (int q = 0; q < kGCluster; ++q) v[q] = cluster.map_shared_rank(sbuf, q)[rank * kGSlice + e];
        float sum = 0.f;
#pragma unroll
        for (int q = 0; q < kGCluster; ++q) sum += v[q];
        cp[e] = sum;
    }
    cluster.sync();  // no CTA leaves while others still read its shared memory
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        int* c = cnt + tile * kGCluster + rank;
        const int done = atomicAdd(c, 1) + 1;
        last_s = done == pl.nc;
        if (done == pl.nc) *c = 0;
    }
    __syncthreads();
    if (!last_s) return;
    // slice `rank` of G: the clusters' sums in cluster order
    __threadfence();
    const float* c0 = cpart + (size_t)tile * pl.nc * (kGT * kGT) + (size_t)rank * kGSlice;
    for (int e = tid; e < kGSlice; e += kGThreads) {
        float sum = 0.f;
        int q = 0;
        for (; q + 7 < pl.nc; q += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(c0 + (size_t)(q + u) * (kGT * kGT) + e);
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += v[u];
        }
        for (; q < pl.nc; ++q) sum += __ldcg(c0 + (size_t)q * (kGT * kGT) + e);
        const int eg = rank * kGSlice + e;
        const int a = ti * kGT + eg / kGT, b = tj * kGT + eg % kGT;
        if (a < ell && b < ell) {
            const double g = f2d_exact(sum);
            out[(int64_t)a * ell + b] = g;
            if (pl.sym && ti != tj) out[(int64_t)b * ell + a] = g;  // the mirror tile, bitwise its own sum
        }
    }
}

__global__ void __launch_bounds__(kGThreads)
gram_f32_kernel(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len, int ell, double* out,
                float* cpart, int* cnt, GramPlan pl, const int* cancel, TcPieces pieces_x, TcPieces pieces_y,
                int writeback) {
    gram_f32_body(x, ldx, y, ldy, len, ell, out, cpart, cnt, pl, cancel, pieces_x, pieces_y, writeback);
}

// One problem of a grouped Gram launch (complete panels: no pieces); blocks
// beyond the problem's own grid return as whole clusters (gx is a multiple
// of 8). Two CTAs per SM as in the one-problem kernel (three measured the
// same and spill).
__global__ void __launch_bounds__(kGThreads) gram_grouped_kernel(const GroupItem<GramArgs>* items) {
    const GroupItem<GramArgs>& it = items[blockIdx.z];
    if (blockIdx.x >= it.gx || blockIdx.y >= it.gy) return;  // whole clusters (gx a multiple of 8)
    const GramArgs& a = it.a;
    GramPlan pl;
    pl.ntile = a.ntile;
    pl.tiles = a.tiles;
    pl.nc = a.nc;
    pl.sym = a.sym;
    const TcPieces none;
    gram_f32_body(a.x, a.ldx, a.y, a.ldy, a.len, a.ell, a.out, a.work, a.cnt, pl, a.cancel, none, none, 0);
}

}  // namespace

// Workspace for either plan (X^T Y, or X^T X on the upper tiles).
int64_t gram_f32_work_floats(int64_t len, int ell, int num_sms) {
    const GramPlan p = gram_plan(len, ell, num_sms, false), q = gram_plan(len, ell, num_sms, true);
    return (int64_t)std::max(p.tiles * p.nc, q.tiles * q.nc) * (kGT * kGT);
}

int64_t gram_f32_counters(int64_t len, int ell, int num_sms) {
    const GramPlan p = gram_plan(len, ell, num_sms, false);
    return (int64_t)p.tiles * kGCluster;
}

cudaError_t launch_gram_f32(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len, int ell,
                            double* out, float* work, int* cnt, int num_sms, const int* cancel, cudaStream_t st,
                            const TcPieces& px, const TcPieces& py, bool writeback) {
    if (ell < 1 || ell > kMaxEllSimt || len < 1 || !work || !cnt) return cudaErrorInvalidValue;
    const GramPlan p = gram_plan(len, ell, num_sms, x == y && ldx == ldy);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.nc * kGCluster), (unsigned)p.tiles, 1);
    cfg.blockDim = dim3(kGThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kGCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    count_launch();
    prefer_max_shared(reinterpret_cast<const void*>(gram_f32_kernel));
    return cudaLaunchKernelEx(&cfg, gram_f32_kernel, x, ldx, y, ldy, len, ell, out, work, cnt, p, cancel, px, py,
                              writeback ? 1 : 0);
}


GroupItem<GramArgs> gram_group_item(const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t len, int ell,
                                    double* out, float* work, int* cnt, const int* cancel, int num_sms) {
    const bool sym = x == y && ldx == ldy;
    const GramPlan full = gram_plan(len, ell, num_sms, sym);
    GramPlan p = full;
    const int64_t nc = (len + 256 * kGCluster - 1) / (256 * kGCluster);  // about 256 rows per CTA
    p.nc = (int)std::max<int64_t>(1, std::min<int64_t>(nc, full.nc));    // within the one-problem workspace
    GroupItem<GramArgs> it;
    it.a = GramArgs{x, ldx, y, ldy, len, ell, out, work, cnt, p.ntile, p.tiles, p.nc, p.sym, cancel};
    it.gx = (unsigned)(p.nc * kGCluster);
    it.gy = (unsigned)p.tiles;
    return it;
}

cudaError_t launch_gram_grouped(const GroupItem<GramArgs>* it, int count, unsigned gx, unsigned gy, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    if (gx % kGCluster != 0) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(gx, gy, (unsigned)count);
    cfg.blockDim = dim3(kGThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kGCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    count_launch();
    auto kern = gram_grouped_kernel;
    prefer_max_shared(reinterpret_cast<const void*>(kern));
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace corutv
