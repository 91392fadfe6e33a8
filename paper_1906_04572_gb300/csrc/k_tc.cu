// Tensor-core sketch products of libcorutv (eqs. 4 and 5): C = A X and
// C = A^T Y with tcgen05.mma (kind::f16 with bf16 operands, kind::tf32 with
// fp32 operands), FP32 accumulators in tensor memory, operands staged by TMA.
//
// Shape: A is m x n row-major; X / Y are tall-skinny panels with ell_p <= 128
// columns (multiple of 16). Each output tile is 128 rows of C by all ell_p
// columns. The MMA M dimension runs along the long side of C (rows of A for
// A X, columns of A for A^T Y), N = ell_p, K along the contracted side.
//   A X  : A is K-major (its rows are contiguous along K = n).
//   A^T Y: A is MN-major (its rows are contiguous along M = n).
// The panels are always K-major (column j of the panel is contiguous).
//
// Schedule: a persistent grid of G CTAs (one per SM) splits the
// (tile, K-chunk) iteration space into G equal contiguous ranges (stream-K),
// so no wave is ever partly empty. A CTA's range crosses at most a few tile
// boundaries. A tile covered by one CTA is written straight to the output
// panel. Otherwise each CTA's segment of it is an FP32 partial (128 x ell_p)
// in `part`; each finished piece bumps the tile's counter, and the CTA that
// finishes last adds the tile's pieces in piece order (in FP32) and writes
// the output, so the sum never depends on which CTA happened to finish last.
// When the caller asks for the pieces (TcPieces), the counting and adding
// are left out: the next kernel that reads the panel adds the same pieces in
// the same order.
//
// Warp roles (192 threads): warps 0-3 read the accumulator out of tensor
// memory (warp w owns TMEM lanes 32w..32w+31 = rows of the tile), warp 4 is
// the TMA producer, warp 5 allocates tensor memory and issues the MMAs.
// Two accumulators alternate so the epilogue of one segment overlaps the
// MMAs of the next.
//
// Every wait on an mbarrier is bounded (about kWaitNs, counted in SM clock
// cycles); on timeout
// the CTA sets FLAG_TIMEOUT, stops issuing work, waits (again bounded) for
// its own copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tc.cuh"

namespace corutv {

namespace {

constexpr int kThreads = 192;
constexpr int kTileM = 128;
constexpr int kMaxStages = 8;
constexpr int kKSteps = 4;  // MMA K steps per 128-byte K chunk: 64 bf16 / 16, or 32 tf32 / 8
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

struct TcParams {
    long long units;      // mtiles * kchunks
    long long kchunks;    // K chunks per tile (kseg segments of kc_seg chunks)
    int kc_seg;           // K chunks per segment
    int seg_stride;       // A column offset between K segments (elements)
    int grid;             // G
    int maxp;             // partial pieces per tile
    int ellp;             // output columns per tile
    int nparts;           // B column groups added in the epilogue (1, or 3 for split products)
    int trans;
    int tf32;
    int stages;
    int a_boxes;          // TMA boxes per A tile (MN-major needs several)
    int a_box_cols;       // columns (MN elements) per A box
    const uint8_t* a_tiles;  // non-null: A is a tiled bf16 copy (see launch_cast_tiled), read by bulk copies
    long long a_ntp;      // tiles per 128-row block of that copy (even)
    long long a_seg_bytes;   // bytes between its K segments (split parts)
    int b_boxes;          // TMA boxes per B tile
    int b_box_rows;       // rows per B box
    uint32_t a_bytes;     // A tile bytes per stage
    uint32_t stage_bytes; // A + B bytes per stage
    uint32_t idesc0, idesc1;  // MMA N chunks: n0 columns, then n1 (0 = none)
    int n0, n1;
    int nacc;             // accumulators in tensor memory (2 = epilogue overlaps the next segment)
    uint32_t acc_cols;    // tensor-memory columns per accumulator
    uint32_t tmem_cols;   // columns allocated
    int kchunk_elems;     // K elements per chunk: kgroup 128-byte boxes (64 bf16 / 32 fp32 each)
    int kgroup;           // 128-byte K boxes per stage (longer runs along each row of A)
    float* part;
    int* tile_cnt;        // per output tile: pieces finished (zero between launches)
    void* out;            // output panel (FP64 or FP32)
    int out_f64;
    int ell;              // valid output columns
    long long ldc;
    long long mtot;       // valid output rows
    int* flags;
    const int* cancel;
    int defer;            // split tiles: leave the pieces for the consumer (no count, no reduction)
};

// One problem of a grouped product launch: the B panel's tensor map and the
// problem's parameters (the CUtensorMap first: 64-byte aligned in the array).
struct alignas(128) TcGroupItem {
    CUtensorMap map_b;
    TcParams p;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false if the phase did not complete within about `limit_ns`
// (measured with the SM cycle counter at the 2.07 GHz maximum clock, checked
// every 256 polls so the poll loop stays tight) or if another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long limit_cycles = (long long)(limit_ns * 2.07);
    const long long t0 = clock64();
    for (uint32_t polls = 1;; ++polls) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((polls & 255u) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (clock64() - t0 > limit_cycles) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing on `bar` with `bytes` of transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Shared-memory matrix descriptor of tcgen05 (start address, leading and
// stride byte offsets, fixed version bits 46-48 = 0b001, swizzle mode in
// bits 61-63: 2 = 128-byte swizzle, 1 = 128-byte swizzle with 32-byte atoms).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(swz & 7u) << 61;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Owner CTA of stream-K unit u when `units` units are split over `grid` CTAs
// as [floor(c U / G), floor((c+1) U / G)).

// Output row rg of a tile split over np pieces: out[j * ldc + rg] = the
// pieces' FP32 partials added in piece order in FP32, for j < ell, then
// converted once to the output type. The partials are FP32-accumulated
// products, so adding a few of them in FP32 in a fixed order costs a few ulp,
// below the error they already carry; an FP64 sum would add nothing but
// FP64-pipe time (about 65 cycles per warp instruction on this GPU). All
// loads of a 16-column chunk (up to four pieces at a time) are issued before
// any add so their L2 latencies overlap.
template <typename TO>
__device__ __forceinline__ void reduce_pieces(const float* src, int np, int ellp, int ell, TO* out, long long ldc,
                                              long long rg) {
    for (int j0 = 0; j0 < ell; j0 += 16) {  // ellp is a multiple of 16, so j0 + 15 < ellp
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        for (int pc0 = 0; pc0 < np; pc0 += 4) {
            // unconditional loads (piece index clamped to a valid one) so that all
            // 64 are issued back to back; pieces beyond np are not added
            float v[4][16];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const float* sp = src + ((long long)min(pc0 + g, np - 1) * ellp + j0) * kTileM;
#pragma unroll
                for (int i = 0; i < 16; ++i) v[g][i] = __ldcg(sp + i * kTileM);
            }
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (pc0 + g < np) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[i] += v[g][i];
                }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (j0 + i < ell) out[(long long)(j0 + i) * ldc + rg] = (TO)acc[i];
    }
}

// The same sum from pieces staged in shared memory (sp = row's element of
// piece 0): per 16-column block, the loads of four pieces are issued back to
// back (piece index clamped, extra pieces not added), then added in order.
template <typename TO>
__device__ __forceinline__ void sum_staged(const float* sp, int np, int ellp, int ell, TO* out, long long ldc,
                                           long long rg) {
#pragma unroll 1
    for (int j0 = 0; j0 < ell; j0 += 16) {
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int pc0 = 0; pc0 < np; pc0 += 4) {
            float v[4][16];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const float* q = sp + ((size_t)min(pc0 + g, np - 1) * ellp + j0) * kTileM;
#pragma unroll
                for (int i = 0; i < 16; ++i) v[g][i] = q[i * kTileM];
            }
#pragma unroll
            for (int g = 0; g < 4; ++g)
                if (pc0 + g < np) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[i] += v[g][i];
                }
        }
        if (j0 + 16 <= ell) {
#pragma unroll
            for (int i = 0; i < 16; ++i) out[(long long)(j0 + i) * ldc + rg] = (TO)acc[i];
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (j0 + i < ell) out[(long long)(j0 + i) * ldc + rg] = (TO)acc[i];
        }
    }
}

template <bool kTf32>
__device__ __forceinline__ void sketch_tc_body(const CUtensorMap* map_a, const CUtensorMap* map_b, const TcParams& p,
                                               bool prefetch_maps) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages];
    __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ __align__(8) uint64_t ep_bar[2];  // pieces stored (4 warps) / counter result ready
    __shared__ __align__(8) uint64_t fix_bar;    // pieces staged into shared memory (last segment)
    __shared__ volatile int last_s;
    __shared__ volatile int fix_issued;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_s;
    __shared__ volatile long long consumed_s;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    const int u0 = (int)((long long)c * p.units / p.grid);
    const int u1 = (int)((long long)(c + 1) * p.units / p.grid);
    const int S = p.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf_bar[a], 1);
            mbar_init(&acce_bar[a], 4);
        }
        mbar_init(&drain_bar, 1);
        mbar_init(&ep_bar[0], 4);
        mbar_init(&ep_bar[1], 1);
        mbar_init(&fix_bar, 1);
        last_s = 0;
        fix_issued = 0;
        abort_s = 0;
        consumed_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4 && lane == 0 && prefetch_maps) {
        if (!p.a_tiles) prefetch_tmap(map_a);
        prefetch_tmap(map_b);
    }
    // setup above overlaps the previous kernel's tail; operands and flags are read below
    pdl_wait();
    if (p.cancel && *p.cancel) return;  // uniform over the grid, before any tensor memory is held
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_holder;
    const int KC = (int)p.kchunks;

    if (warp == 4) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int li = 0, s = 0, r = 0;       // unit index, stage, round (li = r S + s)
            int t = u0 / KC, kc = u0 % KC;  // tile and K chunk of unit u
            int seg = kc / p.kc_seg, kk = kc - seg * p.kc_seg;  // K segment and chunk within it
            const uint32_t box_bytes = p.a_bytes / p.a_boxes;
            const uint32_t b_bytes = (uint32_t)(p.b_boxes * p.b_box_rows) * 128u;
            const int ke = kTf32 ? 32 : 64;
            for (int u = u0; u < u1; ++u, ++li) {
                if (r > 0 && !mbar_wait(&empty_bar[s], (uint32_t)((r - 1) & 1), &abort_s)) {
                    abort_s = 1;
                    break;
                }
                uint8_t* sa = smem + (size_t)s * p.stage_bytes;
                uint8_t* sb = sa + (size_t)p.kgroup * p.a_bytes;
                mbar_expect_tx(&full_bar[s], p.stage_bytes);
                // kgroup boxes along K: A at sa + g a_bytes, B at sb + g b_bytes
                if (p.a_tiles) {
                    // tiled copy: tile (I, J) = rows 128 I.., columns 64 J.. at (I ntp + J) 16 KB,
                    // each the image of a 128-byte-swizzled box; A X takes kgroup tiles of
                    // one row block (adjacent), A^T Y the two tiles of a 128-column block
                    // (adjacent) over kgroup 64-row halves
                    if (!p.trans) {
                        const uint8_t* src = p.a_tiles + seg * p.a_seg_bytes +
                                             (((long long)t * p.a_ntp + (long long)kk * p.kgroup) << 14);
                        bulk_load(sa, src, (uint32_t)p.kgroup << 14, &full_bar[s]);
                    } else if (p.kgroup == 2) {
                        bulk_load(sa, p.a_tiles + seg * p.a_seg_bytes + (((long long)kk * p.a_ntp + 2LL * t) << 14),
                                  32768u, &full_bar[s]);
                    } else {
                        const uint8_t* src = p.a_tiles + seg * p.a_seg_bytes +
                                             (((long long)(kk >> 1) * p.a_ntp + 2LL * t) << 14) + (size_t)(kk & 1) * 8192;
                        bulk_load(sa, src, 8192u, &full_bar[s]);
                        bulk_load(sa + 8192, src + 16384, 8192u, &full_bar[s]);
                    }
                }
                for (int g = 0; g < p.kgroup; ++g) {
                    const int kx = kk * p.kchunk_elems + g * ke;
                    uint8_t* sag = sa + (size_t)g * p.a_bytes;
                    if (p.a_tiles) {
                        // A already requested above
                    } else if (!p.trans) {
                        tma_load_2d(sag, map_a, &full_bar[s], seg * p.seg_stride + kx, (int)(t * kTileM));
                    } else {
                        for (int bx = 0; bx < p.a_boxes; ++bx)
                            tma_load_2d(sag + bx * box_bytes, map_a, &full_bar[s],
                                        (int)(t * kTileM + bx * p.a_box_cols), kx);
                    }
                    uint8_t* sbg = sb + (size_t)g * b_bytes;
                    for (int bx = 0; bx < p.b_boxes; ++bx)
                        tma_load_2d(sbg + bx * p.b_box_rows * 128, map_b, &full_bar[s], kx, bx * p.b_box_rows);
                }
                if (++s == S) { s = 0; ++r; }
                if (++kk == p.kc_seg) { kk = 0; ++seg; }
                if (++kc == KC) { kc = 0; ++t; seg = 0; kk = 0; }
            }
            pdl_trigger();  // all loads issued: the successor may launch during the last MMAs and the fix-up
            if (abort_s) {
                // drain: wait (bounded) for every copy that was issued but not consumed
                const int issued = li;
                for (int j = (int)consumed_s; j < issued; ++j)
                    mbar_wait(&full_bar[j % S], (uint32_t)((j / S) & 1), nullptr, 100000000ull);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            // A single thread issues every MMA, so the issue loop must stay
            // short: the shared-memory descriptors are built once, and per
            // stage and per K step only their start-address field (bits
            // 0-13, in 16-byte units; shared addresses stay below 256 KB so
            // the field never carries into the next one) is advanced.
            const uint32_t sbase = smem_u32(smem);
            uint64_t a_desc0;
            uint32_t a_kstep;
            if (!p.trans) {
                // K-major A: 128 rows x 128 B, 8-row groups 1024 B apart; a K step is 32 B along the row
                a_desc0 = smem_desc(sbase, 16, 1024, 2);
                a_kstep = 32u >> 4;
            } else if (!kTf32) {
                // MN-major A: 64-element MN atoms (a_bytes / a_boxes apart; in a tiled copy the
                // two atoms are whole 64 kgroup-row tiles), 8-row K groups 1024 B apart; a K step
                // of 16 consumes two K groups
                a_desc0 = smem_desc(sbase, p.a_tiles ? (uint32_t)p.kgroup * 8192u : p.a_bytes / p.a_boxes, 1024, 2);
                a_kstep = 2048u >> 4;
            } else {
                // MN-major tf32: 32-element MN atoms, a K step of 8 is one K group
                a_desc0 = smem_desc(sbase, p.a_bytes / p.a_boxes, 1024, 1);
                a_kstep = 1024u >> 4;
            }
            const uint64_t b_desc0 = smem_desc(sbase + (uint32_t)p.kgroup * p.a_bytes, 16, 1024, 2);
            // next K box of A: the next kgroup box (A X), or 64 rows further down both MN atoms
            // of a tiled A^T Y operand
            const uint32_t a_g16 = (p.a_tiles && p.trans) ? (8192u >> 4) : (p.a_bytes >> 4);
            const uint32_t b_g16 = ((uint32_t)(p.b_boxes * p.b_box_rows) * 128u) >> 4;  // next K box of B
            const int kg = p.kgroup;
            const uint32_t b_kstep = 32u >> 4;  // 16 bf16 or 8 tf32 elements of K
            const uint32_t stage16 = p.stage_bytes >> 4;
            const uint32_t n1_off = ((uint32_t)p.n0 * 128u) >> 4;
            const uint32_t idesc0 = p.idesc0, idesc1 = p.idesc1;
            const bool two_n = p.n1 != 0;
            int li = 0, seg = 0, s = 0, r = 0;
            for (int u = u0; u < u1 && !abort_s; ++seg) {
                const int t = u / KC;
                const int seg_end = (u1 < (t + 1) * KC) ? u1 : (t + 1) * KC;
                const int a = seg % p.nacc, use = seg / p.nacc;
                if (use >= 1 && !mbar_wait(&acce_bar[a], (uint32_t)((use - 1) & 1), &abort_s)) {
                    abort_s = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t tacc = tmem_base + (uint32_t)a * p.acc_cols;
                bool first = true;
                for (; u < seg_end; ++u, ++li) {
                    if (!mbar_wait(&full_bar[s], (uint32_t)(r & 1), &abort_s)) {
                        abort_s = 1;
                        break;
                    }
                    consumed_s = li + 1;
                    tc_fence_after();
                    for (int g = 0; g < kg; ++g) {
                        const uint64_t ad = a_desc0 + (uint64_t)((uint32_t)s * stage16 + (uint32_t)g * a_g16);
                        const uint64_t bd = b_desc0 + (uint64_t)((uint32_t)s * stage16 + (uint32_t)g * b_g16);
#pragma unroll
                        for (int kk = 0; kk < kKSteps; ++kk) {
                            const uint32_t acc = (first && g == 0 && kk == 0) ? 0u : 1u;
                            const uint64_t adk = ad + (uint64_t)(kk * a_kstep), bdk = bd + (uint64_t)(kk * b_kstep);
                            if (kTf32) mma_tf32(tacc, adk, bdk, idesc0, acc);
                            else mma_f16(tacc, adk, bdk, idesc0, acc);
                            if (two_n) {  // second N chunk: B rows n0.., accumulator columns n0..
                                if (kTf32) mma_tf32(tacc + (uint32_t)p.n0, adk, bdk + n1_off, idesc1, acc);
                                else mma_f16(tacc + (uint32_t)p.n0, adk, bdk + n1_off, idesc1, acc);
                            }
                        }
                    }
                    first = false;
                    mma_commit(&empty_bar[s]);
                    if (++s == S) { s = 0; ++r; }
                }
                if (abort_s) break;
                mma_commit(&accf_bar[a]);
            }
            if (abort_s) {
                mma_commit(&drain_bar);
                mbar_wait(&drain_bar, 0, nullptr, 100000000ull);
            }
        }
    } else {
        // ---------------- epilogue: warps 0-3 ----------------
        const int row = warp * 32 + lane;
        int seg = 0, nsync = 0;
        for (int u = u0; u < u1; ++seg) {
            const int t = u / KC;
            const int seg_end = (u1 < (t + 1) * KC) ? u1 : (t + 1) * KC;
            const int a = seg % p.nacc;
            if (!mbar_wait(&accf_bar[a], (uint32_t)((seg / p.nacc) & 1), &abort_s)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            const long long first = unit_owner((long long)t * KC, p.units, p.grid);
            const int np = (int)(unit_owner((long long)(t + 1) * KC - 1, p.units, p.grid) - first) + 1;
            const long long piece = c - first;
            const long long rg = (long long)t * kTileM + row;  // output row
            const bool in_range = rg < p.mtot;
            float* dst = p.part + (((long long)t * p.maxp + piece) * p.ellp) * (long long)kTileM + row;
            const uint32_t tacc = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)a * p.acc_cols;
            for (int c0 = 0; c0 < p.ellp; c0 += 16) {
                float v[16];
                tmem_ld16(tacc + (uint32_t)c0, v);
                for (int x = 1; x < p.nparts; ++x) {  // column groups of a split product, added in order
                    float w[16];
                    tmem_ld16(tacc + (uint32_t)(x * p.ellp + c0), w);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w[i];
                }
                if (np > 1) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) dst[(long long)(c0 + i) * kTileM] = v[i];
                } else if (in_range) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (c0 + i >= p.ell) break;
                        const long long o = (long long)(c0 + i) * p.ldc + rg;
                        if (p.out_f64) static_cast<double*>(p.out)[o] = (double)v[i];
                        else static_cast<float*>(p.out)[o] = v[i];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[a]);
            if (np > 1 && !p.defer) {
                // publish this piece, then count it; the CTA completing the count reduces the tile
                __threadfence();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ep_bar[0]);
                if (threadIdx.x == 0) {
                    if (mbar_wait(&ep_bar[0], (uint32_t)(nsync & 1), &abort_s)) {
                        const int done = atomicAdd(&p.tile_cnt[t], 1) + 1;
                        last_s = done == np;
                        if (done == np) p.tile_cnt[t] = 0;  // no other piece of this tile remains in this launch
                    } else {
                        abort_s = 1;
                    }
                    mbar_arrive(&ep_bar[1]);
                }
                if (!mbar_wait(&ep_bar[1], (uint32_t)(nsync & 1), &abort_s)) abort_s = 1;
                ++nsync;
                if (abort_s) break;
                if (last_s) {
                    const float* src = p.part + ((long long)t * p.maxp * p.ellp) * (long long)kTileM;
                    const uint32_t piece_bytes = (uint32_t)p.ellp * kTileM * 4u;
                    if (seg_end == u1 && (uint64_t)np * piece_bytes <= (uint64_t)p.stages * p.stage_bytes) {
                        // Last segment: every MMA has completed and every copy was consumed,
                        // so the operand ring is idle. Each piece is one contiguous block:
                        // stage all of them with one bulk copy each (one round trip) and add
                        // them from shared memory.
                        if (threadIdx.x == 0) {
                            __threadfence();
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                            mbar_expect_tx(&fix_bar, (uint32_t)np * piece_bytes);
                            for (int pc = 0; pc < np; ++pc)
                                bulk_load(smem + (size_t)pc * piece_bytes, src + (long long)pc * p.ellp * kTileM,
                                          piece_bytes, &fix_bar);
                            fix_issued = 1;
                        }
                        if (!mbar_wait(&fix_bar, 0, &abort_s)) {
                            abort_s = 1;
                            break;
                        }
                        if (in_range) {
                            const float* sp = reinterpret_cast<const float*>(smem) + row;
                            if (p.out_f64) sum_staged<double>(sp, np, p.ellp, p.ell, static_cast<double*>(p.out), p.ldc, rg);
                            else sum_staged<float>(sp, np, p.ellp, p.ell, static_cast<float*>(p.out), p.ldc, rg);
                        }
                    } else if (in_range) {
                        __threadfence();
                        if (p.out_f64)
                            reduce_pieces<double>(src + row, np, p.ellp, p.ell, static_cast<double*>(p.out), p.ldc, rg);
                        else
                            reduce_pieces<float>(src + row, np, p.ellp, p.ell, static_cast<float*>(p.out), p.ldc, rg);
                    }
                }
            }
            u = seg_end;
        }
    }
    if (abort_s && threadIdx.x == 0) {
        atomicExch(&p.flags[FLAG_TIMEOUT], 1);
        if (fix_issued) mbar_wait(&fix_bar, 0, nullptr, 100000000ull);  // staged copies in flight
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(p.tmem_cols));
    }
}

template <bool kTf32>
__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                 const __grid_constant__ TcParams p) {
    sketch_tc_body<kTf32>(&map_a, &map_b, p, true);
}

// The products of the problems of a batch in one launch: problem blockIdx.y
// runs the stream-K schedule of its own TcParams (its grid, operands, output,
// partials and counters) on the CTAs blockIdx.x < its grid; the B panel's
// tensor map is read from the item in global memory (written by a copy
// before the launch: the acquire fence orders the tensor-map proxy's read of
// it after that write).
__global__ void __launch_bounds__(kThreads, 1) sketch_tc_grouped_kernel(const TcGroupItem* items) {
    const TcGroupItem* gi = items + blockIdx.y;
    __shared__ TcParams ps;
    if ((int)blockIdx.x >= gi->p.grid) return;
    if (threadIdx.x == 0) ps = gi->p;
    if (threadIdx.x == 128)  // the producer thread
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(&gi->map_b))
                     : "memory");
    __syncthreads();
    sketch_tc_body<false>(nullptr, &gi->map_b, ps, false);
}

// The bounded-wait path of the tensor-core kernels, exercised on purpose:
// one warp allocates 32 columns of tensor memory, waits on an mbarrier that
// nothing ever arrives on, gives up after about limit_ns, raises
// FLAG_TIMEOUT, frees the tensor memory and returns. The context stays usable
// and the next kernel can allocate tensor memory again.
__global__ void __launch_bounds__(32) wait_probe_kernel(int* flags, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_holder;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(32u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    tc_fence_before();
    __syncwarp();
    tc_fence_after();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, nullptr, limit_ns)) atomicExch(&flags[FLAG_TIMEOUT], 1);
    tc_fence_before();
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_holder), "r"(32u));
}

__device__ __forceinline__ __nv_bfloat16 to_bf16(float v) { return __float2bfloat16_rn(v); }
// double -> bf16 without double rounding (round to odd through float).
__device__ __forceinline__ __nv_bfloat16 to_bf16(double v) {
    float f = __double2float_rz(v);
    if ((double)f != v && isfinite(v)) f = __uint_as_float(__float_as_uint(f) | 1u);
    return __float2bfloat16_rn(f);
}

__global__ void copy_f32_padded_kernel(const float* a, long long m, long long n, long long lda, float* out,
                                       long long ldb) {
    pdl_trigger();
    pdl_wait();
    const long long total = m * ldb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / ldb, j = e % ldb;
        out[e] = (j < n) ? a[i * lda + j] : 0.f;
    }
}

// Exact three-way bf16 split of an FP32 value: a = h + m + l with h = bf16(a),
// m = bf16(a - h), l = bf16(a - h - m); each difference is exact in FP32 and
// the last one has at most 8 significant bits, so l is exact too (for
// operands and parts in the normal range).
__device__ __forceinline__ void split3(float a, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(a);
    const float r1 = a - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

// One read of FP32 A (m x n, row stride lda) in 64 x 64 tiles, writing any
// of: at = A^T (n rows, row stride ldt >= round_up(m, 64); columns
// [m, round_up(m, 64)) zero, any further ones untouched), the exact splits
// A_h, A_m, A_l as the three parts of a tiled bf16 copy (a3, the layout of
// launch_cast_tiled, padding zero) and a row-major copy with row stride
// ldc <= round_up(n, 64) (zero for n <= j < ldc). The transposed
// copy makes A^T Y a product with K-major operands (TF32 has no MN-major form
// here). 256 threads, a tile staged in shared memory for the transpose.
constexpr int kPrepT = 64;
__global__ void __launch_bounds__(256)
prep_f32_kernel(const float* a, long long m, long long n, long long lda, float* at, long long ldt,
                uint8_t* a3, long long ntp, long long part_bytes, float* acopy, long long ldc, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    __shared__ float tile[kPrepT][kPrepT + 1];
    const long long i0 = (long long)blockIdx.y * kPrepT, j0 = (long long)blockIdx.x * kPrepT;
    const int tid = threadIdx.x;
    const bool vec = (reinterpret_cast<uintptr_t>(a) & 15) == 0 && (lda & 3) == 0;
    float v[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int idx = tid + 256 * k;
        const int r = idx >> 4, c4 = (idx & 15) * 4;
        const long long i = i0 + r, j = j0 + c4;
        const float* src = a + i * lda + j;
        if (i < m && vec && j + 3 < n) {
            const float4 f = *reinterpret_cast<const float4*>(src);
            v[k][0] = f.x; v[k][1] = f.y; v[k][2] = f.z; v[k][3] = f.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[k][q] = (i < m && j + q < n) ? src[q] : 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int idx = tid + 256 * k;
        const int r = idx >> 4, c4 = (idx & 15) * 4;
        const long long i = i0 + r, j = j0 + c4;
#pragma unroll
        for (int q = 0; q < 4; ++q) tile[r][c4 + q] = v[k][q];
        if (a3 && (j >> 6) < ntp) {  // the grid covers every tile of the copy; padding is written as zero
            __nv_bfloat16 h[4], md[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) split3(v[k][q], h[q], md[q], lo[q]);
            const int rt = (int)(i & (kTileM - 1)), cc = (int)(j & 63);
            const size_t off = ((size_t)((i >> 7) * ntp + (j >> 6)) << 14) + (size_t)rt * 128 +
                               ((size_t)((cc >> 3) ^ (rt & 7)) << 4) + (size_t)(cc & 7) * 2;
            *reinterpret_cast<uint2*>(a3 + off) = *reinterpret_cast<const uint2*>(h);
            *reinterpret_cast<uint2*>(a3 + part_bytes + off) = *reinterpret_cast<const uint2*>(md);
            *reinterpret_cast<uint2*>(a3 + 2 * part_bytes + off) = *reinterpret_cast<const uint2*>(lo);
        }
        if (i >= m) continue;
        if (acopy && j < ldc)
            *reinterpret_cast<float4*>(acopy + i * ldc + j) = make_float4(v[k][0], v[k][1], v[k][2], v[k][3]);
    }
    if (!at) return;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int idx = tid + 256 * k;
        const int jr = idx >> 4, i4 = (idx & 15) * 4;
        const long long j = j0 + jr, i = i0 + i4;
        if (j < n && i < ldt)
            *reinterpret_cast<float4*>(at + j * ldt + i) =
                make_float4(tile[i4][jr], tile[i4 + 1][jr], tile[i4 + 2][jr], tile[i4 + 3][jr]);
    }
}

// q3 column x * ellp + j = part x of panel column j (zero for ell <= j < ellp).
__device__ __forceinline__ void split_panel_body(const float* q, long long ldq, long long rows, int ell, int ellp,
                                                 __nv_bfloat16* q3, long long ldq3, const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const long long total = rows * ellp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / rows, i = e % rows;
        __nv_bfloat16 h, md, lo;
        split3(j < ell ? q[j * ldq + i] : 0.f, h, md, lo);
        q3[j * ldq3 + i] = h;
        q3[(ellp + j) * ldq3 + i] = md;
        q3[(2 * ellp + j) * ldq3 + i] = lo;
    }
}

__global__ void split_panel_kernel(const float* q, long long ldq, long long rows, int ell, int ellp,
                                   __nv_bfloat16* q3, long long ldq3, const int* cancel) {
    split_panel_body(q, ldq, rows, ell, ellp, q3, ldq3, cancel);
}

// Tiled bf16 copy of A for the sketch products (and, with three parts, the
// exact splits A = A_h + A_m + A_l of the projection): tile (I, J) holds rows
// 128 I .. 128 I + 127 and columns 64 J .. 64 J + 63 (zero beyond m, n) in 16 KB
// at byte ((I ntp + J) << 14) of each part, laid out as a 128-byte-swizzled TMA
// box would land in shared memory: row r at 128 r, its 16-byte chunk c at
// chunk position c ^ (r mod 8). A product then moves each stage of A with one
// contiguous bulk copy, and the same tiles serve as the K-major operand of A X
// (128 rows x 64 K) and as the MN-major operand of A^T Y (64-column atoms of
// 128 K rows). ntp (tiles per row block) is even, so 128-column blocks are
// whole pairs. A block converts 128 rows x 512 columns: 128 threads per row,
// four columns each (2 KB of FP32 read per row, 128-byte lines written).
// NP = 1: A_h only; 3: A_h, A_m, A_l; 2: A_m, A_l only (parts 1 and 2).
// Row blocks rb0 + blockIdx.y.
template <typename TI, int NP>
__device__ __forceinline__ void cast_tiled_body(const TI* a, long long m, long long n, long long lda, uint8_t* out,
                                                long long ntp, long long part_bytes, long long rb0,
                                                const int* cancel) {
    pdl_trigger();
    pdl_wait();
    if (cancel && *cancel) return;
    const long long I = rb0 + blockIdx.y;
    const int half = threadIdx.x >> 7, t = threadIdx.x & 127;
    const long long c = (long long)blockIdx.x * 512 + 4 * t;  // first of this thread's four columns
    const long long J = c >> 6;
    if (J >= ntp) return;
    const int cc = (int)(c & 63);
    const bool vec = sizeof(TI) == 4 && (reinterpret_cast<uintptr_t>(a) & 15) == 0 && (lda & 3) == 0;
    uint8_t* tile = out + ((I * ntp + J) << 14);
    for (int r = half; r < kTileM; r += 2) {
        const long long row = I * kTileM + r;
        float v[4];
        if (row < m && vec && c + 3 < n) {
            const float4 f = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a) + row * lda + c);
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = 0.f;
        }
        const size_t off = (size_t)r * 128 + ((size_t)(((cc >> 3) ^ (r & 7))) << 4) + (size_t)(cc & 7) * 2;
        if (NP == 1) {
            __nv_bfloat16 h[4];
            if (row < m && vec && c + 3 < n) {
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = to_bf16(v[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) h[q] = (row < m && c + q < n) ? to_bf16(a[row * lda + c + q]) : to_bf16(0.f);
            }
            *reinterpret_cast<uint2*>(tile + off) = *reinterpret_cast<const uint2*>(h);
        } else {
            if (!(row < m && vec && c + 3 < n)) {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = (row < m && c + q < n) ? (float)a[row * lda + c + q] : 0.f;
            }
            __nv_bfloat16 h[4], md[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) split3(v[q], h[q], md[q], lo[q]);
            if (NP == 3) *reinterpret_cast<uint2*>(tile + off) = *reinterpret_cast<const uint2*>(h);
            *reinterpret_cast<uint2*>(tile + part_bytes + off) = *reinterpret_cast<const uint2*>(md);
            *reinterpret_cast<uint2*>(tile + 2 * part_bytes + off) = *reinterpret_cast<const uint2*>(lo);
        }
    }
}

template <typename TI, int NP>
__global__ void __launch_bounds__(256)
cast_tiled_kernel(const TI* a, long long m, long long n, long long lda, uint8_t* out, long long ntp,
                  long long part_bytes, long long rb0, const int* cancel) {
    cast_tiled_body<TI, NP>(a, m, n, lda, out, ntp, part_bytes, rb0, cancel);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 2-D tiled map over a row-major (outer x inner) matrix with row stride ld elements.
cudaError_t encode_2d(CUtensorMap* map, const void* base, bool f32, long long inner, long long outer, long long ld,
                      uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return cudaErrorMisalignedAddress;
    const int es = f32 ? 4 : 2;
    if ((ld * es) % 16 != 0) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

struct Plan {
    long long mtot, ktot, mtiles, kc, units;
    int grid, maxp;
};

// kseg K segments of ktot_seg elements each (split products use 3); a K
// chunk is kgroup 128-byte boxes.
Plan make_plan(long long mtot, long long ktot_seg, int kseg, bool tf32, int num_sms, int kgroup) {
    Plan pl;
    pl.mtot = mtot;
    pl.ktot = ktot_seg;
    const int ke = (tf32 ? 32 : 64) * kgroup;
    pl.mtiles = (pl.mtot + kTileM - 1) / kTileM;
    pl.kc = kseg * ((ktot_seg + ke - 1) / ke);
    pl.units = pl.mtiles * pl.kc;
    pl.grid = (int)std::min<long long>(num_sms, pl.units);
    pl.maxp = 1;
    for (long long t = 0; t < pl.mtiles; ++t) {
        const long long np = unit_owner((t + 1) * pl.kc - 1, pl.units, pl.grid) - unit_owner(t * pl.kc, pl.units, pl.grid) + 1;
        pl.maxp = std::max<int>(pl.maxp, (int)np);
    }
    return pl;
}

uint32_t make_idesc(bool tf32, bool a_mn_major, int n) {
    uint32_t d = 0;
    d |= 1u << 4;                             // D format: FP32
    d |= (tf32 ? 2u : 1u) << 7;               // A format: TF32 / BF16
    d |= (tf32 ? 2u : 1u) << 10;              // B format
    d |= (a_mn_major ? 1u : 0u) << 15;        // A major-ness
    d |= (uint32_t)(n >> 3) << 17;            // N >> 3
    d |= (uint32_t)(kTileM >> 4) << 24;       // M >> 4
    return d;
}

// Parameters and B tensor map of one product. units_per_cta > 0: the grid is
// the problem's own (about that many units per CTA, at most num_sms CTAs) and
// the ring and accumulators are sized so that two CTAs share an SM (a
// problem of a grouped launch); 0: one CTA per SM on min(num_sms, units).
struct TcBuilt {
    TcParams p;
    CUtensorMap map_b;
    size_t smem;
};

cudaError_t tc_build(TcBuilt& out, bool tf32, long long mtot, long long ktot_seg, int kseg, long long seg_stride,
                     int a_boxes, int a_box_cols, const void* b, long long ldb, long long brows_k, int nparts,
                     int trans, int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* c, ElemType tcout,
                     int64_t ldc, int num_sms, int* flags, const int* cancel, int kgroup, int stages_req,
                     TcPieces* pieces, const uint8_t* a_tiles, long long a_ntp, long long a_seg_bytes,
                     int units_per_cta = 0) {
    Plan pl = make_plan(mtot, ktot_seg, kseg, tf32, num_sms, kgroup);
    if (units_per_cta > 0) {
        const long long g = std::min<long long>(num_sms, (pl.units + units_per_cta - 1) / units_per_cta);
        pl = make_plan(mtot, ktot_seg, kseg, tf32, (int)std::max<long long>(1, g), kgroup);
    }
    const int ke = tf32 ? 32 : 64;  // K elements per 128-byte row
    const int nb = nparts * (int)ellp;
    TcParams& p = out.p;
    p = TcParams{};
    p.units = pl.units;
    p.kchunks = pl.kc;
    p.kc_seg = (int)(pl.kc / kseg);
    p.seg_stride = (int)seg_stride;
    p.grid = pl.grid;
    p.maxp = pl.maxp;
    p.ellp = (int)ellp;
    p.nparts = nparts;
    p.trans = trans;
    p.tf32 = tf32 ? 1 : 0;
    p.kchunk_elems = ke * kgroup;
    p.kgroup = kgroup;
    p.part = static_cast<float*>(part);
    p.tile_cnt = tile_cnt;
    p.out = c;
    p.out_f64 = tcout == T_F64 ? 1 : 0;
    p.ell = (int)ell;
    p.ldc = ldc;
    p.mtot = mtot;
    p.flags = flags;
    p.cancel = cancel;
    p.defer = pieces ? 1 : 0;
    if (pieces) {
        pieces->part = static_cast<const float*>(part);
        pieces->units = pl.units;
        pieces->kc = pl.kc;
        pieces->grid = pl.grid;
        pieces->maxp = pl.maxp;
        pieces->ellp = (int)ellp;
    }
    p.a_boxes = a_boxes;
    p.a_box_cols = a_box_cols;
    p.a_tiles = a_tiles;
    p.a_ntp = a_ntp;
    p.a_seg_bytes = a_seg_bytes;
    if (a_tiles && (tf32 || (reinterpret_cast<uintptr_t>(a_tiles) & 15) != 0))
        return cudaErrorInvalidValue;
    p.b_boxes = nb > 256 ? 2 : 1;
    p.b_box_rows = nb / p.b_boxes;
    cudaError_t e = encode_2d(&out.map_b, b, tf32, brows_k, nb, ldb, (uint32_t)ke, (uint32_t)p.b_box_rows,
                              CU_TENSOR_MAP_SWIZZLE_128B);
    if (e != cudaSuccess) return e;
    // MMA N chunks: one if nb <= 256, else two multiples of 16
    if (nb <= 256) {
        p.n0 = nb;
        p.n1 = 0;
    } else {
        p.n0 = (nb / 2 + 15) / 16 * 16;
        p.n1 = nb - p.n0;
    }
    p.idesc0 = make_idesc(tf32, trans != 0, p.n0);
    p.idesc1 = p.n1 ? make_idesc(tf32, trans != 0, p.n1) : 0;
    p.a_bytes = kTileM * 128;
    p.stage_bytes = (uint32_t)kgroup * (p.a_bytes + (uint32_t)nb * 128);
    // a problem of a grouped launch: a ring of at most 100 KB and 256 tensor-memory
    // columns (two CTAs per SM), unless two stages need more (the widest split
    // projections: then one CTA per SM, as a one-problem launch)
    bool shared_sm = units_per_cta > 0 && 2 * (int)p.stage_bytes <= 100 * 1024;
    const int budget = shared_sm ? 100 * 1024 : 200 * 1024;
    p.stages = std::min<int>(kMaxStages, budget / (int)p.stage_bytes);
    if (stages_req > 0) p.stages = std::min(p.stages, stages_req);
    if (p.stages < 2) return cudaErrorInvalidValue;
    uint32_t cols = 32;
    while (cols < (uint32_t)nb) cols <<= 1;
    const uint32_t tmem_cap = shared_sm ? 256u : 512u;
    p.nacc = (2 * cols <= tmem_cap) ? 2 : 1;
    p.acc_cols = cols;
    p.tmem_cols = p.nacc * cols;
    if (p.tmem_cols > tmem_cap) return cudaErrorInvalidValue;
    out.smem = (size_t)p.stages * p.stage_bytes + 1024;
    return cudaSuccess;
}

// Shared launcher. A: rows x cols row-major (K-major for trans = 0, MN-major
// for trans = 1) with `kseg` K segments `seg_stride` columns apart; B: panel
// with nparts * ellp rows of the K-major operand (ldb); output: the panel c
// (ell columns, type tcout) = sum over the nparts column groups.
// One launch of the product with kgroup K boxes per stage and `stages_req`
// ring stages (0: as many as fit 200 KB).
cudaError_t tc_launch_cfg(const void* a, bool tf32, long long mtot, long long ktot_seg, int kseg, long long seg_stride,
                          const CUtensorMap& map_a, int a_boxes, int a_box_cols, const void* b, long long ldb,
                          long long brows_k, int nparts, int trans, int64_t ell, int64_t ellp, void* part,
                          int* tile_cnt, void* c,
                          ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                          int kgroup, int stages_req, TcPieces* pieces, const uint8_t* a_tiles, long long a_ntp,
                          long long a_seg_bytes) {
    (void)a;
    TcBuilt tb;
    cudaError_t e = tc_build(tb, tf32, mtot, ktot_seg, kseg, seg_stride, a_boxes, a_box_cols, b, ldb, brows_k, nparts,
                             trans, ell, ellp, part, tile_cnt, c, tcout, ldc, num_sms, flags, cancel, kgroup,
                             stages_req, pieces, a_tiles, a_ntp, a_seg_bytes);
    if (e != cudaSuccess) return e;
    auto kern = tf32 ? sketch_tc_kernel<true> : sketch_tc_kernel<false>;
    e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(kern, dim3(tb.p.grid), dim3(kThreads), tb.smem, st, map_a, tb.map_b, tb.p);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Autotuner of the stage shape (corutv_set_autotune): for each product shape
// (M and K extents, K segments, operand kind, B width, direction, output
// handling, grid) the first launch times the candidates -- one or two
// 128-byte K boxes per stage, each with the deepest ring that fits and with
// half of it -- three launches each with CUDA events on the caller's stream,
// keeps the fastest (its best launch) for the process, and launches it;
// later launches of that shape use the kept choice. Off, or while a stream
// is being captured into a graph, the rule of sketch_kgroup applies.
struct TuneKey {
    long long mtot, ktot;
    int kseg, tf32, trans, tiled, nb, sms, out_f64, defer;
    bool operator<(const TuneKey& o) const {
        return std::tie(mtot, ktot, kseg, tf32, trans, tiled, nb, sms, out_f64, defer) <
               std::tie(o.mtot, o.ktot, o.kseg, o.tf32, o.trans, o.tiled, o.nb, o.sms, o.out_f64, o.defer);
    }
};
struct TuneVal {
    int kgroup, stages;
    float us;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
std::vector<TuneKey> g_tune_order;
std::atomic<int> g_tune_on{0};

cudaError_t tc_launch(const void* a, bool tf32, long long mtot, long long ktot_seg, int kseg, long long seg_stride,
                      const CUtensorMap& map_a, int a_boxes, int a_box_cols, const void* b, long long ldb,
                      long long brows_k, int nparts, int trans, int64_t ell, int64_t ellp, void* part,
                      int* tile_cnt, void* c,
                      ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                      int kgroup, TcPieces* pieces, const uint8_t* a_tiles = nullptr, long long a_ntp = 0,
                      long long a_seg_bytes = 0) {
    auto go = [&](int kg, int stages) {
        return tc_launch_cfg(a, tf32, mtot, ktot_seg, kseg, seg_stride, map_a, a_boxes, a_box_cols, b, ldb, brows_k,
                             nparts, trans, ell, ellp, part, tile_cnt, c, tcout, ldc, num_sms, flags, cancel, st, kg,
                             stages, pieces, a_tiles, a_ntp, a_seg_bytes);
    };
    if (!g_tune_on.load(std::memory_order_relaxed)) return go(kgroup, 0);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return go(kgroup, 0);
    }
    const int nb = nparts * (int)ellp;
    const TuneKey key{mtot, ktot_seg, kseg, tf32 ? 1 : 0, trans, a_tiles ? 1 : 0, nb, num_sms,
                      tcout == T_F64 ? 1 : 0, pieces ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return go(it->second.kgroup, it->second.stages);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    TuneVal best{kgroup, 0, 1e30f};
    for (int kg = 1; kg <= 2 && e == cudaSuccess; ++kg) {
        const int smax = std::min<int>(kMaxStages, (200 * 1024) / (kg * (kTileM * 128 + nb * 128)));
        for (int stages : {smax, smax / 2}) {
            if (stages < 2 || (stages == smax / 2 && smax / 2 == smax)) continue;
            float t_best = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, st);
                if (e == cudaSuccess) e = go(kg, stages);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess) t_best = std::min(t_best, 1000.f * ms);
            }
            if (e == cudaSuccess && t_best < best.us) best = TuneVal{kg, stages, t_best};
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune.emplace(key, best).second) g_tune_order.push_back(key);
    }
    return go(best.kgroup, best.stages);
}

}  // namespace

void tc_set_autotune(bool on) { g_tune_on.store(on ? 1 : 0); }

int tc_autotune_entry(int index, long long* mtot, long long* ktot, int* nb, int* trans, int* kgroup, int* stages,
                      float* us) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (index < 0 || index >= (int)g_tune_order.size()) return (int)g_tune_order.size();
    const TuneKey& k = g_tune_order[index];
    const TuneVal& v = g_tune.at(k);
    *mtot = k.mtot;
    *ktot = k.ktot;
    *nb = k.nb;
    *trans = k.trans;
    *kgroup = v.kgroup;
    *stages = v.stages;
    *us = v.us;
    return (int)g_tune_order.size();
}

int64_t tc_counter_elems(int64_t m, int64_t n) { return (std::max(m, n) + kTileM - 1) / kTileM; }

int64_t tc_partial_elems(int64_t m, int64_t n, int64_t ellp, int64_t ldm, int64_t ldn, int num_sms) {
    (void)ldm;
    (void)ldn;
    int64_t best = 0;
    for (int trans = 0; trans < 2; ++trans)
        for (int tf = 0; tf < 2; ++tf)
            for (int kseg : {1, 2, 3})
                for (int kgroup : {1, 2}) {
                    const Plan pl = make_plan(trans ? n : m, trans ? m : n, kseg, tf != 0, num_sms, kgroup);
                    best = std::max<int64_t>(best, pl.mtiles * pl.maxp * ellp * kTileM);
                }
    return best;
}

// Two 128-byte K boxes per stage (twice the bytes per copy; measured about 8 %
// faster on the 8000 x 6000 products at ell = 60 and 12 % at 12000 x 12000,
// ell = 110, where the ring then holds three stages instead of six) whenever
// three such stages fit the 200 KB ring; nb = B columns per stage (nparts x
// ellp), so the split projection's three-times-wider B keeps one box.
int sketch_kgroup(int64_t nb) { return 3 * 2 * (16384 + nb * 128) <= 200 * 1024 ? 2 : 1; }

cudaError_t launch_sketch_tc(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, int trans,
                             const void* x, int64_t ldx, int64_t ell, int64_t ellp, void* part, int* tile_cnt,
                             void* c, ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel,
                             cudaStream_t st, TcPieces* pieces) {
    if (ta != T_BF16 && ta != T_F32) return cudaErrorInvalidValue;
    if (ellp % 16 != 0 || ellp < 16 || ellp > 128 || ell > ellp) return cudaErrorInvalidValue;
    // The MN-major tf32 operand form (A^T Y in TF32) is not enabled.
    if (ta == T_F32 && trans) return cudaErrorNotSupported;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    const bool tf32 = ta == T_F32;
    const int ke = tf32 ? 32 : 64;
    CUtensorMap map_a;
    int a_boxes = 1, a_box_cols = 0;
    if (!trans) {
        e = encode_2d(&map_a, a, tf32, n, m, lda, (uint32_t)ke, kTileM, CU_TENSOR_MAP_SWIZZLE_128B);
    } else {
        // MN-major A: boxes of one 128-byte MN atom (64 bf16 columns) by ke rows
        const int atom = 64;
        e = encode_2d(&map_a, a, false, n, m, lda, (uint32_t)atom, (uint32_t)ke, CU_TENSOR_MAP_SWIZZLE_128B);
        a_boxes = kTileM / atom;
        a_box_cols = atom;
    }
    if (e != cudaSuccess) return e;
    return tc_launch(a, tf32, trans ? n : m, trans ? m : n, 1, 0, map_a, a_boxes, a_box_cols, x, ldx, trans ? m : n,
                     1, trans, ell, ellp, part, tile_cnt, c, tcout, ldc, num_sms, flags, cancel, st,
                     sketch_kgroup(ellp), pieces);
}

int64_t tiled_ntp(int64_t n) { return ((n + 63) / 64 + 1) / 2 * 2; }

int64_t tiled_part_bytes(int64_t m, int64_t n) { return ((m + kTileM - 1) / kTileM) * tiled_ntp(n) * 16384; }

cudaError_t launch_cast_tiled_rows(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* out,
                                   int parts, int64_t rb0, int64_t rb1, const int* cancel, cudaStream_t st) {
    if (m < 1 || n < 1 || lda < n || !out || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return cudaErrorInvalidValue;
    if (parts != 1 && !((parts == 2 || parts == 3) && ta == T_F32)) return cudaErrorInvalidValue;
    const int64_t ntp = tiled_ntp(n), mt = (m + kTileM - 1) / kTileM;
    if (rb0 < 0 || rb1 > mt || rb0 >= rb1 || rb1 - rb0 > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((ntp + 7) / 8), (unsigned)(rb1 - rb0));
    const long long pb = tiled_part_bytes(m, n);
    uint8_t* o = static_cast<uint8_t*>(out);
    count_launch();
    cudaError_t e;
    if (ta == T_F64)
        e = launch_pdl(cast_tiled_kernel<double, 1>, grid, dim3(256), (size_t)0, st, static_cast<const double*>(a),
                       (long long)m, (long long)n, (long long)lda, o, (long long)ntp, pb, (long long)rb0, cancel);
    else if (parts == 1)
        e = launch_pdl(cast_tiled_kernel<float, 1>, grid, dim3(256), (size_t)0, st, static_cast<const float*>(a),
                       (long long)m, (long long)n, (long long)lda, o, (long long)ntp, pb, (long long)rb0, cancel);
    else if (parts == 2)
        e = launch_pdl(cast_tiled_kernel<float, 2>, grid, dim3(256), (size_t)0, st, static_cast<const float*>(a),
                       (long long)m, (long long)n, (long long)lda, o, (long long)ntp, pb, (long long)rb0, cancel);
    else
        e = launch_pdl(cast_tiled_kernel<float, 3>, grid, dim3(256), (size_t)0, st, static_cast<const float*>(a),
                       (long long)m, (long long)n, (long long)lda, o, (long long)ntp, pb, (long long)rb0, cancel);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_cast_tiled(const void* a, ElemType ta, int64_t m, int64_t n, int64_t lda, void* out, int nparts,
                              const int* cancel, cudaStream_t st) {
    if (nparts != 1 && nparts != 3) return cudaErrorInvalidValue;
    return launch_cast_tiled_rows(a, ta, m, n, lda, out, nparts, 0, (m + kTileM - 1) / kTileM, cancel, st);
}

cudaError_t launch_sketch_tc_tiled(const void* a_tiles, int64_t m, int64_t n, int trans, const void* x, int64_t ldx,
                                   int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* c, ElemType tcout,
                                   int64_t ldc, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                                   TcPieces* pieces, int nsegs) {
    if (ellp % 16 != 0 || ellp < 16 || ellp > 128 || ell > ellp || nsegs < 1 || nsegs > 3) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    CUtensorMap unused{};
    const uint8_t* at = static_cast<const uint8_t*>(a_tiles);
    return tc_launch(a_tiles, false, trans ? n : m, trans ? m : n, nsegs, 0, unused, 1, 0, x, ldx, trans ? m : n, 1, trans,
                     ell, ellp, part, tile_cnt, c, tcout, ldc, num_sms, flags, cancel, st, sketch_kgroup(ellp), pieces,
                     at, tiled_ntp(n), tiled_part_bytes(m, n));
}

cudaError_t launch_project_split_tc_tiled(const void* a3, int64_t m, int64_t n, const void* q3, int64_t ldq,
                                          int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* w, ElemType tw,
                                          int64_t ldw, int num_sms, int* flags, const int* cancel, cudaStream_t st,
                                          TcPieces* pieces) {
    if (ellp % 16 != 0 || ellp < 16 || ellp > 128 || ell > ellp) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    CUtensorMap unused{};
    // the K chunks of each split segment stay inside it: the segment's tiles are
    // kgroup-aligned (ntp is even)
    const int kgroup = sketch_kgroup(3 * ellp);
    return tc_launch(a3, false, m, n, 3, 0, unused, 1, 0, q3, ldq, n, 3, 0, ell, ellp, part, tile_cnt, w, tw, ldw,
                     num_sms, flags, cancel, st, kgroup, pieces, static_cast<const uint8_t*>(a3), tiled_ntp(n),
                     tiled_part_bytes(m, n));
}

// ---------------------------------------------------------------------------
// Grouped products (the problems of a batch in one launch)
// ---------------------------------------------------------------------------
namespace {
// stream-K units (128 rows by one 128-byte K box) per CTA of a grouped product; one K box per stage
constexpr int kGroupUnitsPerCta = 64;

// (the host record may sit anywhere: it is assembled aligned and copied in)
cudaError_t group_fill(void* item, const TcBuilt& tb, int* grid, size_t* smem, int64_t* part_floats) {
    TcGroupItem it;
    it.map_b = tb.map_b;
    it.p = tb.p;
    std::memcpy(item, &it, sizeof(it));
    *grid = tb.p.grid;
    *smem = tb.smem;
    const long long mtiles = (tb.p.mtot + kTileM - 1) / kTileM;
    *part_floats = mtiles * tb.p.maxp * (long long)tb.p.ellp * kTileM;
    return cudaSuccess;
}
}  // namespace

size_t tc_group_item_bytes() { return sizeof(TcGroupItem); }

int64_t tc_group_partial_elems(int64_t m, int64_t n, int64_t ellp, int num_sms) {
    int64_t best = 0;
    const long long ext[3][3] = {{m, n, 1}, {n, m, 1}, {m, n, 3}};  // A X, A^T Y, the split projection
    for (const auto& e : ext) {
        Plan pl = make_plan(e[0], e[1], (int)e[2], false, num_sms, 1);
        const long long g = std::min<long long>(num_sms, (pl.units + kGroupUnitsPerCta - 1) / kGroupUnitsPerCta);
        pl = make_plan(e[0], e[1], (int)e[2], false, (int)std::max<long long>(1, g), 1);
        best = std::max<int64_t>(best, pl.mtiles * pl.maxp * ellp * kTileM);
    }
    return best;
}

cudaError_t tc_group_sketch_item(void* item, const void* a_tiles, int64_t m, int64_t n, int trans, const void* x,
                                 int64_t ldx, int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* c,
                                 ElemType tcout, int64_t ldc, int num_sms, int* flags, const int* cancel, int* grid,
                                 size_t* smem, int64_t* part_floats) {
    if (ellp % 16 != 0 || ellp < 16 || ellp > 128 || ell > ellp) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    TcBuilt tb;
    e = tc_build(tb, false, trans ? n : m, trans ? m : n, 1, 0, 1, 0, x, ldx, trans ? m : n, 1, trans, ell, ellp, part,
                 tile_cnt, c, tcout, ldc, num_sms, flags, cancel, 1, 0, nullptr,
                 static_cast<const uint8_t*>(a_tiles), tiled_ntp(n), tiled_part_bytes(m, n), kGroupUnitsPerCta);
    if (e != cudaSuccess) return e;
    return group_fill(item, tb, grid, smem, part_floats);
}

cudaError_t tc_group_project_item(void* item, const void* a3, int64_t m, int64_t n, const void* q3, int64_t ldq,
                                  int64_t ell, int64_t ellp, void* part, int* tile_cnt, void* w, ElemType tw,
                                  int64_t ldw, int num_sms, int* flags, const int* cancel, int* grid, size_t* smem,
                                  int64_t* part_floats) {
    if (ellp % 16 != 0 || ellp < 16 || ellp > 128 || ell > ellp) return cudaErrorInvalidValue;
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    TcBuilt tb;
    e = tc_build(tb, false, m, n, 3, 0, 1, 0, q3, ldq, n, 3, 0, ell, ellp, part, tile_cnt, w, tw, ldw, num_sms, flags,
                 cancel, 1, 0, nullptr, static_cast<const uint8_t*>(a3), tiled_ntp(n), tiled_part_bytes(m, n),
                 kGroupUnitsPerCta);
    if (e != cudaSuccess) return e;
    return group_fill(item, tb, grid, smem, part_floats);
}

cudaError_t launch_sketch_tc_grouped(const void* items, int count, int max_grid, size_t max_smem, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    if (max_grid < 1 || count > 65535 || (reinterpret_cast<uintptr_t>(items) & 127) != 0) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(sketch_tc_grouped_kernel));
    if (e != cudaSuccess) return e;
    count_launch();
    e = launch_pdl(sketch_tc_grouped_kernel, dim3((unsigned)max_grid, (unsigned)count), dim3(kThreads), max_smem, st,
                   static_cast<const TcGroupItem*>(items));
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Grouped three-part cast and panel splits.
namespace {
// tiled_ntp / tiled_part_bytes on the device
__device__ __forceinline__ long long tiled_ntp_dev(long long n) { return ((n + 63) / 64 + 1) / 2 * 2; }
__device__ __forceinline__ long long tiled_part_bytes_dev(long long m, long long n) {
    return ((m + kTileM - 1) / kTileM) * tiled_ntp_dev(n) * 16384;
}
__device__ __forceinline__ void cast3_body(const CastArgs& a) {
    cast_tiled_body<float, 3>(a.a, a.m, a.n, a.lda, static_cast<uint8_t*>(a.out), tiled_ntp_dev(a.n),
                              tiled_part_bytes_dev(a.m, a.n), 0, a.cancel);
}
__device__ __forceinline__ void split_body(const SplitArgs& a) {
    split_panel_body(a.q, a.ldq, a.rows, a.ell, a.ellp, static_cast<__nv_bfloat16*>(a.q3), a.ldq3, a.cancel);
}
}  // namespace

GroupItem<CastArgs> cast3_item(const CastArgs& a) {
    GroupItem<CastArgs> it;
    it.a = a;
    it.gx = (unsigned)((tiled_ntp(a.n) + 7) / 8);
    it.gy = (unsigned)((a.m + kTileM - 1) / kTileM);
    return it;
}

GroupItem<SplitArgs> split_item(const SplitArgs& a) {
    GroupItem<SplitArgs> it;
    it.a = a;
    it.gx = kAnyGrid;
    it.gy = 1;
    return it;
}

cudaError_t launch_cast3_grouped(const GroupItem<CastArgs>* it, int count, unsigned gx, unsigned gy, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    count_launch();
    cudaError_t e = launch_pdl(grouped_kernel<CastArgs, cast3_body, 256>, dim3(gx, gy, (unsigned)count), dim3(256),
                               (size_t)0, st, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_split_grouped(const GroupItem<SplitArgs>* it, int count, unsigned gx, cudaStream_t st) {
    if (count < 1) return cudaSuccess;
    count_launch();
    cudaError_t e = launch_pdl(grouped_kernel<SplitArgs, split_body, 256>, dim3(gx, 1, (unsigned)count), dim3(256),
                               (size_t)0, st, it);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_wait_probe(int* flags, unsigned long long limit_ns, cudaStream_t st) {
    if (!flags) return cudaErrorInvalidValue;
    count_launch();
    cudaError_t e = launch_pdl(wait_probe_kernel, dim3(1), dim3(32), (size_t)0, st, flags, limit_ns);
    return e != cudaSuccess ? e : cudaGetLastError();
}

bool tma_rows_aligned(const void* a, int64_t lda, int elem_bytes) {
    return reinterpret_cast<uintptr_t>(a) % 16 == 0 && (lda * elem_bytes) % 16 == 0;
}

cudaError_t launch_copy_f32_padded(const float* a, int64_t m, int64_t n, int64_t lda, float* out, int64_t ldb,
                                   cudaStream_t st) {
    const long long total = m * ldb;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8192);
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(copy_f32_padded_kernel, dim3(blocks), dim3(256), (size_t)(0), st, a, m, n, lda, out, ldb);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

cudaError_t launch_prep_f32(const float* a, int64_t m, int64_t n, int64_t lda, float* at, int64_t ldt, void* a3,
                            float* acopy, int64_t ldc, const int* cancel, cudaStream_t st) {
    if (m < 1 || n < 1 || lda < n) return cudaErrorInvalidValue;
    // every vector store stays inside its row: the tiles cover columns up to
    // round_up(., 64) and the strides are multiples of 64 / 4
    if (at && (ldt % 64 != 0 || ldt < m || reinterpret_cast<uintptr_t>(at) % 16 != 0)) return cudaErrorInvalidValue;
    if (a3 && reinterpret_cast<uintptr_t>(a3) % 16 != 0) return cudaErrorInvalidValue;
    if (acopy && (ldc % 4 != 0 || ldc < n || ldc > (n + kPrepT - 1) / kPrepT * kPrepT ||
                  reinterpret_cast<uintptr_t>(acopy) % 16 != 0))
        return cudaErrorInvalidValue;
    // with a3, every tile of the tiled copy (128-row blocks, ntp column tiles) is written
    const int64_t ntp = tiled_ntp(n);
    const int64_t gx = a3 ? ntp : (n + kPrepT - 1) / kPrepT;
    const int64_t gy = a3 ? (m + kTileM - 1) / kTileM * (kTileM / kPrepT) : (m + kPrepT - 1) / kPrepT;
    const dim3 grid((unsigned)gx, (unsigned)gy, 1);
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(prep_f32_kernel, grid, dim3(256), (size_t)0, st, a, (long long)m, (long long)n,
                                     (long long)lda, at, (long long)ldt, static_cast<uint8_t*>(a3), (long long)ntp,
                                     (long long)tiled_part_bytes(m, n), acopy, (long long)ldc, cancel);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

cudaError_t launch_split_panel(const float* q, int64_t ldq, int64_t rows, int64_t ell, int64_t ellp, void* q3,
                               int64_t ldq3, const int* cancel, cudaStream_t st) {
    const long long total = rows * ellp;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    count_launch();
    {
        cudaError_t pe_ = launch_pdl(split_panel_kernel, dim3(blocks), dim3(256), (size_t)(0), st, q, ldq, rows, (int)ell, (int)ellp, static_cast<__nv_bfloat16*>(q3),
                                               ldq3, cancel);
        if (pe_ != cudaSuccess) return pe_;
    }
    return cudaGetLastError();
}

}  // namespace corutv
