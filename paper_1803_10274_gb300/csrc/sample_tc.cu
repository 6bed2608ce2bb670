// Fused Gaussian-kernel x block product on sm_103a tensor cores.
//
// Computes S(i, :) = sum_j w_ij K(xa_i, xb_j) R(j, :) (the sampling product
// of the randomized HSS construction; paper Section 1.1 and Section 3.1)
// without ever writing K to memory.  Per 128 x 128 tile of K:
//
//   1. distance GEMM on tcgen05 (TMA-fed, operands in shared memory,
//      accumulator in tensor memory).  The operands are augmented rows
//          A_i = [hx_i | hx_i | lx_i | a_hi a_mid a_lo | 1 1 1 | 0..]
//          B_j = [hy_j | ly_j | hy_j | 1 1 1 | b_hi b_mid b_lo | 0..]
//      where x = hx + lx and y = 2c x_j = hy + ly are FP16 hi/lo splits,
//      a_i = -c ||x_i||^2 and b_j = -c ||x_j||^2 are split into three FP16
//      parts and c = log2(e) / (2 h^2).  The FP32 accumulator then holds
//          e_ij = -c ||x_i - x_j||^2 = log2 K_ij
//      to about 2^-21 relative to the norms (the FP16 products are exact
//      in FP32; only the lo*lo terms are dropped).
//   2. epilogue warps read e_ij from tensor memory, form K_ij = 2^e_ij with
//      the SFU (ex2.approx), zero the masked (same-leaf) pairs, round to
//      FP16 and write K back into the same tensor-memory columns;
//   3. K (A operand from tensor memory) times R_J (B operand, FP16 in
//      shared memory) accumulates into S in tensor memory, FP32.
//
// Warp roles (384 threads, one CTA per SM, persistent over a contiguous
// range of (row tile, column tile) steps): warp 0 issues TMA loads, warp 1
// issues tcgen05.mma, warp 2 owns the tensor-memory allocation, warps 4-11
// (two warpgroups, one per 64-column half of a tile) run the epilogue.
// Partial row sums are added into S with global atomics when a CTA's step
// range ends or crosses a row tile.
#include <cuda.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "prep.cuh"
#include "tc_ptx.cuh"

namespace krr {
namespace tc {

constexpr int kThreads = 384;
constexpr int kBM = 128;             // rows of a tile (tensor-memory lanes)
constexpr int kBN = 128;             // K columns of a tile
constexpr int kChunk = 64;           // FP16 elements per 128-byte swizzled row
constexpr int kChunkBytes = 128 * 128;
constexpr int kMaxStages = 6;
constexpr long long kWaitBudget = kDefaultWaitCycles;  // drain waits at kernel exit

static_assert(kBM == kTcTile && kBN == kTcTile, "tile lists assume square 128-row tiles");

struct Params {
    int64_t ma, nb;
    int64_t n_row_tiles, n_col_tiles;
    int r;        // R / S columns handled by this launch (32, or a multiple of 64 up to 256)
    int r_valid;  // columns actually stored (<= r)
    int nchunk;   // 64-element chunks of an augmented row
    int kmma;     // K=16 MMA steps of the distance GEMM
    int nstage;
    int s_bufs;   // S accumulators in tensor memory (1 or 2)
    int ndist;    // distance / K buffers in tensor memory (2 or 3)
    int dist_col0;
    int split_k;  // 1: K = K_hi + K_lo (two FP16 parts, two product MMAs)
    int a_bufs;   // row-tile (A) buffers in shared memory: 2, or 1 when that buys a stage
    uint32_t chunk_bytes;  // 128 rows x 128 B (64-element chunks), or x 64 B (one 32-element chunk)
    uint32_t ab_hi;        // descriptor high word of the A / B chunks (128- or 64-byte swizzle)
    uint32_t off_a, off_stage, stage_bytes, off_bar;
    const int32_t *leaf_a, *leaf_b;
    // block-diagonal products (many independent problems in one launch):
    // problem id per row of A and B (keep a pair only within a problem),
    // and the tile list: row tile rt covers column tiles [tl_lo, tl_hi],
    // its tiles numbered from tl_off[rt]; NULL = every tile of the grid
    const int32_t *grp_a, *grp_b;
    const int32_t *tl_lo, *tl_hi;
    const int64_t *tl_off;
    int64_t n_tiles;
    float *S;
    int64_t lds;
    DevStatus *status;
    long long wait;  // limit of one hand-off wait, SM clock cycles
};

// Barrier slots (uint64 each) after off_bar.
enum {
    BAR_FULL = 0,
    BAR_EMPTY = BAR_FULL + kMaxStages,
    BAR_AFULL = BAR_EMPTY + kMaxStages,
    BAR_AEMPTY = BAR_AFULL + 2,
    BAR_DFULL = BAR_AEMPTY + 2,
    BAR_PFULL = BAR_DFULL + 3,
    BAR_SFULL = BAR_PFULL + 3,
    BAR_SEMPTY = BAR_SFULL + 2,
    BAR_DRAIN = BAR_SEMPTY + 2,
    BAR_KFREE = BAR_DRAIN + 1,   // two issuers: K buffer free again (product done)
    BAR_DRAIN2 = BAR_KFREE + 3,
    BAR_COUNT = BAR_DRAIN2 + 1
};


__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// K = 2^e for 32 exponents, rounded to FP16 and packed in pairs.
__device__ __forceinline__ void exp_pack(const uint32_t (&v)[32], uint32_t (&pk)[16]) {
#pragma unroll
    for (int c = 0; c < 16; ++c)
        pk[c] = pack_h2(ptx::ex2_approx(__uint_as_float(v[2 * c])), ptx::ex2_approx(__uint_as_float(v[2 * c + 1])));
}

// K = 2^e for 32 exponents as an FP16 pair sum K_hi + K_lo (the low part
// is the FP16-rounded remainder), both packed in pairs.
__device__ __forceinline__ void exp_pack_split(const uint32_t (&v)[32], uint32_t (&hi)[16], uint32_t (&lo)[16]) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const float e0 = ptx::ex2_approx(__uint_as_float(v[2 * c]));
        const float e1 = ptx::ex2_approx(__uint_as_float(v[2 * c + 1]));
        const __half2 h = __floats2half2_rn(e0, e1);
        const float2 hf = __half22float2(h);
        hi[c] = *reinterpret_cast<const uint32_t *>(&h);
        lo[c] = pack_h2(e0 - hf.x, e1 - hf.y);
    }
}

// Zero the FP16 halves whose bit is set in m (only tiles that cross a
// leaf of the cluster tree).
__device__ __forceinline__ void mask_pack(uint32_t (&pk)[16], uint32_t m) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const uint32_t lo = (m >> (2 * c)) & 1u, hi = (m >> (2 * c + 1)) & 1u;
        pk[c] &= (lo ? 0xFFFF0000u : 0xFFFFFFFFu) & (hi ? 0x0000FFFFu : 0xFFFFFFFFu);
    }
}

// Bits of the columns to drop for row i: the same leaf of the cluster
// tree (tiles whose leaf ranges overlap; rows and columns are in the same
// cluster order) or another problem (tiles that straddle a problem
// boundary).
__device__ __forceinline__ void tile_mask(const Params &P, int rt, int ct, int g, int64_t i, uint32_t &mlo,
                                       uint32_t &mhi) {
    const int64_t ia = int64_t(rt) * kBM, ib = min(ia + kBM - 1, P.ma - 1);
    const int64_t ja = int64_t(ct) * kBN, jb = min(ja + kBN - 1, P.nb - 1);
    mlo = mhi = 0;
    bool leaf_x = false, grp_x = false;
    if (P.leaf_a != nullptr) {
        const int32_t lo = max(__ldg(P.leaf_a + ia), __ldg(P.leaf_b + ja));
        const int32_t hi = min(__ldg(P.leaf_a + ib), __ldg(P.leaf_b + jb));
        leaf_x = lo <= hi;
    }
    if (P.grp_a != nullptr) {
        const int32_t g0 = __ldg(P.grp_a + ia);
        grp_x = !(g0 == __ldg(P.grp_a + ib) && g0 == __ldg(P.grp_b + ja) && g0 == __ldg(P.grp_b + jb));
    }
    if (!leaf_x && !grp_x) return;
    const int64_t ic = min(i, P.ma - 1);
    const int32_t li = leaf_x ? __ldg(P.leaf_a + ic) : 0;
    const int32_t gi = grp_x ? __ldg(P.grp_a + ic) : 0;
    const int64_t j0 = int64_t(ct) * kBN + 64 * g;
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
        const int64_t j = j0 + c, j2 = j0 + 32 + c;
        if (j < P.nb && ((leaf_x && __ldg(P.leaf_b + j) == li) || (grp_x && __ldg(P.grp_b + j) != gi)))
            mlo |= 1u << c;
        if (j2 < P.nb && ((leaf_x && __ldg(P.leaf_b + j2) == li) || (grp_x && __ldg(P.grp_b + j2) != gi)))
            mhi |= 1u << c;
    }
}

// Add this warpgroup's half of the row-tile accumulator into S and hand
// the tensor-memory buffer back to the MMA issuer.
// A segment that covers its row tile's whole column range is the only
// contribution to those rows of S (zeroed before the launch): plain stores,
// no read-modify-write.
__device__ __forceinline__ void flush_s(const Params &P, uint64_t *bars, volatile int *abort_flag, uint32_t tmem,
                                     uint32_t lane_off, int64_t seg, int g, int rh, int64_t i, bool whole) {
    using namespace ptx;
    const int lane = threadIdx.x & 31;
    const int sb = P.s_bufs == 2 ? int(seg & 1) : 0;
    const uint32_t par = P.s_bufs == 2 ? uint32_t((seg >> 1) & 1) : uint32_t(seg & 1);
    if (!warp_wait(&bars[BAR_SFULL + sb], par, abort_flag, P.wait, P.status, 8)) return;
    tc_fence_after();
    for (int cc = 0; cc < rh; cc += 32) {
        uint32_t sv[32];
        tmem_ld32(tmem + lane_off + uint32_t(sb * P.r + g * rh + cc), sv);
        tmem_wait_ld();
        if (i < P.ma) {
            float *dst = P.S + i * P.lds;
            const int cbase = g * rh + cc;
            const int cend = min(32, rh - cc);  // r = 32: each half is 16 columns
            if (whole) {
                for (int c = 0; c < cend; ++c)
                    if (cbase + c < P.r_valid) dst[cbase + c] = __uint_as_float(sv[c]);
            } else {
                for (int c = 0; c < cend; ++c)
                    if (cbase + c < P.r_valid) atomicAdd(dst + cbase + c, __uint_as_float(sv[c]));
            }
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars[BAR_SEMPTY + sb]);
}

// Position in a CTA's range of tile steps, advanced incrementally (no
// integer division in the loops): tile (rt, ct), the column-tile range
// [lo, hi] of row tile rt, shared-memory stage and distance-buffer rings
// with their phase bits, row-tile segment count.
struct Cursor {
    int loc, rt, ct, lo, hi, stage, db, seg;
    uint32_t sphase, dphase;
    bool first, last;
    __device__ __forceinline__ void init(const Params &P, int64_t t0, int nct) {
        loc = 0;
        if (P.tl_off != nullptr) {
            int a = 0, b = int(P.n_row_tiles) - 1;  // last row tile whose first tile is <= t0
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (__ldg(P.tl_off + mid) <= t0) a = mid;
                else b = mid - 1;
            }
            rt = a;
            lo = __ldg(P.tl_lo + rt);
            hi = __ldg(P.tl_hi + rt);
            ct = lo + int(t0 - __ldg(P.tl_off + rt));
        } else {
            rt = int(t0 / nct);
            ct = int(t0 % nct);
            lo = 0;
            hi = nct - 1;
        }
        stage = db = 0;
        sphase = dphase = 0;
        seg = 0;
    }
    // flags of the current tile; `first` opens a new row-tile segment
    __device__ __forceinline__ void flags(int nloc) {
        first = (loc == 0) || (ct == lo);
        last = (loc == nloc - 1) || (ct == hi);
    }
    __device__ __forceinline__ void next(const Params &P, int nloc, int NS, int ND) {
        ++loc;
        if (++ct > hi) {
            ++rt;
            if (P.tl_off != nullptr && loc < nloc) {
                lo = __ldg(P.tl_lo + rt);
                hi = __ldg(P.tl_hi + rt);
            }
            ct = lo;
        }
        if (++stage == NS) {
            stage = 0;
            sphase ^= 1u;
        }
        if (++db == ND) {
            db = 0;
            dphase ^= 1u;
        }
    }
};

// PAIR = true: clusters of two CTAs walk the same column tiles for two
// adjacent row tiles (CTA rank q takes row tile 2 u + q of row unit u).
// Each column tile's B rows and R tile are read from L2 once: each CTA
// loads half of them (its half of the B rows, its 64 columns of R^T) and
// multicasts it into both CTAs' stage; a stage is free again once both
// CTAs' MMAs have released it.  P.n_row_tiles then counts row units and
// the tile list (if any) is over row units.
//
// TWO = true: the distance MMAs and the product MMAs are issued by two
// threads (warps 1 and 3), which doubles the issue rate where each tile's
// MMAs are small (r <= 128, or K split into two FP16 parts); the product
// thread releases each K buffer through BAR_KFREE, which the distance
// thread waits for before it rewrites the buffer (one issuing thread gets
// that order from the tensor core's in-order execution).
template <bool PAIR, bool TWO>
__global__ void __launch_bounds__(kThreads, 1)
    sample_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmR, const Params P) {
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + P.off_bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + BAR_COUNT);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int nct = int(P.n_col_tiles);
    const int64_t T = P.n_tiles;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const int64_t unit = PAIR ? blockIdx.x / 2 : blockIdx.x, nunits = PAIR ? gridDim.x / 2 : gridDim.x;
    const int64_t t0 = T * unit / nunits;
    const int nloc = int(T * (unit + 1) / nunits - t0);
    const int NS = P.nstage, ND = P.ndist;
    // this CTA's row tile within row unit u
    auto row_tile = [&](int u) -> int { return PAIR ? 2 * u + int(rank) : u; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[BAR_FULL + s], 1);
            mbar_init(&bars[BAR_EMPTY + s], PAIR ? 2 : 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars[BAR_AFULL + b], 1);
            mbar_init(&bars[BAR_AEMPTY + b], 1);
            mbar_init(&bars[BAR_SFULL + b], 1);
            mbar_init(&bars[BAR_SEMPTY + b], 8);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(&bars[BAR_DFULL + b], 1);
            mbar_init(&bars[BAR_PFULL + b], 8);
        }
        mbar_init(&bars[BAR_DRAIN], 1);
        mbar_init(&bars[BAR_DRAIN2], 1);
        for (int b = 0; b < 3; ++b) mbar_init(&bars[BAR_KFREE + b], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        tma_prefetch_desc(&tmR);
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();  // the peer's barriers are initialized
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_bytes = P.nchunk * P.chunk_bytes;

    if (warp == 0 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ TMA producer
        Cursor c;
        c.init(P, t0, nct);
        int issued = 0, a_issued = -1;
        for (; c.loc < nloc; c.next(P, nloc, NS, 1)) {
            c.flags(nloc);
            if (c.first) {
                const int seg = c.seg++;
                const int ab = P.a_bufs == 2 ? (seg & 1) : 0;
                const int au = P.a_bufs == 2 ? (seg >> 1) : seg;  // use count of that buffer
                if (!mbar_wait(&bars[BAR_AEMPTY + ab], uint32_t(au & 1) ^ 1u, abort_flag, P.wait,
                               P.status, 1))
                    break;
                mbar_expect_tx(&bars[BAR_AFULL + ab], a_bytes);
                for (int ch = 0; ch < P.nchunk; ++ch)
                    tma_load_2d(smem + P.off_a + ab * a_bytes + ch * P.chunk_bytes, &tmA, &bars[BAR_AFULL + ab],
                                ch * kChunk, row_tile(c.rt) * kBM);
                a_issued = seg;
            }
            // PAIR: the wait also covers the peer's MMAs, so both CTAs'
            // copies of this stage are free before either half is sent
            if (!mbar_wait(&bars[BAR_EMPTY + c.stage], c.sphase ^ 1u, abort_flag, P.wait, P.status, 2)) break;
            uint8_t *st = smem + P.off_stage + c.stage * P.stage_bytes;
            mbar_expect_tx(&bars[BAR_FULL + c.stage], P.stage_bytes);
            if (PAIR) {
                // rank q: B rows [64 q, 64 q + 64) of the tile (a 64-row box at
                // byte 8192 q keeps the 128-byte swizzle of the full tile) and
                // R^T columns [64 q, 64 q + 64), both to both CTAs
                const int q = int(rank);
                for (int ch = 0; ch < P.nchunk; ++ch)
                    tma_load_2d_mc(st + ch * P.chunk_bytes + q * (P.chunk_bytes / 2), &tmB, &bars[BAR_FULL + c.stage],
                                   ch * kChunk, c.ct * kBN + 64 * q, uint16_t(3));
                tma_load_2d_mc(st + a_bytes + q * P.r * 128, &tmR, &bars[BAR_FULL + c.stage], c.ct * kBN + 64 * q,
                               0, uint16_t(3));
            } else {
                for (int ch = 0; ch < P.nchunk; ++ch)
                    tma_load_2d(st + ch * P.chunk_bytes, &tmB, &bars[BAR_FULL + c.stage], ch * kChunk, c.ct * kBN);
                tma_load_2d(st + a_bytes, &tmR, &bars[BAR_FULL + c.stage], c.ct * kBN, 0);
                tma_load_2d(st + a_bytes + P.r * 128, &tmR, &bars[BAR_FULL + c.stage], c.ct * kBN + 64, 0);
            }
            ++issued;
        }
        const bool aborted = *abort_flag != 0;
        // Drain: wait (bounded) until every load issued has landed, so no
        // TMA write is in flight when the CTA exits.
        for (int k = 0; k < (issued < NS ? issued : NS); ++k) {
            const int u = issued - 1 - k;
            mbar_wait_bounded(&bars[BAR_FULL + (u % NS)], uint32_t((u / NS) & 1), kWaitBudget);
        }
        // Row-tile loads: only the last a_bufs can still be in flight (an
        // earlier one into the same buffer was consumed before its reuse).
        for (int sg = a_issued; sg >= 0 && sg > a_issued - P.a_bufs; --sg)
            mbar_wait_bounded(&bars[BAR_AFULL + (P.a_bufs == 2 ? (sg & 1) : 0)],
                              uint32_t((P.a_bufs == 2 ? (sg >> 1) : sg) & 1), kWaitBudget);
        if (PAIR) {
            // The peer's MMAs release this CTA's stages by remote commits:
            // wait until the last use of every stage has both releases, so
            // no arrival is still on its way when the CTA exits.  After an
            // abort the peer may have stopped early (short bound), and its
            // multicast halves of steps this CTA never armed get a grace
            // period to land.
            const long long lim = aborted ? 200000ll : kWaitBudget;
            for (int k = 0; k < (issued < NS ? issued : NS); ++k) {
                const int u = issued - 1 - k;
                mbar_wait_bounded(&bars[BAR_EMPTY + (u % NS)], uint32_t((u / NS) & 1), lim);
            }
            if (aborted) {
                const long long tg = clock64();
                while (clock64() - tg < 200000ll) {
                }
            }
        }
    } else if (TWO && warp == 1 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ distance MMA issuer
        const uint32_t idesc_d = idesc_f16_f32(kBM, kBN);
        const uint32_t a_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_a));
        const uint32_t b_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_stage));
        const uint32_t a_units = a_bytes >> 4, stage_units = P.stage_bytes >> 4;
        Cursor cd;
        cd.init(P, t0, nct);
        for (; cd.loc < nloc; cd.next(P, nloc, NS, ND)) {
            cd.flags(nloc);
            if (cd.first) {
                ++cd.seg;
                const int sg = cd.seg - 1;
                if (!mbar_wait(&bars[BAR_AFULL + (P.a_bufs == 2 ? (sg & 1) : 0)],
                               uint32_t((P.a_bufs == 2 ? (sg >> 1) : sg) & 1), abort_flag, P.wait, P.status, 3))
                    break;
            }
            if (!mbar_wait(&bars[BAR_FULL + cd.stage], cd.sphase, abort_flag, P.wait, P.status, 4)) break;
            // buffer db is free once the product of tile loc - ND completed
            if (cd.loc >= ND && !mbar_wait(&bars[BAR_KFREE + cd.db], cd.dphase ^ 1u, abort_flag, P.wait, P.status, 10))
                break;
            tc_fence_after();
            const int abuf = P.a_bufs == 2 ? ((cd.seg - 1) & 1) : 0;
            const uint32_t a_lo = a_lo0 + uint32_t(abuf) * a_units;
            const uint32_t b_lo = b_lo0 + uint32_t(cd.stage) * stage_units;
            const uint32_t d_tmem = tmem + uint32_t(P.dist_col0 + cd.db * kBN);
            mma_ss_w(d_tmem, a_lo, b_lo, P.ab_hi, idesc_d, 0u);
#pragma unroll 1
            for (int k = 1; k < P.kmma; ++k) {
                const uint32_t off = uint32_t(k >> 2) * (P.chunk_bytes >> 4) + uint32_t((k & 3) * 2);
                mma_ss_w(d_tmem, a_lo + off, b_lo + off, P.ab_hi, idesc_d, 1u);
            }
            tc_commit(&bars[BAR_DFULL + cd.db]);
            if (cd.last) tc_commit(&bars[BAR_AEMPTY + abuf]);
        }
        tc_commit(&bars[BAR_DRAIN2]);
        mbar_wait_bounded(&bars[BAR_DRAIN2], 0, kWaitBudget);
    } else if (TWO && warp == 3 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ product MMA issuer
        const uint32_t idesc_p = idesc_f16_f32(kBM, P.r);
        const uint32_t r_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_stage + a_bytes));
        const uint32_t stage_units = P.stage_bytes >> 4;
        const uint32_t rbox_units = uint32_t(P.r * 128) >> 4;
        Cursor cp;
        cp.init(P, t0, nct);
        for (; cp.loc < nloc; cp.next(P, nloc, NS, ND)) {
            cp.flags(nloc);
            if (cp.first) {
                const int seg = cp.seg++;
                const uint32_t par = P.s_bufs == 2 ? uint32_t((seg >> 1) & 1) : uint32_t(seg & 1);
                if (!mbar_wait(&bars[BAR_SEMPTY + (P.s_bufs == 2 ? (seg & 1) : 0)], par ^ 1u, abort_flag,
                               P.wait, P.status, 5))
                    break;
            }
            const int sb = P.s_bufs == 2 ? ((cp.seg - 1) & 1) : 0;
            if (!mbar_wait(&bars[BAR_PFULL + cp.db], cp.dphase, abort_flag, P.wait, P.status, 6)) break;
            tc_fence_after();
            const uint32_t r_lo = r_lo0 + uint32_t(cp.stage) * stage_units;
            const uint32_t s_tmem = tmem + uint32_t(sb * P.r);
            const uint32_t p_tmem = tmem + uint32_t(P.dist_col0 + cp.db * kBN);
            mma_ts_w(s_tmem, p_tmem, r_lo, kSdescHiSw128, idesc_p, cp.first ? 0u : 1u);
#pragma unroll
            for (int k = 1; k < 8; ++k)
                mma_ts_w(s_tmem, p_tmem + uint32_t((k >> 2) * 64 + (k & 3) * 8),
                         r_lo + uint32_t(k >> 2) * rbox_units + uint32_t((k & 3) * 2), kSdescHiSw128, idesc_p, 1u);
            if (P.split_k) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    mma_ts_w(s_tmem, p_tmem + uint32_t((k >> 2) * 64 + 32 + (k & 3) * 8),
                             r_lo + uint32_t(k >> 2) * rbox_units + uint32_t((k & 3) * 2), kSdescHiSw128, idesc_p,
                             1u);
            }
            if (PAIR) tc_commit_mc(&bars[BAR_EMPTY + cp.stage], uint16_t(3));
            else tc_commit(&bars[BAR_EMPTY + cp.stage]);
            tc_commit(&bars[BAR_KFREE + cp.db]);
            if (cp.last) tc_commit(&bars[BAR_SFULL + sb]);
        }
        tc_commit(&bars[BAR_DRAIN]);
        mbar_wait_bounded(&bars[BAR_DRAIN], 0, kWaitBudget);
    } else if (!TWO && warp == 1 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ MMA issuer
        // The distance GEMM of tile loc + ND - 1 is issued before waiting for
        // the epilogue of tile loc, so the tensor core always has the next
        // distances queued.  MMAs from this thread execute in issue order,
        // so a distance buffer is rewritten only after the product that
        // read its K values.
        const uint32_t idesc_d = idesc_f16_f32(kBM, kBN);
        const uint32_t idesc_p = idesc_f16_f32(kBM, P.r);
        // descriptor low words of buffer 0 / stage 0 and the strides between
        // buffers (16-byte units): each MMA then costs one 32-bit add
        const uint32_t a_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_a));
        const uint32_t b_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_stage));
        const uint32_t r_lo0 = sdesc_lo_sw128(smem_u32(smem + P.off_stage + a_bytes));
        const uint32_t a_units = a_bytes >> 4, stage_units = P.stage_bytes >> 4;
        const uint32_t rbox_units = uint32_t(P.r * 128) >> 4;  // second 64-row box of the R tile
        Cursor cd, cp;  // distance-side and product-side positions
        cd.init(P, t0, nct);
        cp.init(P, t0, nct);
        bool ok = true;
        auto issue_dist = [&]() -> bool {
            cd.flags(nloc);
            if (cd.first) {
                ++cd.seg;
                const int sg = cd.seg - 1;
                if (!mbar_wait(&bars[BAR_AFULL + (P.a_bufs == 2 ? (sg & 1) : 0)],
                               uint32_t((P.a_bufs == 2 ? (sg >> 1) : sg) & 1), abort_flag,
                               P.wait, P.status, 3))
                    return false;
            }
            if (!mbar_wait(&bars[BAR_FULL + cd.stage], cd.sphase, abort_flag, P.wait, P.status, 4)) return false;
            tc_fence_after();
            const int abuf = P.a_bufs == 2 ? ((cd.seg - 1) & 1) : 0;
            const uint32_t a_lo = a_lo0 + uint32_t(abuf) * a_units;
            const uint32_t b_lo = b_lo0 + uint32_t(cd.stage) * stage_units;
            const uint32_t d_tmem = tmem + uint32_t(P.dist_col0 + cd.db * kBN);
            mma_ss_w(d_tmem, a_lo, b_lo, P.ab_hi, idesc_d, 0u);
#pragma unroll 1
            for (int k = 1; k < P.kmma; ++k) {
                // 32 bytes per 16-element K step inside a chunk (a 32-element
                // chunk has at most two steps, so k >> 2 is 0 there)
                const uint32_t off = uint32_t(k >> 2) * (P.chunk_bytes >> 4) + uint32_t((k & 3) * 2);
                mma_ss_w(d_tmem, a_lo + off, b_lo + off, P.ab_hi, idesc_d, 1u);
            }
            tc_commit(&bars[BAR_DFULL + cd.db]);
            if (cd.last) tc_commit(&bars[BAR_AEMPTY + abuf]);
            cd.next(P, nloc, NS, ND);
            return true;
        };
        for (int k = 0; ok && k < ND - 1 && k < nloc; ++k) ok = issue_dist();
        for (; ok && cp.loc < nloc; cp.next(P, nloc, NS, ND)) {
            if (cd.loc < nloc && !issue_dist()) break;
            cp.flags(nloc);
            if (cp.first) {
                const int seg = cp.seg++;
                const uint32_t par = P.s_bufs == 2 ? uint32_t((seg >> 1) & 1) : uint32_t(seg & 1);
                if (!mbar_wait(&bars[BAR_SEMPTY + (P.s_bufs == 2 ? (seg & 1) : 0)], par ^ 1u, abort_flag,
                               P.wait, P.status, 5))
                    break;
            }
            const int sb = P.s_bufs == 2 ? ((cp.seg - 1) & 1) : 0;
            if (!mbar_wait(&bars[BAR_PFULL + cp.db], cp.dphase, abort_flag, P.wait, P.status, 6)) break;
            tc_fence_after();
            const uint32_t r_lo = r_lo0 + uint32_t(cp.stage) * stage_units;
            const uint32_t s_tmem = tmem + uint32_t(sb * P.r);
            const uint32_t p_tmem = tmem + uint32_t(P.dist_col0 + cp.db * kBN);
            // K of warpgroup k/4 sits in its first 32 columns, 8 columns per 16 K;
            // R rows of K step k: box k/4, 32 bytes per step inside the box
            mma_ts_w(s_tmem, p_tmem, r_lo, kSdescHiSw128, idesc_p, cp.first ? 0u : 1u);
#pragma unroll
            for (int k = 1; k < 8; ++k)
                mma_ts_w(s_tmem, p_tmem + uint32_t((k >> 2) * 64 + (k & 3) * 8),
                         r_lo + uint32_t(k >> 2) * rbox_units + uint32_t((k & 3) * 2), kSdescHiSw128, idesc_p, 1u);
            if (P.split_k) {
                // K_lo sits 32 columns after K_hi
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    mma_ts_w(s_tmem, p_tmem + uint32_t((k >> 2) * 64 + 32 + (k & 3) * 8),
                             r_lo + uint32_t(k >> 2) * rbox_units + uint32_t((k & 3) * 2), kSdescHiSw128, idesc_p,
                             1u);
            }
            if (PAIR) tc_commit_mc(&bars[BAR_EMPTY + cp.stage], uint16_t(3));
            else tc_commit(&bars[BAR_EMPTY + cp.stage]);
            if (cp.last) tc_commit(&bars[BAR_SFULL + sb]);
        }
        // Drain: every MMA issued has completed before tensor memory is freed.
        tc_commit(&bars[BAR_DRAIN]);
        mbar_wait_bounded(&bars[BAR_DRAIN], 0, kWaitBudget);
    } else if (warp >= 4 && nloc > 0) {
        // ------------------------------------------------ epilogue
        // Warpgroup g owns columns [64 g, 64 g + 64) of every tile, read as
        // two 32-column chunks; thread (warp quarter q, lane) owns row
        // 32 q + lane.  The tensor-memory load of chunk 1 is in flight while
        // chunk 0 is exponentiated, and the next tile's chunk 0 is requested
        // right after this tile's K is handed over.  K for chunk k is written
        // (FP16 pairs) into columns [64 g + 16 k, +16), already read.
        const int q = warp & 3;
        const int g = (warp - 4) >> 2;
        const uint32_t lane_off = uint32_t(32 * q) << 16;
        const int rh = P.r >> 1;
        Cursor c;
        c.init(P, t0, nct);
        uint32_t va[32], vb[32];
        bool ok = warp_wait(&bars[BAR_DFULL + 0], 0u, abort_flag, P.wait, P.status, 7);
        if (ok) {
            tc_fence_after();
            tmem_ld32(tmem + lane_off + uint32_t(P.dist_col0 + 64 * g), va);
        }
        bool seg_whole = false;  // the current segment began at its row tile's first column tile
        for (; ok && c.loc < nloc; c.next(P, nloc, 1, ND)) {
            c.flags(nloc);
            if (c.first) {
                ++c.seg;
                seg_whole = c.ct == c.lo;
            }
            const uint32_t base = tmem + lane_off + uint32_t(P.dist_col0 + c.db * kBN + 64 * g);
            const int rt = row_tile(c.rt);
            const int64_t i = int64_t(rt) * kBM + 32 * q + lane;
            uint32_t mlo = 0, mhi = 0;
            if ((P.leaf_a != nullptr || P.grp_a != nullptr) && int64_t(rt) * kBM < P.ma)
                tile_mask(P, rt, c.ct, g, i, mlo, mhi);
            tmem_wait_ld_regs(va);                 // chunk 0 of this tile
            tmem_ld32(base + 32, vb);              // chunk 1 in flight
            uint32_t pk[16];
            if (!P.split_k) {
                exp_pack(va, pk);
                if (mlo) mask_pack(pk, mlo);
                tmem_st16(base, pk);
                tmem_wait_ld_regs(vb);             // chunk 1 of this tile
                exp_pack(vb, pk);
                if (mhi) mask_pack(pk, mhi);
                tmem_st16(base + 16, pk);
            } else {
                // K_hi of chunk k -> columns [16 k, +16), K_lo -> [32 + 16 k, +16)
                uint32_t pl[16];
                exp_pack_split(va, pk, pl);
                if (mlo) { mask_pack(pk, mlo); mask_pack(pl, mlo); }
                tmem_st16(base, pk);
                tmem_wait_ld_regs(vb);             // chunk 1 read: its columns are free
                tmem_st16(base + 32, pl);
                exp_pack_split(vb, pk, pl);
                if (mhi) { mask_pack(pk, mhi); mask_pack(pl, mhi); }
                tmem_st16(base + 16, pk);
                tmem_st16(base + 48, pl);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[BAR_PFULL + c.db]);
            // K of this tile is handed over before waiting for the next
            // tile's distances, so the MMA issuer never waits on that wait.
            if (c.loc + 1 < nloc) {
                const int nd = c.db + 1 == ND ? 0 : c.db + 1;
                const uint32_t np = c.db + 1 == ND ? (c.dphase ^ 1u) : c.dphase;
                if (!warp_wait(&bars[BAR_DFULL + nd], np, abort_flag, P.wait, P.status, 7))
                    ok = false;
                else {
                    tc_fence_after();
                    tmem_ld32(tmem + lane_off + uint32_t(P.dist_col0 + nd * kBN + 64 * g), va);
                }
            }
            if (c.last) flush_s(P, bars, abort_flag, tmem, lane_off, c.seg - 1, g, rh, i, seg_whole && c.ct == c.hi);
        }
        tmem_wait_ld();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem, 512);
    if (PAIR) cluster_sync();  // neither CTA exits while the other may still signal it
}

}  // namespace tc

// ------------------------------------------------------------------ host
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D FP16 tensor map: `cols` contiguous elements per row (row stride
// ld_elems), box of box_cols x box_rows with the 128-byte swizzle (or the
// 64-byte one for 32-element boxes).
int make_map(CUtensorMap *m, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_cols,
             int box_rows, bool swizzle64 = false) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return fail(KRR_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld_elems * 2)};
    cuuint32_t box[2] = {cuuint32_t(box_cols), cuuint32_t(box_rows)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(KRR_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
    return KRR_OK;
}

// One launch of variant v (bit 1: pairs of row tiles in clusters of two
// CTAs, bit 0: two MMA-issuing threads); P describes single row tiles.
int launch_variant(Ctx *c, int v, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mR, tc::Params P,
                   size_t smem, const __half *XB, int kpad, int box_k, int64_t nb, bool narrow) {
    const bool pair = (v & 2) != 0, two = (v & 1) != 0;
    auto kernel = pair ? (two ? tc::sample_tc_kernel<true, true> : tc::sample_tc_kernel<true, false>)
                       : (two ? tc::sample_tc_kernel<false, true> : tc::sample_tc_kernel<false, false>);
    static SmemLimitOnce smem_limit[4];
    KRR_CUDA(raise_smem_limit(smem_limit[v & 3], c->device, kernel, 227 * 1024));
    if (!pair) {
        const int64_t T = P.n_tiles;
        const int grid = int(T < c->num_sms ? T : c->num_sms);
        { kernel<<<grid, tc::kThreads, smem, c->stream>>>(mA, mB, mR, P); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        return KRR_OK;
    }
    CUtensorMap mBh;
    KRR_TRY(make_map(&mBh, XB, kpad, nb, kpad, box_k, tc::kBN / 2, narrow));  // half-tile boxes
    P.n_row_tiles = cdiv(P.n_row_tiles, 2);  // row units of two row tiles
    P.n_tiles = P.n_row_tiles * P.n_col_tiles;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(tc::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // clusters that can be resident at once (one CTA per SM), per device
    static std::atomic<int> max_clusters[kMaxDevices][2];
    const bool cached = c->device >= 0 && c->device < kMaxDevices;
    int mc = cached ? max_clusters[c->device][two ? 1 : 0].load() : 0;
    if (mc <= 0) {
        cfg.gridDim = dim3(2 * (c->num_sms / 2));
        KRR_CUDA(cudaOccupancyMaxActiveClusters(&mc, kernel, &cfg));
        if (mc <= 0) return fail(KRR_ERR_CUDA, "sample_tc: no cluster of two CTAs fits on the device");
        if (cached) max_clusters[c->device][two ? 1 : 0].store(mc);
    }
    const int64_t units = P.n_tiles < mc ? P.n_tiles : mc;
    cfg.gridDim = dim3(unsigned(2 * units));
    KRR_CUDA(cudaLaunchKernelEx(&cfg, kernel, mA, mBh, mR, P));
    ::krr::count_launch();
    return KRR_OK;
}

// The fused product's autotuner: a shape class (device, feature chunks,
// narrow rows, column width, split K, leaf masks, log2 of the tile count)
// maps to the fastest variant measured on its first launch.  Each trial
// clears this launch's block of S, runs one variant and times it with CUDA
// events; the winner runs last, so S holds its result.
struct TuneKey {
    int device, nchunk, narrow, rpad, split_k, masked, tiles_log2;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, nchunk, narrow, rpad, split_k, masked, tiles_log2) <
               std::tie(o.device, o.nchunk, o.narrow, o.rpad, o.split_k, o.masked, o.tiles_log2);
    }
};

int tune_variant(Ctx *c, const CUtensorMap &mA, const CUtensorMap &mB, const CUtensorMap &mR, const tc::Params &P,
                 size_t smem, const __half *XB, int kpad, int box_k, int64_t nb, bool narrow, bool pair_ok, float *S,
                 int64_t lds, int &variant) {
    static std::mutex mu;
    static std::map<TuneKey, int> cache;
    int tl = 0;
    for (int64_t t = P.n_tiles; t > 1; t >>= 1) ++tl;
    const TuneKey key{c->device, P.nchunk, narrow ? 1 : 0, P.r, P.split_k, P.leaf_a != nullptr ? 1 : 0, tl};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            variant = it->second;
            return KRR_OK;
        }
    }
    cudaEvent_t e0, e1;
    KRR_CUDA(cudaEventCreate(&e0));
    KRR_CUDA(cudaEventCreate(&e1));
    int best = variant;
    float best_ms = 0.f;
    for (int v = pair_ok ? 3 : 1; v >= 0; --v) {
        KRR_CUDA(cudaMemset2DAsync(S, size_t(lds) * 4, 0, size_t(P.r_valid) * 4, size_t(P.ma), c->stream));
        KRR_CUDA(cudaEventRecord(e0, c->stream));
        const int st = launch_variant(c, v, mA, mB, mR, P, smem, XB, kpad, box_k, nb, narrow);
        if (st != KRR_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        KRR_CUDA(cudaEventRecord(e1, c->stream));
        KRR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        KRR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (v == (pair_ok ? 3 : 1) || ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KRR_CUDA(cudaMemset2DAsync(S, size_t(lds) * 4, 0, size_t(P.r_valid) * 4, size_t(P.ma), c->stream));
    variant = best;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return KRR_OK;
}

}  // namespace

// S (+)= W o K(XA rows, XB rows) RT^T, accumulated atomically into S
// (which the caller zeroes).  XA, XB: augmented FP16 rows (Kpad = 64 *
// nchunk elements each, or 32 when nchunk = 1 and kmma <= 2: the rows of
// d <= 8); RT: FP16, rpad x ldrt (row c = column c of R).
int launch_sample_tc(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int nchunk, int kmma,
                     const __half *RT, int rpad, int64_t ldrt, int r_valid, const int32_t *leaf_a,
                     const int32_t *leaf_b, float *S, int64_t lds, bool split_k, const BlockDiag *bd) {
    if ((rpad % 64 != 0 && rpad != 32) || rpad < 32 || rpad > 256)
        return fail(KRR_ERR_INVALID_ARG, "sample_tc: r must be 32, or 64..256 in steps of 64");
    if (nchunk < 1 || nchunk > 4) return fail(KRR_ERR_INVALID_ARG, "sample_tc: feature dimension too large");
    if (ma <= 0 || nb <= 0) return KRR_OK;
    if (ldrt % 8 != 0) return fail(KRR_ERR_INVALID_ARG, "sample_tc: ldrt must be a multiple of 8");
    CUtensorMap mA, mB, mR;
    const bool narrow = nchunk == 1 && kmma <= 2;
    const int kpad = narrow ? 32 : 64 * nchunk, box_k = narrow ? 32 : 64;
    KRR_TRY(make_map(&mA, XA, kpad, ma, kpad, box_k, tc::kBM, narrow));
    KRR_TRY(make_map(&mB, XB, kpad, nb, kpad, box_k, tc::kBN, narrow));
    KRR_TRY(make_map(&mR, RT, nb, rpad, ldrt, 64, rpad));

    tc::Params P{};
    P.ma = ma;
    P.nb = nb;
    P.n_row_tiles = cdiv(ma, tc::kBM);
    P.n_col_tiles = cdiv(nb, tc::kBN);
    P.r = rpad;
    P.r_valid = r_valid;
    P.split_k = split_k ? 1 : 0;
    P.nchunk = nchunk;
    P.kmma = kmma;
    // Tensor memory (512 columns): S accumulators first, then 128-column
    // distance / K buffers.
    P.s_bufs = (2 * rpad <= 128) ? 2 : 1;
    P.dist_col0 = P.s_bufs * rpad;
    if (P.dist_col0 < 128) P.dist_col0 = 128;
    P.ndist = (512 - P.dist_col0) / 128;
    if (P.ndist > 3) P.ndist = 3;
    P.chunk_bytes = narrow ? tc::kChunkBytes / 2 : tc::kChunkBytes;
    P.ab_hi = narrow ? ptx::kSdescHiSw64 : ptx::kSdescHiSw128;
    const uint32_t a_bytes = nchunk * P.chunk_bytes;
    P.stage_bytes = a_bytes + 2 * rpad * 128;
    const int budget = 227 * 1024 - 1024 - 256;  // alignment slack + barriers
    // two row-tile buffers (the next row tile loads while the current one
    // is in use), unless a single buffer makes room for a third stage
    const int ns2 = int((budget - 2 * int(a_bytes)) / int(P.stage_bytes));
    const int ns1 = int((budget - int(a_bytes)) / int(P.stage_bytes));
    P.a_bufs = (ns2 >= 3 || (ns2 >= 2 && ns1 == ns2)) ? 2 : 1;
    P.off_a = 0;
    P.off_stage = P.a_bufs * a_bytes;
    int ns = int((budget - int(P.off_stage)) / int(P.stage_bytes));
    if (ns > tc::kMaxStages) ns = tc::kMaxStages;
    if (ns < 2) return fail(KRR_ERR_INVALID_ARG, "sample_tc: tile does not fit in shared memory");
    P.nstage = ns;
    // The issuer runs the distance GEMM ndist - 1 tiles ahead of the
    // product, so those tiles' stages must all be resident at once.
    if (P.ndist > ns) P.ndist = ns;
    P.off_bar = P.off_stage + ns * P.stage_bytes;
    size_t smem = size_t(P.off_bar) + tc::BAR_COUNT * 8 + 16 + 1024;
    // The kernel allocates all 512 tensor-memory columns, so two CTAs must
    // never share an SM: asking for more than half of the SM's shared
    // memory guarantees that.
    if (smem < 120 * 1024) smem = 120 * 1024;
    P.leaf_a = leaf_a;
    P.leaf_b = leaf_b;
    P.n_tiles = P.n_row_tiles * P.n_col_tiles;
    if (bd) {
        P.grp_a = bd->grp_a;
        P.grp_b = bd->grp_b;
        P.tl_lo = bd->tl_lo;
        P.tl_hi = bd->tl_hi;
        P.tl_off = bd->tl_off;
        P.n_tiles = bd->tiles;
    }
    P.S = S;
    P.lds = lds;
    P.status = c->status;
    P.wait = c->wait_cycles;

    if (P.n_tiles <= 0) return KRR_OK;
    // Variant: pairs of row tiles sharing every column tile's loads
    // (clusters of two CTAs, multicast; not for block-diagonal tile lists)
    // and one or two MMA-issuing threads.  Rules measured on GB300: pairs
    // whenever allowed; two issuers where each tile's MMAs are small
    // (+22 % at r = 64, 5 % slower at r = 256).  With the context's
    // autotuner on, the first launch of a shape class times every allowed
    // variant on this very call and caches the fastest per device.
    const bool pair_ok = bd == nullptr && P.n_row_tiles >= 2;
    int variant = (pair_ok ? 2 : 0) + ((rpad <= 128 || split_k) ? 1 : 0);
#ifdef KRR_PAIR_OFF
    variant &= 1;
#endif
    if (c->autotune && bd == nullptr) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        KRR_CUDA(cudaStreamIsCapturing(c->stream, &cs));
        if (cs == cudaStreamCaptureStatusNone) KRR_TRY(tune_variant(c, mA, mB, mR, P, smem, XB, kpad, box_k, nb,
                                                                    narrow, pair_ok, S, lds, variant));
    }
    return launch_variant(c, variant, mA, mB, mR, P, smem, XB, kpad, box_k, nb, narrow);
}

}  // namespace krr
