// Fused Gaussian-kernel x block product for wide feature rows (augmented
// rows longer than four 64-element chunks, d > 82), on sm_103a tensor cores.
//
// Same operation, operands and epilogue as the resident-row kernel in
// sample_tc.cu: per 128 x 128 tile a distance GEMM on tcgen05 gives
// log2 K_ij in tensor memory, the epilogue warps form K = 2^e in FP16 back
// into tensor memory, and K times the tile's rows of R accumulates S in
// tensor memory.  What differs is the feeding of the distance GEMM: the
// augmented rows (3d + 6 FP16 elements) no longer fit in shared memory as
// a resident row tile, so every tile streams its A and B rows through a
// ring of stages, one 64-element chunk of each per stage (32 KB), and the
// R tile of the step comes through a separate ring of two buffers.  The
// A chunks are re-read for every column tile (from L2: a row tile of the
// augmented operand is 128 x (3d + 6) FP16).
//
// Warp roles as in the resident kernel (384 threads, one CTA per SM,
// persistent over a contiguous range of tile steps or a block-diagonal
// tile list): warp 0 issues TMA loads, warp 1 issues tcgen05.mma, warp 2
// owns the tensor memory, warps 4-11 run the epilogue.
#include <cuda.h>

#include "common.cuh"
#include "prep.cuh"
#include "tc_ptx.cuh"

namespace krr {
namespace tcw {

constexpr int kThreads = 384;
constexpr int kBM = 128;             // rows of a tile (tensor-memory lanes)
constexpr int kBN = 128;             // K columns of a tile
constexpr int kChunk = 64;           // FP16 elements per 128-byte swizzled row
constexpr int kChunkBytes = 128 * 128;
constexpr int kMaxStages = 6;
constexpr long long kWaitBudget = kDefaultWaitCycles;  // drain waits at kernel exit

static_assert(kBM == kTcTile && kBN == kTcTile, "tile lists assume square 128-row tiles");
constexpr int kStageBytes = 2 * kChunkBytes;  // one 64-element chunk of the A and the B tile
constexpr int kRBufs = 2;                       // R tiles in flight

struct Params {
    int64_t ma, nb;
    int64_t n_row_tiles, n_col_tiles;
    int r;        // R / S columns handled by this launch (multiple of 64, <= 256)
    int r_valid;  // columns actually stored (<= r)
    int nchunk;   // 64-element chunks of an augmented row
    int kmma;     // K=16 MMA steps of the distance GEMM
    int nstage;
    int s_bufs;   // S accumulators in tensor memory (1 or 2)
    int ndist;    // distance / K buffers in tensor memory (2 or 3)
    int dist_col0;
    int split_k;  // 1: K = K_hi + K_lo (two FP16 parts, two product MMAs)
    uint32_t off_stage, off_r, r_bytes, off_bar;  // chunk stages, R tile ring, barriers
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
    BAR_RFULL = BAR_EMPTY + kMaxStages,
    BAR_REMPTY = BAR_RFULL + kRBufs,
    BAR_DFULL = BAR_REMPTY + kRBufs,
    BAR_PFULL = BAR_DFULL + 3,
    BAR_SFULL = BAR_PFULL + 3,
    BAR_SEMPTY = BAR_SFULL + 2,
    BAR_DRAIN = BAR_SEMPTY + 2,
    BAR_COUNT = BAR_DRAIN + 1
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
__device__ __forceinline__ void flush_s(const Params &P, uint64_t *bars, volatile int *abort_flag, uint32_t tmem,
                                     uint32_t lane_off, int64_t seg, int g, int rh, int64_t i) {
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
            for (int c = 0; c < 32; ++c)
                if (cbase + c < P.r_valid) atomicAdd(dst + cbase + c, __uint_as_float(sv[c]));
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

__global__ void __launch_bounds__(kThreads, 1)
    sample_tc_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
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
    const int64_t t0 = T * blockIdx.x / gridDim.x;
    const int nloc = int(T * (blockIdx.x + 1) / gridDim.x - t0);
    const int NS = P.nstage, ND = P.ndist;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[BAR_FULL + s], 1);
            mbar_init(&bars[BAR_EMPTY + s], 1);
        }
        for (int b = 0; b < kRBufs; ++b) {
            mbar_init(&bars[BAR_RFULL + b], 1);
            mbar_init(&bars[BAR_REMPTY + b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars[BAR_SFULL + b], 1);
            mbar_init(&bars[BAR_SEMPTY + b], 8);
        }
        for (int b = 0; b < 3; ++b) {
            mbar_init(&bars[BAR_DFULL + b], 1);
            mbar_init(&bars[BAR_PFULL + b], 8);
        }
        mbar_init(&bars[BAR_DRAIN], 1);
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
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ TMA producer
        // per tile: its nchunk (A chunk, B chunk) stages, then its R tile
        Cursor c;
        c.init(P, t0, nct);
        int st = 0, issued = 0, rb = 0, r_issued = 0;
        uint32_t sph = 0, rph = 0;
        bool ok = true;
        for (; ok && c.loc < nloc; c.next(P, nloc, 1, 1)) {
            for (int ch = 0; ch < P.nchunk; ++ch) {
                if (!mbar_wait(&bars[BAR_EMPTY + st], sph ^ 1u, abort_flag, P.wait, P.status, 1)) {
                    ok = false;
                    break;
                }
                uint8_t *sp = smem + P.off_stage + st * kStageBytes;
                mbar_expect_tx(&bars[BAR_FULL + st], kStageBytes);
                tma_load_2d(sp, &tmA, &bars[BAR_FULL + st], ch * kChunk, c.rt * kBM);
                tma_load_2d(sp + kChunkBytes, &tmB, &bars[BAR_FULL + st], ch * kChunk, c.ct * kBN);
                ++issued;
                if (++st == NS) {
                    st = 0;
                    sph ^= 1u;
                }
            }
            if (!ok) break;
            if (!mbar_wait(&bars[BAR_REMPTY + rb], rph ^ 1u, abort_flag, P.wait, P.status, 2)) break;
            uint8_t *rp = smem + P.off_r + rb * P.r_bytes;
            mbar_expect_tx(&bars[BAR_RFULL + rb], P.r_bytes);
            tma_load_2d(rp, &tmR, &bars[BAR_RFULL + rb], c.ct * kBN, 0);
            tma_load_2d(rp + P.r * 128, &tmR, &bars[BAR_RFULL + rb], c.ct * kBN + 64, 0);
            ++r_issued;
            if (++rb == kRBufs) {
                rb = 0;
                rph ^= 1u;
            }
        }
        // Drain: wait (bounded) until every load issued has landed, so no
        // TMA write is in flight when the CTA exits.
        for (int k = 0; k < (issued < NS ? issued : NS); ++k) {
            const int u = issued - 1 - k;
            mbar_wait_bounded(&bars[BAR_FULL + (u % NS)], uint32_t((u / NS) & 1), kWaitBudget);
        }
        for (int k = 0; k < (r_issued < kRBufs ? r_issued : kRBufs); ++k) {
            const int u = r_issued - 1 - k;
            mbar_wait_bounded(&bars[BAR_RFULL + (u % kRBufs)], uint32_t((u / kRBufs) & 1), kWaitBudget);
        }
    } else if (warp == 1 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ MMA issuer
        // The distance GEMM of tile loc + ND - 1 is issued before waiting
        // for the epilogue of tile loc.  A chunk stage is released when the
        // MMAs that read it complete; the R tile after the product.
        const uint32_t idesc_d = idesc_f16_f32(kBM, kBN);
        const uint32_t idesc_p = idesc_f16_f32(kBM, P.r);
        Cursor cd, cp;
        cd.init(P, t0, nct);
        cp.init(P, t0, nct);
        int st = 0, rb = 0;
        uint32_t sph = 0, rph = 0;
        bool ok = true;
        auto issue_dist = [&]() -> bool {
            cd.flags(nloc);
            const uint32_t d_tmem = tmem + uint32_t(P.dist_col0 + cd.db * kBN);
            for (int ch = 0; ch < P.nchunk; ++ch) {
                if (!mbar_wait(&bars[BAR_FULL + st], sph, abort_flag, P.wait, P.status, 4)) return false;
                tc_fence_after();
                const uint32_t a_base = smem_u32(smem + P.off_stage + st * kStageBytes);
                const uint32_t b_base = a_base + kChunkBytes;
                for (int kk = 0; kk < 4; ++kk) {
                    const int k = ch * 4 + kk;
                    if (k >= P.kmma) break;
                    mma_ss(d_tmem, sdesc_k_sw128(a_base + kk * 32), sdesc_k_sw128(b_base + kk * 32), idesc_d,
                           k > 0 ? 1u : 0u);
                }
                tc_commit(&bars[BAR_EMPTY + st]);
                if (++st == NS) {
                    st = 0;
                    sph ^= 1u;
                }
            }
            tc_commit(&bars[BAR_DFULL + cd.db]);
            cd.next(P, nloc, 1, ND);
            return true;
        };
        for (int k = 0; ok && k < ND - 1 && k < nloc; ++k) ok = issue_dist();
        for (; ok && cp.loc < nloc; cp.next(P, nloc, 1, ND)) {
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
            if (!mbar_wait(&bars[BAR_RFULL + rb], rph, abort_flag, P.wait, P.status, 9)) break;
            tc_fence_after();
            const uint32_t r_base = smem_u32(smem + P.off_r + rb * P.r_bytes);
            const uint32_t s_tmem = tmem + uint32_t(sb * P.r);
            const uint32_t p_tmem = tmem + uint32_t(P.dist_col0 + cp.db * kBN);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                // K of warpgroup k/4 sits in its first 32 columns, 8 columns per 16 K
                const uint32_t a_t = p_tmem + uint32_t((k >> 2) * 64 + (k & 3) * 8);
                const uint32_t roff = uint32_t((k >> 2) * P.r * 128 + (k & 3) * 32);
                mma_ts(s_tmem, a_t, sdesc_k_sw128(r_base + roff), idesc_p, (cp.first && k == 0) ? 0u : 1u);
            }
            if (P.split_k) {
                // K_lo sits 32 columns after K_hi
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t a_t = p_tmem + uint32_t((k >> 2) * 64 + 32 + (k & 3) * 8);
                    const uint32_t roff = uint32_t((k >> 2) * P.r * 128 + (k & 3) * 32);
                    mma_ts(s_tmem, a_t, sdesc_k_sw128(r_base + roff), idesc_p, 1u);
                }
            }
            tc_commit(&bars[BAR_REMPTY + rb]);
            if (++rb == kRBufs) {
                rb = 0;
                rph ^= 1u;
            }
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
        for (; ok && c.loc < nloc; c.next(P, nloc, 1, ND)) {
            c.flags(nloc);
            if (c.first) ++c.seg;
            const uint32_t base = tmem + lane_off + uint32_t(P.dist_col0 + c.db * kBN + 64 * g);
            const int64_t i = int64_t(c.rt) * kBM + 32 * q + lane;
            uint32_t mlo = 0, mhi = 0;
            if (P.leaf_a != nullptr || P.grp_a != nullptr) tile_mask(P, c.rt, c.ct, g, i, mlo, mhi);
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
            if (c.last) flush_s(P, bars, abort_flag, tmem, lane_off, c.seg - 1, g, rh, i);
        }
        tmem_wait_ld();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem, 512);
}

}  // namespace tcw

// ------------------------------------------------------------------ host
namespace {

typedef CUresult (*EncodeTiledFnW)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFnW encode_fn_w() {
    static EncodeTiledFnW fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFnW>(p);
    }
    return fn;
}

// 2-D FP16 tensor map with the 128-byte swizzle (see sample_tc.cu)
int make_map_w(CUtensorMap *m, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_cols,
               int box_rows) {
    EncodeTiledFnW fn = encode_fn_w();
    if (!fn) return fail(KRR_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld_elems * 2)};
    cuuint32_t box[2] = {cuuint32_t(box_cols), cuuint32_t(box_rows)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(KRR_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
    return KRR_OK;
}

}  // namespace

// S (+)= W o K(XA rows, XB rows) RT^T for augmented rows of any number of
// 64-element chunks (see launch_sample_tc for the arguments).
int launch_sample_tc_wide(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int nchunk, int kmma,
                          const __half *RT, int rpad, int64_t ldrt, int r_valid, const int32_t *leaf_a,
                          const int32_t *leaf_b, float *S, int64_t lds, bool split_k, const BlockDiag *bd) {
    if (rpad % 64 != 0 || rpad < 64 || rpad > 128) return fail(KRR_ERR_INVALID_ARG, "sample_tc_wide: r must be 64 or 128");
    if (nchunk < 1 || kmma < 1 || kmma > 4 * nchunk) return fail(KRR_ERR_INVALID_ARG, "sample_tc_wide: bad chunks");
    if (ma <= 0 || nb <= 0) return KRR_OK;
    if (ldrt % 8 != 0) return fail(KRR_ERR_INVALID_ARG, "sample_tc_wide: ldrt must be a multiple of 8");
    CUtensorMap mA, mB, mR;
    const int kpad = 64 * nchunk;
    KRR_TRY(make_map_w(&mA, XA, kpad, ma, kpad, 64, tcw::kBM));
    KRR_TRY(make_map_w(&mB, XB, kpad, nb, kpad, 64, tcw::kBN));
    KRR_TRY(make_map_w(&mR, RT, nb, rpad, ldrt, 64, rpad));

    tcw::Params P{};
    P.ma = ma;
    P.nb = nb;
    P.n_row_tiles = cdiv(ma, tcw::kBM);
    P.n_col_tiles = cdiv(nb, tcw::kBN);
    P.r = rpad;
    P.r_valid = r_valid;
    P.split_k = split_k ? 1 : 0;
    P.nchunk = nchunk;
    P.kmma = kmma;
    // Tensor memory (512 columns): S accumulators first, then 128-column
    // distance / K buffers (at most 3; the R ring of two buffers keeps the
    // issuer's lead of ndist - 1 tiles free of deadlock).
    P.s_bufs = (2 * rpad <= 128) ? 2 : 1;
    P.dist_col0 = P.s_bufs * rpad;
    if (P.dist_col0 < 128) P.dist_col0 = 128;
    P.ndist = (512 - P.dist_col0) / 128;
    if (P.ndist > 3) P.ndist = 3;
    P.r_bytes = uint32_t(2 * rpad * 128);
    const int budget = 227 * 1024 - 1024 - 256;  // alignment slack + barriers
    P.off_r = 0;
    P.off_stage = tcw::kRBufs * P.r_bytes;
    int ns = int((budget - int(P.off_stage)) / tcw::kStageBytes);
    if (ns > tcw::kMaxStages) ns = tcw::kMaxStages;
    if (ns < 2) return fail(KRR_ERR_INVALID_ARG, "sample_tc_wide: stages do not fit in shared memory");
    P.nstage = ns;
    P.off_bar = P.off_stage + ns * tcw::kStageBytes;
    size_t smem = size_t(P.off_bar) + tcw::BAR_COUNT * 8 + 16 + 1024;
    if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM: it holds all 512 TMEM columns
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

    static SmemLimitOnce smem_limit;
    KRR_CUDA(raise_smem_limit(smem_limit, c->device, tcw::sample_tc_wide_kernel, 227 * 1024));
    const int64_t T = P.n_tiles;
    if (T <= 0) return KRR_OK;
    const int grid = int(T < c->num_sms ? T : c->num_sms);
    { tcw::sample_tc_wide_kernel<<<grid, tcw::kThreads, smem, c->stream>>>(mA, mB, mR, P); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

}  // namespace krr
