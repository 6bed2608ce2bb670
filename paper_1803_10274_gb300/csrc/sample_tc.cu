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

#include "common.cuh"
#include "tc_ptx.cuh"

namespace krr {
namespace tc {

constexpr int kThreads = 384;
constexpr int kBM = 128;             // rows of a tile (tensor-memory lanes)
constexpr int kBN = 128;             // K columns of a tile
constexpr int kChunk = 64;           // FP16 elements per 128-byte swizzled row
constexpr int kChunkBytes = 128 * 128;
constexpr int kMaxStages = 6;
constexpr int kDistCol0 = 256;       // tensor-memory columns of the two distance buffers
constexpr long long kWaitBudget = 4000000000ll;  // ~2 s of SM clock per wait

struct Params {
    int64_t ma, nb;
    int64_t n_row_tiles, n_col_tiles;
    int r;        // R / S columns handled by this launch (multiple of 64, <= 256)
    int r_valid;  // columns actually stored (<= r)
    int nchunk;   // 64-element chunks of an augmented row
    int kmma;     // K=16 MMA steps of the distance GEMM
    int nstage;
    int s_bufs;   // S accumulators in tensor memory (1 or 2)
    uint32_t off_a, off_stage, stage_bytes, off_bar;
    const int32_t *leaf_a, *leaf_b;
    float *S;
    int64_t lds;
    DevStatus *status;
};

// Barrier slots (uint64 each) after off_bar.
enum {
    BAR_FULL = 0,
    BAR_EMPTY = BAR_FULL + kMaxStages,
    BAR_AFULL = BAR_EMPTY + kMaxStages,
    BAR_AEMPTY = BAR_AFULL + 2,
    BAR_DFULL = BAR_AEMPTY + 2,
    BAR_PFULL = BAR_DFULL + 2,
    BAR_SFULL = BAR_PFULL + 2,
    BAR_SEMPTY = BAR_SFULL + 2,
    BAR_DRAIN = BAR_SEMPTY + 2,
    BAR_COUNT = BAR_DRAIN + 1
};

__device__ __forceinline__ bool first_in_seg(int64_t t, int64_t t0, int64_t nct) { return t == t0 || (t % nct) == 0; }
__device__ __forceinline__ bool last_in_seg(int64_t t, int64_t t1, int64_t nct) {
    return t == t1 - 1 || (t % nct) == nct - 1;
}

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

    const int64_t nct = P.n_col_tiles;
    const int64_t T = P.n_row_tiles * nct;
    const int64_t t0 = T * blockIdx.x / gridDim.x;
    const int64_t t1 = T * (blockIdx.x + 1) / gridDim.x;
    const int64_t nloc = t1 - t0;
    const int NS = P.nstage;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[BAR_FULL + s], 1);
            mbar_init(&bars[BAR_EMPTY + s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars[BAR_AFULL + b], 1);
            mbar_init(&bars[BAR_AEMPTY + b], 1);
            mbar_init(&bars[BAR_DFULL + b], 1);
            mbar_init(&bars[BAR_PFULL + b], 8);
            mbar_init(&bars[BAR_SFULL + b], 1);
            mbar_init(&bars[BAR_SEMPTY + b], 8);
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
    const uint32_t a_bytes = P.nchunk * kChunkBytes;

    if (warp == 0 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t ph = 0;
        int64_t seg = -1;
        int64_t issued = 0;
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t rt = t / nct, ct = t % nct;
            if (first_in_seg(t, t0, nct)) {
                ++seg;
                const int ab = int(seg & 1);
                if (!mbar_wait(&bars[BAR_AEMPTY + ab], uint32_t((seg >> 1) & 1) ^ 1u, abort_flag, kWaitBudget,
                               P.status, 1))
                    break;
                mbar_expect_tx(&bars[BAR_AFULL + ab], a_bytes);
                for (int c = 0; c < P.nchunk; ++c)
                    tma_load_2d(smem + P.off_a + ab * a_bytes + c * kChunkBytes, &tmA, &bars[BAR_AFULL + ab],
                                c * kChunk, int(rt * kBM));
            }
            if (!mbar_wait(&bars[BAR_EMPTY + stage], ph ^ 1u, abort_flag, kWaitBudget, P.status, 2)) break;
            uint8_t *st = smem + P.off_stage + stage * P.stage_bytes;
            mbar_expect_tx(&bars[BAR_FULL + stage], P.stage_bytes);
            for (int c = 0; c < P.nchunk; ++c)
                tma_load_2d(st + c * kChunkBytes, &tmB, &bars[BAR_FULL + stage], c * kChunk, int(ct * kBN));
            tma_load_2d(st + a_bytes, &tmR, &bars[BAR_FULL + stage], int(ct * kBN), 0);
            tma_load_2d(st + a_bytes + P.r * 128, &tmR, &bars[BAR_FULL + stage], int(ct * kBN + 64), 0);
            ++issued;
            if (++stage == NS) {
                stage = 0;
                ph ^= 1u;
            }
        }
        // Drain: wait (bounded) until every load issued has landed, so no
        // TMA write is in flight when the CTA exits.
        for (int64_t k = 0; k < (issued < NS ? issued : NS); ++k) {
            int64_t u = issued - 1 - k;  // use index of that fill
            int s = int(u % NS);
            uint32_t parity = uint32_t((u / NS) & 1);
            if (!mbar_try_wait(&bars[BAR_FULL + s], parity)) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&bars[BAR_FULL + s], parity) && clock64() - c0 < kWaitBudget) {
                }
            }
        }
    } else if (warp == 1 && lane == 0 && nloc > 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc_d = idesc_f16_f32(kBM, kBN);
        const uint32_t idesc_p = idesc_f16_f32(kBM, P.r);
        int64_t seg_next = -1;  // segment of the tile whose distance GEMM was issued last
        int64_t seg_cur = -1;
        bool ok = true;
        auto stage_of = [&](int64_t loc) { return int(loc % NS); };
        auto phase_of = [&](int64_t loc) { return uint32_t((loc / NS) & 1); };
        auto issue_dist = [&](int64_t loc) -> bool {
            const int64_t t = t0 + loc;
            if (first_in_seg(t, t0, nct)) {
                ++seg_next;
                if (!mbar_wait(&bars[BAR_AFULL + (seg_next & 1)], uint32_t((seg_next >> 1) & 1), abort_flag,
                               kWaitBudget, P.status, 3))
                    return false;
            }
            const int s = stage_of(loc);
            if (!mbar_wait(&bars[BAR_FULL + s], phase_of(loc), abort_flag, kWaitBudget, P.status, 4)) return false;
            tc_fence_after();
            const uint32_t a_base = smem_u32(smem + P.off_a + (seg_next & 1) * a_bytes);
            const uint32_t b_base = smem_u32(smem + P.off_stage + s * P.stage_bytes);
            const uint32_t d_tmem = tmem + kDistCol0 + uint32_t(loc & 1) * kBN;
            for (int k = 0; k < P.kmma; ++k) {
                const uint32_t off = (k >> 2) * kChunkBytes + (k & 3) * 32;
                mma_ss(d_tmem, sdesc_k_sw128(a_base + off), sdesc_k_sw128(b_base + off), idesc_d, k > 0);
            }
            tc_commit(&bars[BAR_DFULL + (loc & 1)]);
            if (last_in_seg(t, t1, nct)) tc_commit(&bars[BAR_AEMPTY + (seg_next & 1)]);
            return true;
        };
        ok = issue_dist(0);
        for (int64_t loc = 0; ok && loc < nloc; ++loc) {
            const int64_t t = t0 + loc;
            if (loc + 1 < nloc && !issue_dist(loc + 1)) break;
            if (first_in_seg(t, t0, nct)) {
                ++seg_cur;
                const int sb = int(seg_cur % P.s_bufs);
                if (!mbar_wait(&bars[BAR_SEMPTY + sb], uint32_t((seg_cur / P.s_bufs) & 1) ^ 1u, abort_flag,
                               kWaitBudget, P.status, 5))
                    break;
            }
            const int sb = int(seg_cur % P.s_bufs);
            const int b = int(loc & 1);
            if (!mbar_wait(&bars[BAR_PFULL + b], uint32_t((loc >> 1) & 1), abort_flag, kWaitBudget, P.status, 6))
                break;
            tc_fence_after();
            const int s = stage_of(loc);
            const uint32_t r_base = smem_u32(smem + P.off_stage + s * P.stage_bytes + a_bytes);
            const uint32_t s_tmem = tmem + uint32_t(sb * P.r);
            const uint32_t p_tmem = tmem + kDistCol0 + uint32_t(b) * kBN;
            const bool first = first_in_seg(t, t0, nct);
            for (int k = 0; k < 8; ++k) {
                const uint32_t a_t = p_tmem + uint32_t((k >> 2) * 64 + (k & 3) * 8);
                const uint32_t roff = uint32_t((k >> 2) * P.r * 128 + (k & 3) * 32);
                mma_ts(s_tmem, a_t, sdesc_k_sw128(r_base + roff), idesc_p, (first && k == 0) ? 0u : 1u);
            }
            tc_commit(&bars[BAR_EMPTY + s]);
            if (last_in_seg(t, t1, nct)) tc_commit(&bars[BAR_SFULL + sb]);
        }
        // Drain: every MMA issued has completed before tensor memory is freed.
        tc_commit(&bars[BAR_DRAIN]);
        if (!mbar_try_wait(&bars[BAR_DRAIN], 0)) {
            const long long c0 = clock64();
            while (!mbar_try_wait(&bars[BAR_DRAIN], 0) && clock64() - c0 < kWaitBudget) {
            }
        }
    } else if (warp >= 4 && nloc > 0) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;          // lane quarter of tensor memory
        const int g = (warp - 4) >> 2;   // 64-column half of the tile
        const uint32_t lane_off = uint32_t(32 * q) << 16;
        int64_t seg = -1;
        const bool masked = P.leaf_a != nullptr;
        const int rh = P.r >> 1;
        for (int64_t loc = 0; loc < nloc; ++loc) {
            const int64_t t = t0 + loc;
            const int64_t rt = t / nct, ct = t % nct;
            if (first_in_seg(t, t0, nct)) ++seg;
            const int b = int(loc & 1);
            if (!mbar_wait(&bars[BAR_DFULL + b], uint32_t((loc >> 1) & 1), abort_flag, kWaitBudget, P.status, 7))
                break;
            tc_fence_after();
            const uint32_t base = tmem + lane_off + kDistCol0 + uint32_t(b) * kBN + uint32_t(64 * g);
            uint32_t v0[32], v1[32];
            tmem_ld32(base, v0);
            tmem_ld32(base + 32, v1);
            tmem_wait_ld();
            const int64_t i = rt * kBM + 32 * q + lane;
            bool tile_masked = false;
            int32_t li = 0;
            const int64_t j0 = ct * kBN + 64 * g;
            if (masked) {
                const int64_t ia = rt * kBM, ib = min(rt * kBM + kBM - 1, P.ma - 1);
                const int64_t ja = ct * kBN, jb = min(ct * kBN + kBN - 1, P.nb - 1);
                const int32_t lo = max(__ldg(P.leaf_a + ia), __ldg(P.leaf_b + ja));
                const int32_t hi = min(__ldg(P.leaf_a + ib), __ldg(P.leaf_b + jb));
                tile_masked = lo <= hi;
                li = __ldg(P.leaf_a + min(i, P.ma - 1));
            }
            uint32_t pk[32];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float e0 = ex2_approx(__uint_as_float(v0[2 * c]));
                float e1 = ex2_approx(__uint_as_float(v0[2 * c + 1]));
                float f0 = ex2_approx(__uint_as_float(v1[2 * c]));
                float f1 = ex2_approx(__uint_as_float(v1[2 * c + 1]));
                if (tile_masked) {
                    const int64_t ja = j0 + 2 * c, jb2 = j0 + 32 + 2 * c;
                    if (ja < P.nb && __ldg(P.leaf_b + ja) == li) e0 = 0.f;
                    if (ja + 1 < P.nb && __ldg(P.leaf_b + ja + 1) == li) e1 = 0.f;
                    if (jb2 < P.nb && __ldg(P.leaf_b + jb2) == li) f0 = 0.f;
                    if (jb2 + 1 < P.nb && __ldg(P.leaf_b + jb2 + 1) == li) f1 = 0.f;
                }
                __half2 h0 = __floats2half2_rn(e0, e1);
                __half2 h1 = __floats2half2_rn(f0, f1);
                pk[c] = *reinterpret_cast<uint32_t *>(&h0);
                pk[16 + c] = *reinterpret_cast<uint32_t *>(&h1);
            }
            tmem_st32(base, pk);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[BAR_PFULL + b]);
            if (last_in_seg(t, t1, nct)) {
                const int sb = int(seg % P.s_bufs);
                if (!mbar_wait(&bars[BAR_SFULL + sb], uint32_t((seg / P.s_bufs) & 1), abort_flag, kWaitBudget,
                               P.status, 8))
                    break;
                tc_fence_after();
                for (int cc = 0; cc < rh; cc += 32) {
                    uint32_t sv[32];
                    tmem_ld32(tmem + lane_off + uint32_t(sb * P.r + g * rh + cc), sv);
                    tmem_wait_ld();
                    if (i < P.ma) {
                        float *dst = P.S + i * P.lds;
                        const int cbase = g * rh + cc;
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (cbase + c < P.r_valid) atomicAdd(dst + cbase + c, __uint_as_float(sv[c]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[BAR_SEMPTY + sb]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem, 512);
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
// ld_elems), box of box_cols x box_rows with the 128-byte swizzle.
int make_map(CUtensorMap *m, const void *base, int64_t cols, int64_t rows, int64_t ld_elems, int box_cols,
             int box_rows) {
    EncodeTiledFn fn = encode_fn();
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

// S (+)= W o K(XA rows, XB rows) RT^T, accumulated atomically into S
// (which the caller zeroes).  XA, XB: augmented FP16 rows (Kpad = 64 *
// nchunk elements each); RT: FP16, rpad x ldrt (row c = column c of R).
int launch_sample_tc(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int nchunk, int kmma,
                     const __half *RT, int rpad, int64_t ldrt, int r_valid, const int32_t *leaf_a,
                     const int32_t *leaf_b, float *S, int64_t lds) {
    if (rpad % 64 != 0 || rpad < 64 || rpad > 256) return fail(KRR_ERR_INVALID_ARG, "sample_tc: r must be 64..256, /64");
    if (nchunk < 1 || nchunk > 2) return fail(KRR_ERR_INVALID_ARG, "sample_tc: feature dimension too large");
    if (ma <= 0 || nb <= 0) return KRR_OK;
    if (ldrt % 8 != 0) return fail(KRR_ERR_INVALID_ARG, "sample_tc: ldrt must be a multiple of 8");
    CUtensorMap mA, mB, mR;
    const int kpad = 64 * nchunk;
    KRR_TRY(make_map(&mA, XA, kpad, ma, kpad, 64, tc::kBM));
    KRR_TRY(make_map(&mB, XB, kpad, nb, kpad, 64, tc::kBN));
    KRR_TRY(make_map(&mR, RT, nb, rpad, ldrt, 64, rpad));

    tc::Params P{};
    P.ma = ma;
    P.nb = nb;
    P.n_row_tiles = cdiv(ma, tc::kBM);
    P.n_col_tiles = cdiv(nb, tc::kBN);
    P.r = rpad;
    P.r_valid = r_valid;
    P.nchunk = nchunk;
    P.kmma = kmma;
    P.s_bufs = (2 * rpad <= tc::kDistCol0) ? 2 : 1;
    const uint32_t a_bytes = nchunk * tc::kChunkBytes;
    P.off_a = 0;
    P.off_stage = 2 * a_bytes;
    P.stage_bytes = a_bytes + 2 * rpad * 128;
    const int budget = 227 * 1024 - 1024 - 256;  // alignment slack + barriers
    int ns = int((budget - int(P.off_stage)) / int(P.stage_bytes));
    if (ns > tc::kMaxStages) ns = tc::kMaxStages;
    if (ns < 2) return fail(KRR_ERR_INVALID_ARG, "sample_tc: tile does not fit in shared memory");
    P.nstage = ns;
    P.off_bar = P.off_stage + ns * P.stage_bytes;
    size_t smem = size_t(P.off_bar) + tc::BAR_COUNT * 8 + 16 + 1024;
    // The kernel allocates all 512 tensor-memory columns, so two CTAs must
    // never share an SM: asking for more than half of the SM's shared
    // memory guarantees that.
    if (smem < 120 * 1024) smem = 120 * 1024;
    P.leaf_a = leaf_a;
    P.leaf_b = leaf_b;
    P.S = S;
    P.lds = lds;
    P.status = c->status;

    static bool attr_set = false;
    if (!attr_set) {
        KRR_CUDA(cudaFuncSetAttribute(tc::sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024));
        attr_set = true;
    }
    const int64_t T = P.n_row_tiles * P.n_col_tiles;
    const int grid = int(T < c->num_sms ? T : c->num_sms);
    tc::sample_tc_kernel<<<grid, tc::kThreads, smem, c->stream>>>(mA, mB, mR, P);
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

}  // namespace krr
