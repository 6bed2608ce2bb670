// Grouped FP32 products C = alpha op(A) op(B) + beta C on the sm_103a
// tensor cores (tcgen05.mma kind::tf32), for the node products of the
// interpolative decompositions and the factorization (Gram matrices,
// Schur-complement updates).
//
// FP32 accuracy from TF32 operands: every element is split as
//     x = x_hi + x_lo,   x_hi = x with its low 13 mantissa bits cleared,
//     x_lo = x - x_hi (exact; the tensor core reads its TF32 bits)
// and the product is accumulated (FP32, tensor memory) as
//     A_hi B_hi + A_hi B_lo + A_lo B_hi,
// which leaves out A_lo B_lo and the low bits of x_lo (together about
// 2^-21 relative to |A||B|) next to the FP32 accumulation itself.
//
// One CTA per SM walks a list of 128 x 128 output tiles over all problems,
// in 32-wide K chunks through a three-step pipeline:
//   1. warps 0-7 copy (cp.async) the chunk's FP32 blocks of A and B
//      (zero-filled past the matrix edges, coalesced along whichever
//      dimension is contiguous) into one of two raw stages, two chunks ahead;
//   2. warps 0-7 split the raw block into the four operand tiles (A_hi,
//      A_lo, B_hi, B_lo: 128 rows of 128 bytes, K-major, 128-byte swizzle)
//      of one of two MMA stages and arrive on its FULL barrier;
//   3. warp 8 waits FULL, issues the chunk's 12 MMAs (4 K-steps x 3 terms)
//      and commits them to the stage's EMPTY barrier.
// The epilogue (warps 0-7) reads the accumulator with tcgen05.ld (warps w
// and w + 4 own tensor-memory lanes 32 (w mod 4) ..; one column half each),
// stages it in shared memory and writes C row by row, coalesced.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "grouped.cuh"
#include "tc_ptx.cuh"

namespace krr {
namespace gtc {

constexpr int kProducers = 256;           // warps 0-7: copies, splits, epilogue
constexpr int kThreads = kProducers + 32;  // warp 8: MMA issue
constexpr int kBM = 128;                 // tile rows (tensor-memory lanes)
constexpr int kBN = 128;                 // tile columns (MMA N, tensor-memory columns)
constexpr int kBK = 32;                  // K per chunk: one 128-byte row of FP32
constexpr int kTileBytes = 128 * 128;    // one operand tile: 128 rows x 128 bytes
constexpr int kMmaStageBytes = 4 * kTileBytes;  // A_hi, A_lo, B_hi, B_lo
constexpr int kRawStageBytes = 2 * kTileBytes;  // FP32 blocks of A and B
constexpr int kStages = 2;
constexpr int kSmemBytes = kStages * (kMmaStageBytes + kRawStageBytes) + 1024 + 8 * 8;

struct Params {
    const GemmProb<float> *probs;  // tile0 / tn counted in 128 x 128 tiles
    const int32_t *tile_prob;      // problem of each tile
    int tiles;
    DevStatus *status;
    long long wait;
};

// Instruction descriptor, kind::tf32: TF32 A and B (format code 2), FP32
// accumulator, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "mov.b64 da, {%1, %5};\n\tmov.b64 db, {%2, %5};\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_lo), "r"(b_lo), "r"(idesc), "r"(accumulate), "r"(hi)
        : "memory");
}

// Byte offset of element (r, k) in a 128-row x 32-column K-major tile with
// the 128-byte swizzle (16-byte chunk index XOR row mod 8).
__device__ __forceinline__ uint32_t sw128(int r, int k) {
    return uint32_t((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ void cp_async4(void *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(ptx::smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_le1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy (cp.async) rows [r0, r0 + 128) x columns [k0, k0 + 32) of an operand
// whose element (r, k) is X[r * sr + k * sk] (sr or sk is 1) into a raw
// 128 x 32 FP32 block, zero past rows R and columns K.  Contiguous along K
// (sk == 1): raw[r * 32 + k]; contiguous along rows: raw[k * 128 + r].
// Consecutive threads take consecutive addresses of the contiguous
// dimension.
__device__ __forceinline__ void copy_block(const float *X, int64_t sr, int64_t sk, int r0, int R, int k0, int K,
                                           float *raw) {
#pragma unroll
    for (int j = 0; j < (kBM * kBK) / kProducers; ++j) {
        const int e = threadIdx.x + kProducers * j;
        int r, k;
        if (sk == 1) { r = e >> 5; k = e & 31; }
        else { k = e >> 7; r = e & 127; }
        const bool valid = r0 + r < R && k0 + k < K;
        const float *src = valid ? X + int64_t(r0 + r) * sr + int64_t(k0 + k) * sk : X;
        cp_async4(raw + e, src, valid);
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const float *src, int valid_floats) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(ptx::smem_u32(dst)), "l"(src),
                 "r"(valid_floats * 4)
                 : "memory");
}

// copy_block in 16-byte copies, for operands whose contiguous dimension
// starts 16-byte aligned in every row (base and stride multiples of 4
// floats): four consecutive elements per copy, the copy zero-filled past
// the matrix edge.
__device__ __forceinline__ void copy_block16(const float *X, int64_t sr, int64_t sk, int r0, int R, int k0, int K,
                                             float *raw) {
#pragma unroll
    for (int j = 0; j < (kBM * kBK) / (4 * kProducers); ++j) {
        const int e4 = threadIdx.x + kProducers * j;
        int r, k, nv;
        if (sk == 1) {
            r = e4 >> 3;
            k = 4 * (e4 & 7);
            nv = r0 + r < R ? min(4, max(0, K - (k0 + k))) : 0;
        } else {
            k = e4 >> 5;
            r = 4 * (e4 & 31);
            nv = k0 + k < K ? min(4, max(0, R - (r0 + r))) : 0;
        }
        const float *src = nv > 0 ? X + int64_t(r0 + r) * sr + int64_t(k0 + k) * sk : X;
        cp_async16(raw + 4 * e4, src, nv);
    }
}

// The raw block split into the hi / lo operand tiles, four elements at a
// time (raw as copy_block / copy_block16 leave it).  Along K the four
// elements share one 16-byte chunk of a swizzled row (one vector store per
// tile); along rows they sit in four rows.
__device__ __forceinline__ void split_block16(const float *raw, bool along_k, uint8_t *hi, uint8_t *lo) {
#pragma unroll
    for (int j = 0; j < (kBM * kBK) / (4 * kProducers); ++j) {
        const int e4 = threadIdx.x + kProducers * j;
        const float4 x = *reinterpret_cast<const float4 *>(raw + 4 * e4);
        const float xs[4] = {x.x, x.y, x.z, x.w};
        uint32_t h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            h[u] = __float_as_uint(xs[u]) & 0xFFFFE000u;          // the TF32 bits of x (truncated)
            l[u] = __float_as_uint(xs[u] - __uint_as_float(h[u]));  // exact remainder; the MMA reads its TF32 bits
        }
        if (along_k) {
            const int r = e4 >> 3, k = 4 * (e4 & 7);
            const uint32_t o = sw128(r, k);
            *reinterpret_cast<uint4 *>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
        } else {
            const int k = e4 >> 5, r = 4 * (e4 & 31);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t o = sw128(r + u, k);
                *reinterpret_cast<uint32_t *>(hi + o) = h[u];
                *reinterpret_cast<uint32_t *>(lo + o) = l[u];
            }
        }
    }
}

constexpr int kEpiLd = kBN + 1;  // staging row stride of the epilogue (floats)
static_assert(kBM * kEpiLd * 4 <= kStages * kMmaStageBytes, "the epilogue stages the tile in the MMA stages");

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(kProducers) : "memory");
}

// Warp-specialized: warps 0-7 copy and split each chunk into an MMA stage
// and arrive on its FULL barrier; warp 8 waits FULL, issues the chunk's
// MMAs and commits them to the stage's EMPTY barrier (and, after a tile's
// last chunk, to TILE); warps 0-7 then read the accumulator and arrive on
// TFREE, which warp 8 waits for before the next tile's first MMA.
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(Params P) {
    extern __shared__ unsigned char gtc_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gtc_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *mma_st = smem;                                                      // kStages x kMmaStageBytes
    float *raw_st = reinterpret_cast<float *>(smem + kStages * kMmaStageBytes);  // kStages x kRawStageBytes
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * (kMmaStageBytes + kRawStageBytes));
    uint64_t *full = bars, *empty = bars + 2, *tile_bar = bars + 4, *tfree = bars + 5, *drain = bars + 6;
    float *E = reinterpret_cast<float *>(smem);  // epilogue staging, kBM x kEpiLd (the MMA stages are free then)
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&full[b], kProducers);
            ptx::mbar_init(&empty[b], 1);
        }
        ptx::mbar_init(tile_bar, 1);
        ptx::mbar_init(tfree, kProducers);
        ptx::mbar_init(drain, 1);
        ptx::fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_slot, kBN);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t issued = 0, tiles_done = 0;
    if (warp == kProducers / 32) {
        // ------------------------------------------------ MMA issue
        constexpr uint32_t idesc = idesc_tf32(kBM, kBN);
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
            const GemmProb<float> &G = P.probs[P.tile_prob[tile]];
            const int nk = (G.K + kBK - 1) / kBK;
            if (nk == 0) continue;
            if (tiles_done > 0 &&  // the previous accumulator has been read
                !ptx::warp_wait(tfree, (tiles_done - 1) & 1u, &abort_flag, P.wait, P.status, 403)) {
                ok = false;
                break;
            }
            for (int kc = 0; kc < nk; ++kc) {
                const uint32_t s = issued & 1u;
                if (!ptx::warp_wait(&full[s], (issued >> 1) & 1u, &abort_flag, P.wait, P.status, 404)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                if (lane == 0) {
                    uint8_t *st = mma_st + s * kMmaStageBytes;
                    const uint32_t ahi = ptx::sdesc_lo_sw128(ptx::smem_u32(st));
                    const uint32_t alo = ptx::sdesc_lo_sw128(ptx::smem_u32(st + kTileBytes));
                    const uint32_t bhi = ptx::sdesc_lo_sw128(ptx::smem_u32(st + 2 * kTileBytes));
                    const uint32_t blo = ptx::sdesc_lo_sw128(ptx::smem_u32(st + 3 * kTileBytes));
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks) {  // K = 8 per MMA: 32 bytes, +2 in 16-byte units
                        const uint32_t d = 2u * ks;
                        mma_tf32(tmem, ahi + d, bhi + d, ptx::kSdescHiSw128, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                        mma_tf32(tmem, ahi + d, blo + d, ptx::kSdescHiSw128, idesc, 1u);
                        mma_tf32(tmem, alo + d, bhi + d, ptx::kSdescHiSw128, idesc, 1u);
                    }
                    ptx::tc_commit(&empty[s]);
                }
                __syncwarp();
                ++issued;
            }
            if (!ok) break;
            if (lane == 0) ptx::tc_commit(tile_bar);
            __syncwarp();
            ++tiles_done;
        }
        // every MMA issued has completed before tensor memory is freed
        if (lane == 0 && issued > 0) {
            ptx::tc_commit(drain);
            ptx::mbar_wait_bounded(drain, 0, P.wait);
        }
        __syncwarp();
    } else {
        // -------------------------------- copies, splits, epilogue
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
            const GemmProb<float> &G = P.probs[P.tile_prob[tile]];
            const int t = tile - G.tile0;
            const int m0 = (t / G.tn) * kBM, n0 = (t % G.tn) * kBN;
            const int nk = (G.K + kBK - 1) / kBK;
            // op(A)(i, k) = ta ? A[k lda + i] : A[i lda + k];  op(B)^T(j, k) = tb ? B[j ldb + k] : B[k ldb + j]
            const int64_t asr = G.ta ? 1 : G.lda, ask = G.ta ? G.lda : 1;
            const int64_t bsr = G.tb ? G.ldb : 1, bsk = G.tb ? 1 : G.ldb;
            // 16-byte copies where every row of the contiguous dimension starts aligned
            const bool a16 = (reinterpret_cast<uintptr_t>(G.A) & 15) == 0 && ((ask == 1 ? asr : ask) & 3) == 0;
            const bool b16 = (reinterpret_cast<uintptr_t>(G.B) & 15) == 0 && ((bsk == 1 ? bsr : bsk) & 3) == 0;
            auto copy_chunk = [&](int kc) {
                float *raw = raw_st + (kc & 1) * (kRawStageBytes / 4);
                if (a16) copy_block16(G.A, asr, ask, m0, G.M, kc * kBK, G.K, raw);
                else copy_block(G.A, asr, ask, m0, G.M, kc * kBK, G.K, raw);
                if (b16) copy_block16(G.B, bsr, bsk, n0, G.N, kc * kBK, G.K, raw + kBM * kBK);
                else copy_block(G.B, bsr, bsk, n0, G.N, kc * kBK, G.K, raw + kBM * kBK);
                cp_async_commit();
            };
            if (nk > 0) copy_chunk(0);
            if (nk > 1) copy_chunk(1);
            for (int kc = 0; kc < nk; ++kc) {
                const uint32_t s = issued & 1u;
                if (kc + 1 < nk) cp_async_wait_le1();  // this chunk's copies landed (the next may be in flight)
                else cp_async_wait_all();
                if (issued >= 2 &&  // the MMA stage's previous chunk (issued - 2) has been consumed
                    !ptx::warp_wait(&empty[s], ((issued - 2) >> 1) & 1u, &abort_flag, P.wait, P.status, 401))
                    abort_flag = 1;
                producers_sync();  // every producer warp then takes the same branch
                if (abort_flag) {
                    ok = false;
                    break;
                }
                uint8_t *st = mma_st + s * kMmaStageBytes;
                const float *raw = raw_st + (kc & 1) * (kRawStageBytes / 4);
                split_block16(raw, ask == 1, st, st + kTileBytes);
                split_block16(raw + kBM * kBK, bsk == 1, st + 2 * kTileBytes, st + 3 * kTileBytes);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor core reads
                ptx::mbar_arrive(&full[s]);
                producers_sync();  // the raw stage is consumed
                if (kc + 2 < nk) copy_chunk(kc + 2);
                ++issued;
            }
            if (!ok) break;
            if (nk > 0) {
                if (!ptx::warp_wait(tile_bar, tiles_done & 1u, &abort_flag, P.wait, P.status, 402)) abort_flag = 1;
                producers_sync();
                if (abort_flag) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
            }
            // epilogue: warp w reads tensor-memory lanes 32 (w mod 4) ..
            // (tile rows) and the column half w / 4, staged in shared
            // memory, then C is written row by row with coalesced accesses
            {
                const int q = warp & 3, half = warp >> 2;
                for (int c0 = half * (kBN / 2); c0 < (half + 1) * (kBN / 2) && n0 + c0 < G.N; c0 += 32) {
                    uint32_t v[32];
                    if (nk > 0) {
                        ptx::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), v);
                        ptx::tmem_wait_ld_regs(v);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0u;
                    }
                    float *er = E + (q * 32 + lane) * kEpiLd + c0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) er[j] = __uint_as_float(v[j]);
                }
            }
            ptx::tc_fence_before();
            if (nk > 0) ptx::mbar_arrive(tfree);  // this thread's reads of the accumulator are done
            producers_sync();
            {
                const int col = n0 + (tid & (kBN - 1));
                const int rows = min(kBM, G.M - m0);
                if (col < G.N) {
                    float *cc = G.C + int64_t(m0) * G.ldc + col;
                    for (int r = tid >> 7; r < rows; r += kProducers / kBN) {
                        const float a = G.alpha * E[r * kEpiLd + (tid & (kBN - 1))];
                        float *cp = cc + int64_t(r) * G.ldc;
                        if (G.atomic) atomicAdd(cp, a);
                        else *cp = G.beta == 0.f ? a : a + G.beta * *cp;
                    }
                }
            }
            if (nk > 0) ++tiles_done;
            producers_sync();  // the staging is read before the next tile's splits overwrite it
        }
        cp_async_wait_all();  // no copy lands after the CTA is gone
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, kBN);
}

}  // namespace gtc

// The tensor-core path pays off for batches with enough work in full
// tiles: at least 1 GFLOP, the problems' tiles on average at least a
// quarter full, and K at least 256 on average (weighted by output size).
#ifndef KRR_TC_MIN_K
#define KRR_TC_MIN_K 256
#endif
#ifndef KRR_TC_MIN_FLOPS
#define KRR_TC_MIN_FLOPS 1e9
#endif
constexpr int kTcMinK = KRR_TC_MIN_K;           // average K (weighted by output size) at least
constexpr double kTcMinFlops = KRR_TC_MIN_FLOPS;  // batch work at least

bool tc_gemm_wanted(const Ctx *c, const std::vector<GemmProb<float>> &v) {
    if (v.empty()) return false;
    double flops = 0, tile_area = 0, area = 0;
    for (const GemmProb<float> &p : v) {
        if (p.skip) return false;  // run-time skips are the CUDA-core kernel's
        flops += 2.0 * p.M * p.N * double(p.K);
        area += double(p.M) * p.N;
        tile_area += double(cdiv(p.M, gtc::kBM) * gtc::kBM) * double(cdiv(p.N, gtc::kBN) * gtc::kBN);
    }
    double mnk = 0;
    for (const GemmProb<float> &p : v) mnk += double(p.M) * p.N * double(p.K);
    // short K (panel updates, R-hat, S_loc corrections) stays on the CUDA
    // cores, whose epilogue costs less per output
    return flops >= kTcMinFlops && area >= 0.25 * tile_area && mnk >= double(kTcMinK) * area;
}

int launch_grouped_tc(Ctx *c, const std::vector<GemmProb<float>> &v) {
    std::vector<GemmProb<float>> w(v);
    std::vector<int32_t> tp;
    int tiles = 0;
    for (size_t q = 0; q < w.size(); ++q) {
        w[q].tile0 = tiles;
        w[q].tn = int(cdiv(w[q].N, gtc::kBN));
        const int nt = int(cdiv(w[q].M, gtc::kBM)) * w[q].tn;
        tp.insert(tp.end(), size_t(nt), int32_t(q));
        tiles += nt;
    }
    if (tiles == 0) return KRR_OK;
    DBuf<GemmProb<float>> d(c, w.size());
    DBuf<int32_t> dtp(c, tp.size());
    if (!d.get() || !dtp.get()) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
    KRR_CUDA(cudaMemcpyAsync(d.get(), w.data(), w.size() * sizeof(GemmProb<float>), cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaMemcpyAsync(dtp.get(), tp.data(), tp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    static SmemLimitOnce smem_limit;
    KRR_CUDA(raise_smem_limit(smem_limit, c->device, gtc::tc_gemm_kernel, gtc::kSmemBytes));
    gtc::Params P;
    P.probs = d.get();
    P.tile_prob = dtp.get();
    P.tiles = tiles;
    P.status = c->status;
    P.wait = c->wait_cycles;
    const int grid = std::min(tiles, c->num_sms);
    { gtc::tc_gemm_kernel<<<grid, gtc::kThreads, gtc::kSmemBytes, c->stream>>>(P); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

}  // namespace krr

extern "C" int krr_gemm_f32_batched(krr_ctx *k, int32_t batch, int32_t M, int32_t N, int32_t K, float alpha,
                                    const float *A, int64_t lda, int64_t sA, int32_t ta, const float *B, int64_t ldb,
                                    int64_t sB, int32_t tb, float beta, float *C, int64_t ldc, int64_t sC,
                                    int32_t path) {
    using namespace krr;
    if (!k || batch < 0 || M < 0 || N < 0 || K < 0 || path < 0 || path > 2 || (ta != 0 && ta != 1) ||
        (tb != 0 && tb != 1))
        return fail(KRR_ERR_INVALID_ARG, "krr_gemm_f32_batched: bad arguments");
    if (batch == 0 || M == 0 || N == 0) return KRR_OK;
    // output tiles are counted in int on both paths
    if (int64_t(batch) * cdiv(M, gtc::kBM) * cdiv(N, gtc::kBN) > 0x7FFFFFFF)
        return fail(KRR_ERR_INVALID_ARG, "krr_gemm_f32_batched: more than 2^31 - 1 output tiles");
    if (!C || ldc < N || (K > 0 && (!A || !B || lda < (ta ? M : K) || ldb < (tb ? K : N))))
        return fail(KRR_ERR_INVALID_ARG, "krr_gemm_f32_batched: bad pointer or leading dimension");
    Ctx *c = &k->c;
    GemmBatch<float> gb;
    for (int32_t b = 0; b < batch; ++b)
        gb.push(M, N, K, alpha, A + int64_t(b) * sA, lda, ta != 0, B + int64_t(b) * sB, ldb, tb != 0, beta,
                C + int64_t(b) * sC, ldc, 0);
    if (path == 1) {
        KRR_TRY(launch_grouped_tc(c, gb.v));
        return KRR_OK;
    }
    gb.force_cuda_cores = path == 2;
    return gb.launch(c);
}

