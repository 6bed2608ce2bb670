// Grouped GEMM: many independent products C = alpha op(A) op(B) + beta C
// (one per tree node, of different sizes) in one launch.  The 64 x 64
// output tiles of all problems form one list that persistent CTAs walk, so
// a level with two large nodes still spreads over every SM.
#pragma once
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace krr {

template <class T>
struct GemmProb {
    const T *A, *B;
    T *C;
    int64_t lda, ldb, ldc;
    int M, N, K, ta, tb;
    T alpha, beta;
    int tile0, tn;  // first tile index of this problem, tiles along N
    int atomic;     // 1: one K-slice of a split product, added into C atomically
    const int *skip;  // the product is skipped when *skip != 0 at run time (NULL: never)
};

// A region of C to clear before split products add into it.
template <class T>
struct ZeroJob {
    T *C;
    int64_t ldc;
    int M, N;
};

template <class T>
__global__ void zero_jobs_kernel(const ZeroJob<T> *jobs, int nj) {
    const ZeroJob<T> z = jobs[blockIdx.y];
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < int64_t(z.M) * z.N;
         e += int64_t(gridDim.x) * blockDim.x)
        z.C[(e / z.N) * z.ldc + e % z.N] = T(0);
}

// Tile: 64 rows x TN columns (TN = 64, or 16 for right-hand-side blocks);
// each of the 256 threads owns (64 / (256 / (TN / 4))) x 4 outputs.
template <class T, int TN>
__global__ void __launch_bounds__(256) grouped_gemm_kernel(const GemmProb<T> *probs, int np, int total_tiles) {
    constexpr int CG = TN / 4;          // column groups of 4
    constexpr int RG = 256 / CG;        // row groups
    constexpr int RPT = 64 / RG;        // rows per thread
    __shared__ T As[16][68];
    __shared__ T Bs[16][TN + 4];
    const int tid = threadIdx.x;
    const int tr = tid / CG, tc = tid % CG;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].tile0 <= tile) lo = mid;
            else hi = mid - 1;
        }
        const GemmProb<T> &P = probs[lo];
        if (P.skip && __ldcg(P.skip)) continue;  // the same for the whole CTA
        const int t = tile - P.tile0;
        const int i0 = (t / P.tn) * 64, j0 = (t % P.tn) * TN;
        const int M = P.M, N = P.N, K = P.K;
        T acc[RPT][4];
#pragma unroll
        for (int a = 0; a < RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int k0 = 0; k0 < K; k0 += 16) {
            for (int e = tid; e < 1024; e += 256) {
                int ii, kk;
                if (!P.ta) { ii = e >> 4; kk = e & 15; } else { kk = e >> 6; ii = e & 63; }
                const int gi = i0 + ii, gk = k0 + kk;
                T v = T(0);
                if (gi < M && gk < K) v = P.ta ? P.A[int64_t(gk) * P.lda + gi] : P.A[int64_t(gi) * P.lda + gk];
                As[kk][ii] = v;
            }
            for (int e = tid; e < 16 * TN; e += 256) {
                int jj, kb;
                if (!P.tb) { kb = e / TN; jj = e % TN; } else { jj = e >> 4; kb = e & 15; }
                const int gj = j0 + jj, gkb = k0 + kb;
                T w = T(0);
                if (gj < N && gkb < K) w = P.tb ? P.B[int64_t(gj) * P.ldb + gkb] : P.B[int64_t(gkb) * P.ldb + gj];
                Bs[kb][jj] = w;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                T av[RPT], bv[4];
#pragma unroll
                for (int a = 0; a < RPT; ++a) av[a] = As[kk][tr * RPT + a];
#pragma unroll
                for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tc * 4 + b];
#pragma unroll
                for (int a = 0; a < RPT; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
            }
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < RPT; ++a) {
            const int gi = i0 + tr * RPT + a;
            if (gi >= M) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int gj = j0 + tc * 4 + b;
                if (gj >= N) continue;
                T *c = P.C + int64_t(gi) * P.ldc + gj;
                if (P.atomic) atomicAdd(c, P.alpha * acc[a][b]);
                else *c = P.beta == T(0) ? P.alpha * acc[a][b] : P.alpha * acc[a][b] + P.beta * *c;
            }
        }
    }
}

// Skinny products (N <= 16 columns per output tile: right-hand-side blocks
// of the ULV solve) are bound by reading A once.  A streams from global
// memory with coalesced loads; only the item's rows of B (at most 512 x 16)
// are staged in shared memory.  Every thread owns one output row (lane =
// row within a 32-row half; the warp picks the half and one of four K
// quarters, summed at the end), so no shuffle reductions are needed:
//   op(A) = A^T (A stored K x M): consecutive lanes read consecutive rows;
//   op(A) = A (A stored M x K): the warp reads 32 x 32 blocks row by row
//     (coalesced along K) into its own shared-memory tile and reads them
//     back transposed (only warp-level synchronization).
template <class T>
struct SkinnyCfg {
    static constexpr int KB = 512;  // K of B staged at a time
    static constexpr size_t smem() {
        return sizeof(T) * (size_t(KB) * 16 + size_t(4) * 64 * 16 + size_t(8) * 32 * 33);
    }
};

// One output tile of a skinny product list, by a CTA of 256 threads with
// SkinnyCfg<T>::smem() bytes of shared memory (every thread calls it).
// tp: the problem of every tile (plans), or NULL (binary search over tile0).
template <class T>
__device__ void skinny_tile(const GemmProb<T> *probs, int np, int tile, unsigned char *smem, const int32_t *tp) {
    constexpr int KB = SkinnyCfg<T>::KB;
    T *Bs = reinterpret_cast<T *>(smem);          // KB x 16
    T *red = Bs + KB * 16;                        // [4][64][16]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T *tw = red + 4 * 64 * 16 + warp * 32 * 33;   // this warp's 32 x 33 transpose tile
    const int row = 32 * (warp & 1) + lane, grp = warp >> 1;
    {
        int lo = 0, hi = np - 1;
        if (tp) lo = tp[tile];
        else
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (probs[mid].tile0 <= tile) lo = mid;
                else hi = mid - 1;
            }
        const GemmProb<T> &P = probs[lo];
        const int t = tile - P.tile0;
        const int i0 = (t / P.tn) * 64, j0 = (t % P.tn) * 16;
        const int M = P.M, K = P.K, nc = min(16, P.N - j0);
        const int gi = i0 + row;
        T acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = T(0);
        for (int kb0 = 0; kb0 < K; kb0 += KB) {
            const int kbn = min(KB, K - kb0);
            __syncthreads();
            for (int e = tid; e < kbn * 16; e += 256) {
                const int k = e >> 4, c = e & 15;
                // B (a right-hand-side block another CTA may have written
                // earlier in a one-launch sweep) is read through L2
                Bs[e] = c < nc ? (P.tb ? __ldcg(P.B + int64_t(j0 + c) * P.ldb + kb0 + k)
                                       : __ldcg(P.B + int64_t(kb0 + k) * P.ldb + j0 + c))
                               : T(0);
            }
            __syncthreads();
            const int qn = (kbn + 3) / 4;
            const int q0 = grp * qn, q1 = min(kbn, q0 + qn);
            if (P.ta) {
                if (gi < M) {
                    const T *a = P.A + int64_t(kb0) * P.lda + gi;
                    int k = q0;
                    for (; k + 4 <= q1; k += 4) {
                        const T a0 = a[int64_t(k) * P.lda], a1 = a[int64_t(k + 1) * P.lda];
                        const T a2 = a[int64_t(k + 2) * P.lda], a3 = a[int64_t(k + 3) * P.lda];
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[c] += a0 * Bs[k * 16 + c] + a1 * Bs[(k + 1) * 16 + c] + a2 * Bs[(k + 2) * 16 + c] +
                                      a3 * Bs[(k + 3) * 16 + c];
                    }
                    for (; k < q1; ++k) {
                        const T a0 = a[int64_t(k) * P.lda];
#pragma unroll
                        for (int c = 0; c < 16; ++c) acc[c] += a0 * Bs[k * 16 + c];
                    }
                }
            } else {
                const int r0 = i0 + 32 * (warp & 1);  // first row of this warp's half
                for (int k = q0; k < q1; k += 32) {
                    const int kn = min(32, q1 - k);
                    // rows r0 .. r0 + 31, K columns k .. k + kn - 1, read along K
                    // all 32 loads issued before the first shared-memory store
                    T av[32];
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr)
                        av[rr] = (r0 + rr < M && lane < kn) ? P.A[int64_t(r0 + rr) * P.lda + kb0 + k + lane] : T(0);
                    __syncwarp();
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) tw[rr * 33 + lane] = av[rr];
                    __syncwarp();
                    for (int kk = 0; kk < kn; ++kk) {
                        const T a0 = tw[lane * 33 + kk];
#pragma unroll
                        for (int c = 0; c < 16; ++c) acc[c] += a0 * Bs[(k + kk) * 16 + c];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 16; ++c) red[(grp * 64 + row) * 16 + c] = acc[c];
        __syncthreads();
        for (int e = tid; e < 64 * 16; e += 256) {
            const int ii = e >> 4, c = e & 15;
            const int go = i0 + ii;
            if (go >= M || c >= nc) continue;
            const T v = red[ii * 16 + c] + red[(64 + ii) * 16 + c] + red[(128 + ii) * 16 + c] +
                        red[(192 + ii) * 16 + c];
            T *cp = P.C + int64_t(go) * P.ldc + j0 + c;
            if (P.atomic) atomicAdd(cp, P.alpha * v);
            else *cp = P.beta == T(0) ? P.alpha * v : P.alpha * v + P.beta * __ldcg(cp);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) skinny_gemm_kernel(const GemmProb<T> *probs, int np, int total_tiles,
                                                          const int32_t *tp) {
    extern __shared__ __align__(16) unsigned char skinny_smem[];
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x)
        skinny_tile<T>(probs, np, tile, skinny_smem, tp);
}

template <class T, int TN>
inline cudaError_t launch_grouped(Ctx *c, const GemmProb<T> *probs, int np, int tiles, const int32_t *tp = nullptr) {
    const int grid = tiles < 4 * c->num_sms ? tiles : 4 * c->num_sms;
    if (TN == 16) {
        static SmemLimitOnce once;
        const int bytes = int(SkinnyCfg<T>::smem());
        const cudaError_t e = raise_smem_limit(once, c->device, skinny_gemm_kernel<T>, bytes);
        if (e != cudaSuccess) return e;
        skinny_gemm_kernel<T><<<grid, 256, bytes, c->stream>>>(probs, np, tiles, tp);
    } else {
        grouped_gemm_kernel<T, TN><<<grid, 256, 0, c->stream>>>(probs, np, tiles);
    }
    ::krr::count_launch();
    return cudaGetLastError();
}

// A problem list uploaded once and launched many times.
template <class T, int TN>
struct GemmPlan {
    DBuf<GemmProb<T>> d;
    DBuf<ZeroJob<T>> z;
    DBuf<int32_t> tp;  // problem of each tile (skinny plans)
    int np = 0, tiles = 0, nz = 0, zmax = 0;
    int run(Ctx *c) const {
        if (nz > 0) {
            const dim3 g(unsigned(cdiv(zmax, 256) < 64 ? cdiv(zmax, 256) : 64), unsigned(nz));
            { zero_jobs_kernel<T><<<g, 256, 0, c->stream>>>(z.get(), nz); ::krr::count_launch(); }
        }
        if (np == 0) return KRR_OK;
        KRR_CUDA((launch_grouped<T, TN>(c, d.get(), np, tiles, tp.get())));
        return KRR_OK;
    }
};

// Large FP32 batches on the tensor cores (tcgen05 kind::tf32 with a
// three-term split, FP32 accuracy; gemm_tc.cu): whether a batch qualifies,
// and its launch.
bool tc_gemm_wanted(const Ctx *c, const std::vector<GemmProb<float>> &v);
int launch_grouped_tc(Ctx *c, const std::vector<GemmProb<float>> &v);

template <class T, int TN = 64>
struct GemmBatch {
    std::vector<GemmProb<T>> v;
    std::vector<ZeroJob<T>> zj;
    int tiles = 0;
    // Skinny products (TN = 16: few output tiles over a long K) are split
    // into K-slices of kSlice that add into C atomically, so one product
    // spreads over several CTAs (the top levels of the tree have one or two
    // nodes); a product that overwrites C has C cleared first (only in
    // plans, which run the clearing before the GEMMs).
    static constexpr int kSlice = 64;
    bool split_ok = false;
    bool force_cuda_cores = false;  // never the tensor-core path (comparisons)
    void add(int M, int N, int K, T alpha, const T *A, int64_t lda, bool ta, const T *B, int64_t ldb, bool tb, T beta,
             T *C, int64_t ldc) {
        if (M <= 0 || N <= 0) return;
        if (K <= 0 && beta == T(1)) return;
        if (split_ok && TN == 16 && K > 2 * kSlice && (beta == T(1) || beta == T(0))) {
            if (beta == T(0)) zj.push_back(ZeroJob<T>{C, ldc, M, N});
            for (int k0 = 0; k0 < K; k0 += kSlice) {
                const int kk = K - k0 < kSlice ? K - k0 : kSlice;
                const T *As = ta ? A + int64_t(k0) * lda : A + k0;
                const T *Bs = tb ? B + k0 : B + int64_t(k0) * ldb;
                push(M, N, kk, alpha, As, lda, ta, Bs, ldb, tb, T(1), C, ldc, 1);
            }
            return;
        }
        push(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, 0);
    }
    void push(int M, int N, int K, T alpha, const T *A, int64_t lda, bool ta, const T *B, int64_t ldb, bool tb,
              T beta, T *C, int64_t ldc, int atomic) {
        GemmProb<T> p;
        p.atomic = atomic;
        p.skip = nullptr;
        p.A = A;
        p.B = B;
        p.C = C;
        p.lda = lda;
        p.ldb = ldb;
        p.ldc = ldc;
        p.M = M;
        p.N = N;
        p.K = K < 0 ? 0 : K;
        p.ta = ta ? 1 : 0;
        p.tb = tb ? 1 : 0;
        p.alpha = alpha;
        p.beta = beta;
        p.tile0 = tiles;
        p.tn = int(cdiv(N, TN));
        tiles += int(cdiv(M, 64)) * p.tn;
        v.push_back(p);
    }
    // upload into a reusable plan (the batch is left empty)
    int freeze(Ctx *c, GemmPlan<T, TN> &plan) {
        plan.np = int(v.size());
        plan.tiles = tiles;
        plan.nz = int(zj.size());
        plan.zmax = 0;
        for (const ZeroJob<T> &z : zj) plan.zmax = plan.zmax > z.M * z.N ? plan.zmax : z.M * z.N;
        if (!v.empty()) {
            if (!plan.d.reset(c, v.size())) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
            KRR_CUDA(cudaMemcpyAsync(plan.d.get(), v.data(), v.size() * sizeof(GemmProb<T>), cudaMemcpyHostToDevice,
                                     c->stream));
            if (TN == 16 && tiles > 0) {
                std::vector<int32_t> tp(size_t(tiles), 0);
                for (size_t q = 0; q < v.size(); ++q) {
                    const int nt = int(cdiv(v[q].M, 64)) * v[q].tn;
                    for (int t = 0; t < nt; ++t) tp[size_t(v[q].tile0 + t)] = int32_t(q);
                }
                if (!plan.tp.reset(c, tp.size())) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
                KRR_CUDA(cudaMemcpyAsync(plan.tp.get(), tp.data(), tp.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                         c->stream));
            }
        }
        if (!zj.empty()) {
            if (!plan.z.reset(c, zj.size())) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
            KRR_CUDA(cudaMemcpyAsync(plan.z.get(), zj.data(), zj.size() * sizeof(ZeroJob<T>), cudaMemcpyHostToDevice,
                                     c->stream));
        }
        KRR_CUDA(cudaStreamSynchronize(c->stream));
        v.clear();
        zj.clear();
        tiles = 0;
        return KRR_OK;
    }
    int launch(Ctx *c) {
        if (!zj.empty()) {
            DBuf<ZeroJob<T>> z(c, zj.size());
            if (!z.get()) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
            KRR_CUDA(cudaMemcpyAsync(z.get(), zj.data(), zj.size() * sizeof(ZeroJob<T>), cudaMemcpyHostToDevice,
                                     c->stream));
            int zmax = 0;
            for (const ZeroJob<T> &q : zj) zmax = zmax > q.M * q.N ? zmax : q.M * q.N;
            const dim3 g(unsigned(cdiv(zmax, 256) < 64 ? cdiv(zmax, 256) : 64), unsigned(zj.size()));
            { zero_jobs_kernel<T><<<g, 256, 0, c->stream>>>(z.get(), int(zj.size())); ::krr::count_launch(); }
            zj.clear();
        }
        if (v.empty()) return KRR_OK;
        if constexpr (std::is_same<T, float>::value && TN == 64) {
            if (!force_cuda_cores && tc_gemm_wanted(c, v)) {
                KRR_TRY(launch_grouped_tc(c, v));
                v.clear();
                tiles = 0;
                return KRR_OK;
            }
        }
        DBuf<GemmProb<T>> d(c, v.size());
        if (!d.get()) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
        KRR_CUDA(cudaMemcpyAsync(d.get(), v.data(), v.size() * sizeof(GemmProb<T>), cudaMemcpyHostToDevice, c->stream));
        KRR_CUDA((launch_grouped<T, TN>(c, d.get(), int(v.size()), tiles)));
        v.clear();
        tiles = 0;
        return KRR_OK;
    }
};

// A sequence of CUDA-core batches (the steps of a blocked triangular solve,
// the panels of a blocked factorization) uploaded in one copy and launched
// one by one without a host-to-device copy or an allocation per step.
template <class T, int TN = 64>
struct GemmSeq {
    std::vector<GemmProb<T>> all;
    std::vector<int> off, np, tiles;
    DBuf<GemmProb<T>> d;
    // appends the batch as the next step (the batch is left empty; no
    // clearing jobs: every product of a sequence accumulates into C)
    void add_step(GemmBatch<T, TN> &b) {
        off.push_back(int(all.size()));
        np.push_back(int(b.v.size()));
        tiles.push_back(b.tiles);
        all.insert(all.end(), b.v.begin(), b.v.end());
        b.v.clear();
        b.tiles = 0;
    }
    int upload(Ctx *c) {
        if (all.empty()) return KRR_OK;
        if (!d.reset(c, all.size())) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
        KRR_CUDA(cudaMemcpyAsync(d.get(), all.data(), all.size() * sizeof(GemmProb<T>), cudaMemcpyHostToDevice,
                                 c->stream));
        return KRR_OK;
    }
    int launch(Ctx *c, int step) const {
        if (np[step] == 0) return KRR_OK;
        KRR_CUDA((launch_grouped<T, TN>(c, d.get() + off[step], np[step], tiles[step])));
        return KRR_OK;
    }
};

}  // namespace krr
