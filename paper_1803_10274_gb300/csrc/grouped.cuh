// Grouped GEMM: many independent products C = alpha op(A) op(B) + beta C
// (one per tree node, of different sizes) in one launch.  The 64 x 64
// output tiles of all problems form one list that persistent CTAs walk, so
// a level with two large nodes still spreads over every SM.
#pragma once
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

// A problem list uploaded once and launched many times.
template <class T, int TN>
struct GemmPlan {
    DBuf<GemmProb<T>> d;
    DBuf<ZeroJob<T>> z;
    int np = 0, tiles = 0, nz = 0, zmax = 0;
    int run(Ctx *c) const {
        if (nz > 0) {
            const dim3 g(unsigned(cdiv(zmax, 256) < 64 ? cdiv(zmax, 256) : 64), unsigned(nz));
            { zero_jobs_kernel<T><<<g, 256, 0, c->stream>>>(z.get(), nz); ::krr::count_launch(); }
        }
        if (np == 0) return KRR_OK;
        const int grid = tiles < 4 * c->num_sms ? tiles : 4 * c->num_sms;
        { grouped_gemm_kernel<T, TN><<<grid, 256, 0, c->stream>>>(d.get(), np, tiles); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        return KRR_OK;
    }
};

template <class T, int TN = 64>
struct GemmBatch {
    std::vector<GemmProb<T>> v;
    std::vector<ZeroJob<T>> zj;
    int tiles = 0;
    // Skinny products (TN = 16: few output tiles over a long K) are split
    // into K-slices of kSlice that add into C atomically, so one product
    // spreads over several CTAs; a product that overwrites C has C cleared
    // first (only in plans, which run the clearing before the GEMMs).
    static constexpr int kSlice = 256;
    bool split_ok = false;
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
        DBuf<GemmProb<T>> d(c, v.size());
        if (!d.get()) return fail(KRR_ERR_OOM, "grouped gemm: out of memory");
        KRR_CUDA(cudaMemcpyAsync(d.get(), v.data(), v.size() * sizeof(GemmProb<T>), cudaMemcpyHostToDevice, c->stream));
        const int grid = tiles < 4 * c->num_sms ? tiles : 4 * c->num_sms;
        { grouped_gemm_kernel<T, TN><<<grid, 256, 0, c->stream>>>(d.get(), int(v.size()), tiles); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        v.clear();
        tiles = 0;
        return KRR_OK;
    }
};

}  // namespace krr
