// Batched pivot-step kernels for the large nodes of the top tree levels,
// where one CTA per node leaves the GPU idle: every pivot step is one
// launch that chooses the pivot (one CTA per matrix) and one launch that
// applies it to all rows of all matrices (a grid over row blocks), so a
// single 1000 x 2000 decomposition spreads over every SM.
//
//   * Gauss-Jordan inverse with partial pivoting (the eliminated blocks
//     and the root block of the ULV-type factorization), in panels of
//     kGjPanel pivots: one launch per panel per step, the rest as grouped
//     GEMMs;
//   * Householder QR with column pivoting of W^T (pivoting over the rows
//     of W), stopped at the numerical rank: the row interpolative
//     decomposition of the node samples.
#pragma once
#include <algorithm>
#include <vector>
#include "common.cuh"
#include "dense.cuh"
#include "grouped.cuh"

namespace krr {
namespace big {

constexpr int kRowsPerBlock = 8;  // rows per CTA in the apply launches (one warp per row)

// ------------------------------------------------------- Gauss-Jordan
struct InvItem {
    int64_t off;   // matrix (n x n, row-major, ld n) in the arena
    int64_t ipiv;  // int arena offset, n entries
    int n;
};

template <class T>
__global__ void __launch_bounds__(256) gj_unswap_kernel(const InvItem *items, T *F, const int32_t *I) {
    const InvItem it = items[blockIdx.x];
    const int n = it.n;
    T *A = F + it.off;
    for (int j = n - 1; j >= 0; --j) {
        const int p = I[it.ipiv + j];
        if (p != j)
            for (int r = threadIdx.x; r < n; r += 256) {
                const T t = A[int64_t(r) * n + j];
                A[int64_t(r) * n + j] = A[int64_t(r) * n + p];
                A[int64_t(r) * n + p] = t;
            }
        __syncthreads();
    }
}

// ------------------------------------------- blocked Gauss-Jordan inverse
// The same in-place elimination, kGjPanel pivots at a time.  Within a panel
// (one CTA per matrix) rows are interchanged over their full width but the
// eliminations touch only the panel's columns; those columns then hold the
// composite transform M of the panel's steps (in-place Gauss-Jordan leaves
// the transform's columns where the eliminated columns were).  Every other
// column c is then updated at once: A(:, c) <- M A(:, c), i.e. with the
// panel rows J, A(J, c) copied out and zeroed, A(:, c) += A(:, J-columns)
// A_old(J, c) -- one grouped GEMM per panel over all matrices.
constexpr int kGjPanel = 32;

template <class T>
__global__ void __launch_bounds__(1024) gjb_panel_kernel(const InvItem *items, T *F, int32_t *I, int j0,
                                                        DevStatus *st) {
    const InvItem it = items[blockIdx.x];
    const int n = it.n;
    if (j0 >= n) return;
    T *A = F + it.off;
    const int jend = min(j0 + kGjPanel, n);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __shared__ T sv[32];
    __shared__ int si[32];
    for (int j = j0; j < jend; ++j) {
        // pivot: largest |A(i, j)| over i >= j, ties to the lowest row
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + threadIdx.x; i < n; i += 1024) {
            const T v = cta::tabs(A[int64_t(i) * n + j]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (l == 0) { sv[w] = best; si[w] = bi; }
        __syncthreads();
        if (w == 0) {
            best = sv[l];
            bi = si[l];
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (l == 0) { sv[0] = best; si[0] = bi; }
        }
        __syncthreads();
        const int p = si[0];
        __syncthreads();
        if (p != j)
            for (int c = threadIdx.x; c < n; c += 1024) {
                const T t = A[int64_t(j) * n + c];
                A[int64_t(j) * n + c] = A[int64_t(p) * n + c];
                A[int64_t(p) * n + c] = t;
            }
        if (threadIdx.x == 0) I[it.ipiv + j] = p;
        __syncthreads();
        const T piv = A[int64_t(j) * n + j];
        if (piv == T(0)) {
            if (threadIdx.x == 0) dev_fail(st, KRR_ERR_SINGULAR, 203);
            return;  // every thread read the same pivot
        }
        const T inv = T(1) / piv;
        __syncthreads();
        for (int c = j0 + threadIdx.x; c < jend; c += 1024) {
            const T v = c == j ? T(1) : A[int64_t(j) * n + c];
            A[int64_t(j) * n + c] = v * inv;
        }
        __syncthreads();
        // other rows, panel columns only: lane c - j0 of a warp owns column c
        const T rj = (j0 + l < jend) ? A[int64_t(j) * n + j0 + l] : T(0);
        for (int i = w; i < n; i += 32) {
            if (i == j) continue;
            T *ri = A + int64_t(i) * n;
            const T f = ri[j];
            __syncwarp();
            if (j0 + l < jend) {
                const int c = j0 + l;
                ri[c] = (c == j ? T(0) : ri[c]) - f * rj;
            }
        }
        __syncthreads();
    }
}

// The same panel with its n x kGjPanel block staged in shared memory (row
// stride kGjPanel + 1, so column reads hit distinct banks): the pivot
// search, scaling and eliminations run there, latency-free; only the row
// interchanges of the columns outside the panel touch global memory.
constexpr int kGjLd = kGjPanel + 1;
constexpr int kGjSmemMax = 200 * 1024;  // panel bytes staged in shared memory at most

template <class T>
__global__ void __launch_bounds__(1024) gjb_panel_smem_kernel(const InvItem *items, T *F, int32_t *I, int j0,
                                                             DevStatus *st) {
    extern __shared__ __align__(16) unsigned char gj_smem[];
    T *P = reinterpret_cast<T *>(gj_smem);  // P[i * kGjLd + c] = A(i, j0 + c)
    const InvItem it = items[blockIdx.x];
    const int n = it.n;
    if (j0 >= n) return;
    T *A = F + it.off;
    const int jend = min(j0 + kGjPanel, n), b = jend - j0;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __shared__ T sv[32];
    __shared__ int si[32];
    for (int i = w; i < n; i += 32) P[i * kGjLd + l] = l < b ? A[int64_t(i) * n + j0 + l] : T(0);
    __syncthreads();
    for (int j = j0; j < jend; ++j) {
        const int jl = j - j0;
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + threadIdx.x; i < n; i += 1024) {
            const T v = cta::tabs(P[i * kGjLd + jl]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (l == 0) { sv[w] = best; si[w] = bi; }
        __syncthreads();
        if (w == 0) {
            best = sv[l];
            bi = si[l];
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (l == 0) { sv[0] = best; si[0] = bi; }
        }
        __syncthreads();
        const int p = si[0];
        if (p != j) {
            for (int c = threadIdx.x; c < n - b; c += 1024) {  // columns outside the panel
                const int cc = c < j0 ? c : c + b;
                const T t = A[int64_t(j) * n + cc];
                A[int64_t(j) * n + cc] = A[int64_t(p) * n + cc];
                A[int64_t(p) * n + cc] = t;
            }
            if (w == 0) {
                const T t = P[j * kGjLd + l];
                P[j * kGjLd + l] = P[p * kGjLd + l];
                P[p * kGjLd + l] = t;
            }
        }
        if (threadIdx.x == 0) I[it.ipiv + j] = p;
        __syncthreads();
        const T piv = P[j * kGjLd + jl];
        if (piv == T(0)) {
            if (threadIdx.x == 0) dev_fail(st, KRR_ERR_SINGULAR, 204);
            return;  // every thread read the same pivot
        }
        const T inv = T(1) / piv;
        __syncthreads();
        if (w == 0 && l < b) {
            const T v = l == jl ? T(1) : P[j * kGjLd + l];
            P[j * kGjLd + l] = v * inv;
        }
        __syncthreads();
        // other rows, panel columns: lane c of a warp owns panel column c
        const T rj = P[j * kGjLd + l];
        for (int i = w; i < n; i += 32) {
            if (i == j) continue;
            const T f = P[i * kGjLd + jl];
            __syncwarp();
            P[i * kGjLd + l] = (l == jl ? T(0) : P[i * kGjLd + l]) - f * rj;
        }
        __syncthreads();
    }
    for (int i = w; i < n; i += 32)
        if (l < b) A[int64_t(i) * n + j0 + l] = P[i * kGjLd + l];
}

// Rows [j0, jend) outside the panel's columns: copied to Tt (kGjPanel rows
// of n - (jend - j0), in column order with the panel removed) and zeroed.
template <class T>
__global__ void gjb_copyout_kernel(const InvItem *items, T *F, T *Tt, int64_t tstride, int j0) {
    const InvItem it = items[blockIdx.y];
    const int n = it.n;
    if (j0 >= n) return;
    const int jend = min(j0 + kGjPanel, n);
    const int b = jend - j0, nr = n - b;
    T *A = F + it.off;
    T *Tp = Tt + int64_t(blockIdx.y) * tstride;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < int64_t(b) * nr;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int t = int(e / nr), cc = int(e % nr);
        const int c = cc < j0 ? cc : cc + b;
        T *a = A + int64_t(j0 + t) * n + c;
        Tp[e] = *a;
        *a = T(0);
    }
}

template <class T>
int gj_inverse_blocked(Ctx *c, const std::vector<InvItem> &items, T *F, int32_t *I) {
    if (items.empty()) return KRR_OK;
    int nmax = 0;
    for (const InvItem &it : items) nmax = it.n > nmax ? it.n : nmax;
    if (nmax == 0) return KRR_OK;
    const int ni = int(items.size());
    DBuf<InvItem> d(c, ni);
    const int64_t tstride = int64_t(kGjPanel) * nmax;
    DBuf<T> Tt(c, size_t(ni) * tstride);
    if (!d.get() || !Tt.get()) return fail(KRR_ERR_OOM, "inverse: out of memory");
    KRR_CUDA(cudaMemcpyAsync(d.get(), items.data(), ni * sizeof(InvItem), cudaMemcpyHostToDevice, c->stream));
    const size_t psmem = size_t(nmax) * kGjLd * sizeof(T);
    const bool staged = psmem <= size_t(kGjSmemMax);
    if (staged) {
        static SmemLimitOnce smem_limit;
        KRR_CUDA(raise_smem_limit(smem_limit, c->device, gjb_panel_smem_kernel<T>, kGjSmemMax));
    }
    for (int j0 = 0; j0 < nmax; j0 += kGjPanel) {
        if (staged)
            { gjb_panel_smem_kernel<T><<<ni, 1024, psmem, c->stream>>>(d.get(), F, I, j0, c->status); ::krr::count_launch(); }
        else
            { gjb_panel_kernel<T><<<ni, 1024, 0, c->stream>>>(d.get(), F, I, j0, c->status); ::krr::count_launch(); }
        const dim3 cg(unsigned(std::min<int64_t>(cdiv(int64_t(kGjPanel) * nmax, 256), 64)), unsigned(ni));
        { gjb_copyout_kernel<T><<<cg, 256, 0, c->stream>>>(d.get(), F, Tt.get(), tstride, j0); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        // every column outside the panel: A(:, c) += A(:, panel) Tt
        GemmBatch<T> gb;
        for (int a = 0; a < ni; ++a) {
            const InvItem &it = items[a];
            const int n = it.n;
            if (j0 >= n) continue;
            const int jend = std::min(j0 + kGjPanel, n), b = jend - j0, nr = n - b;
            T *A = F + it.off;
            const T *Tp = Tt.get() + int64_t(a) * tstride;
            gb.add(n, j0, b, T(1), A + j0, n, false, Tp, nr, false, T(1), A, n);
            gb.add(n, n - jend, b, T(1), A + j0, n, false, Tp + j0, nr, false, T(1), A + jend, n);
        }
        KRR_TRY(gb.launch(c));
    }
    { gj_unswap_kernel<T><<<ni, 256, 0, c->stream>>>(d.get(), F, I); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// ------------------------------------------------- pivoted QR (row ID)
struct QrItem {
    int64_t w;      // W (m x rfull, row-major, ld rfull) in the arena
    int64_t norm;   // squared trailing norms, m entries
    int64_t v;      // Householder vector, rid entries
    int64_t piv;    // int arena, m entries
    int m, rid, rfull, kmax;
};

// per-item state: k (rank so far), done flag, r11, beta, total squared norm
struct QrState {
    int k, done;
    double r11, beta, tot0;
};

template <class T>
__global__ void __launch_bounds__(256) qr_init_kernel(const QrItem *items, QrState *state, T *F, int32_t *I) {
    const QrItem it = items[blockIdx.y];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = blockIdx.x * kRowsPerBlock + w; i < min(it.m, (blockIdx.x + 1) * kRowsPerBlock); i += 8) {
        const T *row = F + it.w + int64_t(i) * it.rfull;
        T s = T(0);
        for (int t = l; t < it.rid; t += 32) s += row[t] * row[t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) {
            F[it.norm + i] = s;
            I[it.piv + i] = i;
            atomicAdd(&state[blockIdx.y].tot0, double(s));
        }
    }
}

// One CTA per item: pivot choice, rank test, row swap, Householder vector.
template <class T>
__global__ void __launch_bounds__(256) qr_pivot_kernel(const QrItem *items, QrState *state, T *F, int32_t *I, int j,
                                                       double eps, double eps_abs, double r11_cap) {
    const QrItem it = items[blockIdx.x];
    QrState &S = state[blockIdx.x];
    if (S.done) return;
    const int m = it.m, rid = it.rid;
    if (j >= m || j >= rid || j >= it.kmax) {
        if (threadIdx.x == 0) { S.done = 1; S.k = j; }
        return;
    }
    T *norm2 = F + it.norm;
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = j + threadIdx.x; i < m; i += 256)
        if (norm2[i] > best) { best = norm2[i]; bi = i; }
    cta::argmax_block(best, bi);
    const double nrm = sqrt(double(best));
    const double r11 = j == 0 ? (nrm < r11_cap ? nrm : r11_cap) : S.r11;
    if (!(nrm > eps * r11) || !(nrm > eps_abs)) {
        if (threadIdx.x == 0) { S.done = 1; S.k = j; if (j == 0) S.r11 = nrm; }
        return;
    }
    const int p = bi;
    T *W = F + it.w;
    const int64_t ld = it.rfull;
    if (p != j) {
        for (int t = threadIdx.x; t < it.rfull; t += 256) {
            const T a = W[int64_t(j) * ld + t];
            W[int64_t(j) * ld + t] = W[int64_t(p) * ld + t];
            W[int64_t(p) * ld + t] = a;
        }
        if (threadIdx.x == 0) {
            int32_t *piv = I + it.piv;
            const int a = piv[j]; piv[j] = piv[p]; piv[p] = a;
            const T b = norm2[j]; norm2[j] = norm2[p]; norm2[p] = b;
        }
    }
    __syncthreads();
    T *v = F + it.v;
    const T x0 = W[int64_t(j) * ld + j];
    const T alpha = x0 >= T(0) ? T(-nrm) : T(nrm);
    T vv = T(0);
    for (int t = j + threadIdx.x; t < rid; t += 256) {
        const T x = t == j ? x0 - alpha : W[int64_t(j) * ld + t];
        v[t] = x;
        vv += x * x;
    }
    vv = cta::sum_block(vv);
    for (int t = j + threadIdx.x; t < rid; t += 256) W[int64_t(j) * ld + t] = t == j ? alpha : T(0);
    if (threadIdx.x == 0) {
        S.r11 = r11;
        S.beta = vv > T(0) ? 2.0 / double(vv) : 0.0;
        S.k = j + 1;
    }
}

// grid: (row blocks, items): reflect rows > j, recompute trailing norms.
template <class T>
__global__ void __launch_bounds__(256) qr_apply_kernel(const QrItem *items, const QrState *state, T *F, int j) {
    const QrItem it = items[blockIdx.y];
    const QrState &S = state[blockIdx.y];
    if (S.done || S.k != j + 1) return;  // no reflector was made at this step
    const int rid = it.rid;
    const T beta = T(S.beta);
    const T *v = F + it.v;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int i0 = blockIdx.x * kRowsPerBlock;
    for (int i = i0 + w; i < min(it.m, i0 + kRowsPerBlock); i += 8) {
        if (i <= j) continue;
        T *row = F + it.w + int64_t(i) * it.rfull;
        T dot = T(0);
        for (int t = j + l; t < rid; t += 32) dot += v[t] * row[t];
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const T f = beta * dot;
        T s = T(0);
        for (int t = j + l; t < rid; t += 32) {
            const T y = row[t] - f * v[t];
            row[t] = y;
            if (t > j) s += y * y;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) F[it.norm + i] = s;
    }
}

}  // namespace big
}  // namespace krr
