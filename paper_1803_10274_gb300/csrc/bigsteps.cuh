// Batched pivot-step kernels for the large nodes of the top tree levels,
// where one CTA per node leaves the GPU idle: every pivot step is one
// launch that chooses the pivot (one CTA per matrix) and one launch that
// applies it to all rows of all matrices (a grid over row blocks), so a
// single 1000 x 2000 decomposition spreads over every SM.
//
//   * Gauss-Jordan inverse with partial pivoting (the eliminated blocks
//     and the root block of the ULV-type factorization);
//   * Householder QR with column pivoting of W^T (pivoting over the rows
//     of W), stopped at the numerical rank: the row interpolative
//     decomposition of the node samples.
#pragma once
#include "common.cuh"
#include "dense.cuh"

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
__global__ void __launch_bounds__(256) gj_pivot_kernel(const InvItem *items, T *F, int32_t *I, int j,
                                                       DevStatus *st) {
    const InvItem it = items[blockIdx.x];
    const int n = it.n;
    if (j >= n) return;
    T *A = F + it.off;
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = j + threadIdx.x; i < n; i += 256) {
        const T v = cta::tabs(A[int64_t(i) * n + j]);
        if (v > best) { best = v; bi = i; }
    }
    cta::argmax_block(best, bi);
    const int p = bi;
    if (p != j)
        for (int c = threadIdx.x; c < n; c += 256) {
            const T t = A[int64_t(j) * n + c];
            A[int64_t(j) * n + c] = A[int64_t(p) * n + c];
            A[int64_t(p) * n + c] = t;
        }
    __syncthreads();
    const T piv = A[int64_t(j) * n + j];
    if (threadIdx.x == 0) I[it.ipiv + j] = p;
    if (piv == T(0)) {
        if (threadIdx.x == 0) dev_fail(st, KRR_ERR_SINGULAR, 202);
        return;
    }
    __syncthreads();
    const T inv = T(1) / piv;
    for (int c = threadIdx.x; c < n; c += 256) {
        const T v = c == j ? T(1) : A[int64_t(j) * n + c];
        A[int64_t(j) * n + c] = v * inv;
    }
}

// grid: (row blocks of the largest matrix, items)
template <class T>
__global__ void __launch_bounds__(256) gj_elim_kernel(const InvItem *items, T *F, int j) {
    const InvItem it = items[blockIdx.y];
    const int n = it.n;
    if (j >= n) return;
    T *A = F + it.off;
    const T *rj = A + int64_t(j) * n;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = blockIdx.x * kRowsPerBlock + w; i < min(n, (blockIdx.x + 1) * kRowsPerBlock); i += 8) {
        if (i == j) continue;
        T *ri = A + int64_t(i) * n;
        const T f = ri[j];
        __syncwarp();
        if (f == T(0)) continue;
        for (int c = l; c < n; c += 32) ri[c] = (c == j ? T(0) : ri[c]) - f * rj[c];
    }
}

// undo the row interchanges as column interchanges (one CTA per matrix)
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

template <class T>
int gj_inverse_batched(Ctx *c, const std::vector<InvItem> &items, T *F, int32_t *I) {
    if (items.empty()) return KRR_OK;
    int nmax = 0;
    for (const InvItem &it : items) nmax = it.n > nmax ? it.n : nmax;
    if (nmax == 0) return KRR_OK;
    DBuf<InvItem> d(c, items.size());
    if (!d.get()) return fail(KRR_ERR_OOM, "inverse: out of memory");
    KRR_CUDA(cudaMemcpyAsync(d.get(), items.data(), items.size() * sizeof(InvItem), cudaMemcpyHostToDevice, c->stream));
    const int ni = int(items.size());
    const dim3 eg(unsigned(cdiv(nmax, kRowsPerBlock)), unsigned(ni));
    for (int j = 0; j < nmax; ++j) {
        { gj_pivot_kernel<T><<<ni, 256, 0, c->stream>>>(d.get(), F, I, j, c->status); ::krr::count_launch(); }
        { gj_elim_kernel<T><<<eg, 256, 0, c->stream>>>(d.get(), F, j); ::krr::count_launch(); }
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
