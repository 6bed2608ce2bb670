// CTA-level dense linear algebra on global-memory operands (row-major,
// explicit leading dimensions), used by the per-node HSS kernels where one
// CTA of kNT threads owns one tree node.  Every routine must be called by
// all threads of the CTA (they synchronize internally).
#pragma once
#include "common.cuh"

namespace krr {
namespace cta {

constexpr int kNT = 256;

template <class T>
__device__ __forceinline__ T tabs(T x) {
    return x < T(0) ? -x : x;
}

// C (M x N) = alpha * op(A) * op(B) + beta * C.  op(A) is M x K: A[i*lda+k]
// or, transposed, A[k*lda+i]; op(B) is K x N: B[k*ldb+j] or B[j*ldb+k].
// beta == 0 ignores C's previous contents.
template <class T, bool TA, bool TB>
__device__ void gemm(int M, int N, int K, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb, T beta, T *C,
                     int64_t ldc) {
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;
    for (int i0 = 0; i0 < M; i0 += 64) {
        for (int j0 = 0; j0 < N; j0 += 64) {
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
            for (int k0 = 0; k0 < K; k0 += 16) {
                for (int e = tid; e < 1024; e += kNT) {
                    int ii, kk;
                    if (!TA) { ii = e >> 4; kk = e & 15; } else { kk = e >> 6; ii = e & 63; }
                    const int gi = i0 + ii, gk = k0 + kk;
                    T v = T(0);
                    if (gi < M && gk < K) v = TA ? A[int64_t(gk) * lda + gi] : A[int64_t(gi) * lda + gk];
                    As[kk][ii] = v;
                    int jj, kb;
                    if (!TB) { kb = e >> 6; jj = e & 63; } else { jj = e >> 4; kb = e & 15; }
                    const int gj = j0 + jj, gkb = k0 + kb;
                    T w = T(0);
                    if (gj < N && gkb < K) w = TB ? B[int64_t(gj) * ldb + gkb] : B[int64_t(gkb) * ldb + gj];
                    Bs[kb][jj] = w;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    T av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) av[a] = As[kk][tr * 4 + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tc * 4 + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
                }
                __syncthreads();
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int gi = i0 + tr * 4 + a;
                if (gi >= M) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int gj = j0 + tc * 4 + b;
                    if (gj >= N) continue;
                    T *c = C + int64_t(gi) * ldc + gj;
                    *c = beta == T(0) ? alpha * acc[a][b] : alpha * acc[a][b] + beta * *c;
                }
            }
        }
    }
    __syncthreads();
}

// Block-wide argmax of (value, index) with ties to the lowest index.
template <class T>
__device__ void argmax_block(T &val, int &idx) {
    __shared__ T sv[kNT / 32];
    __shared__ int si[kNT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, val, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = val; si[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x < 32) {
        val = threadIdx.x < kNT / 32 ? sv[threadIdx.x] : T(-1);
        idx = threadIdx.x < kNT / 32 ? si[threadIdx.x] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, val, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
        }
        if (threadIdx.x == 0) { sv[0] = val; si[0] = idx; }
    }
    __syncthreads();
    val = sv[0];
    idx = si[0];
    __syncthreads();
}

template <class T>
__device__ T sum_block(T v) {
    __shared__ T s[kNT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    for (int w = 0; w < kNT / 32; ++w) t += s[w];
    __syncthreads();
    return t;
}

// In-place LU with partial pivoting of the n x n matrix A (row-major):
// P A = L U with unit-lower L.  ipiv[j] = row swapped with row j at step
// j.  Returns false on an exactly zero pivot.
template <class T>
__device__ bool lu(int n, T *A, int64_t lda, int *ipiv) {
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + threadIdx.x; i < n; i += kNT) {
            const T v = tabs(A[int64_t(i) * lda + j]);
            if (v > best) { best = v; bi = i; }
        }
        argmax_block(best, bi);
        const int p = bi;
        if (p != j)
            for (int c = threadIdx.x; c < n; c += kNT) {
                const T t = A[int64_t(j) * lda + c];
                A[int64_t(j) * lda + c] = A[int64_t(p) * lda + c];
                A[int64_t(p) * lda + c] = t;
            }
        if (threadIdx.x == 0) ipiv[j] = p;
        __syncthreads();
        const T piv = A[int64_t(j) * lda + j];
        if (piv == T(0)) {
            ok = false;
            break;
        }
        for (int i = j + 1 + threadIdx.x; i < n; i += kNT) A[int64_t(i) * lda + j] /= piv;
        __syncthreads();
        // trailing update, one warp per row
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int i = j + 1 + w; i < n; i += kNT / 32) {
            const T lij = A[int64_t(i) * lda + j];
            if (lij == T(0)) continue;
            T *ri = A + int64_t(i) * lda;
            const T *rj = A + int64_t(j) * lda;
            for (int c = j + 1 + l; c < n; c += 32) ri[c] -= lij * rj[c];
        }
        __syncthreads();
    }
    __syncthreads();
    return ok;
}

// Solve (P L U) X = B in place for B (n x nr, row-major, ldb).
template <class T>
__device__ void lu_solve(int n, const T *A, int64_t lda, const int *ipiv, int nr, T *B, int64_t ldb) {
    for (int j = 0; j < n; ++j) {
        const int p = ipiv[j];
        if (p != j)
            for (int c = threadIdx.x; c < nr; c += kNT) {
                const T t = B[int64_t(j) * ldb + c];
                B[int64_t(j) * ldb + c] = B[int64_t(p) * ldb + c];
                B[int64_t(p) * ldb + c] = t;
            }
        __syncthreads();
    }
    // forward: unit lower
    for (int j = 0; j < n; ++j) {
        for (int e = threadIdx.x; e < (n - j - 1) * nr; e += kNT) {
            const int i = j + 1 + e / nr, c = e % nr;
            B[int64_t(i) * ldb + c] -= A[int64_t(i) * lda + j] * B[int64_t(j) * ldb + c];
        }
        __syncthreads();
    }
    // backward: upper
    for (int j = n - 1; j >= 0; --j) {
        const T d = A[int64_t(j) * lda + j];
        for (int c = threadIdx.x; c < nr; c += kNT) B[int64_t(j) * ldb + c] /= d;
        __syncthreads();
        for (int e = threadIdx.x; e < j * nr; e += kNT) {
            const int i = e / nr, c = e % nr;
            B[int64_t(i) * ldb + c] -= A[int64_t(i) * lda + j] * B[int64_t(j) * ldb + c];
        }
        __syncthreads();
    }
}

// T = R11^{-1} R12 (k x (m-k), row-major, ld m-k) from a pivoted QR stored
// transposed in the first k rows of W (row b, coordinate a = R[a][b]):
// one thread per redundant row (column of R12), back substitution.
template <class T>
__device__ void id_T(int m, int k, const T *W, int64_t ldw, T *Tout) {
    const int nr = m - k;
    for (int c = threadIdx.x; c < nr; c += kNT) {
        for (int a = k - 1; a >= 0; --a) {
            T s = W[int64_t(k + c) * ldw + a];  // R12[a][c]
            for (int b = a + 1; b < k; ++b) s -= W[int64_t(b) * ldw + a] * Tout[int64_t(b) * nr + c];
            Tout[int64_t(a) * nr + c] = s / W[int64_t(a) * ldw + a];
        }
    }
}

// Row interpolative decomposition of the m x r matrix W (row-major,
// overwritten): Householder QR with column pivoting of W^T, pivoting over
// the rows of W.  Only the first r columns enter the QR; rows are swapped
// over the full width rfull, so columns [r, rfull) stay the original values
// (held-out samples for an error estimate).  At step j the pivot is the remaining row with the
// largest 2-norm of its coordinates [j, r) (norms recomputed after every
// update; ties to the lowest index); the rank is the number of pivots with
// norm > eps * min(first pivot norm, r11_cap) and > eps_abs.  Rows are physically
// swapped, piv[a] gives the original position of row a.  On return the
// first k rows hold R^T (row b, coordinate a = R[a][b]) and T = R11^{-1}
// R12 (k x (m-k), row-major, ldt = m - k) is written to Tout.
template <class T>
__device__ int row_id(int m, int r, int rfull, T *W, int64_t ldw, T eps, T eps_abs, int *piv, T *norm2, T *Tout,
                       int kmax, T *in_err, T r11_cap) {
    __shared__ int s_k;
    extern __shared__ unsigned char dyn_smem_raw[];
    T *v = reinterpret_cast<T *>(dyn_smem_raw);  // Householder vector, length r
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = threadIdx.x; i < m; i += kNT) piv[i] = i;
    // initial squared norms, one warp per row
    for (int i = w; i < m; i += kNT / 32) {
        T s = T(0);
        for (int t = l; t < r; t += 32) {
            const T x = W[int64_t(i) * ldw + t];
            s += x * x;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) norm2[i] = s;
    }
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    T tot0 = T(0);
    for (int i = threadIdx.x; i < m; i += kNT) tot0 += norm2[i];
    tot0 = sum_block(tot0);
    T r11 = T(0);
    const int jmax = min(min(m, r), kmax);
    for (int j = 0; j < jmax; ++j) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + threadIdx.x; i < m; i += kNT)
            if (norm2[i] > best) { best = norm2[i]; bi = i; }
        argmax_block(best, bi);
        const T nrm = sqrt(best);
        if (j == 0) r11 = nrm < r11_cap ? nrm : r11_cap;
        if (!(nrm > eps * r11) || !(nrm > eps_abs)) break;
        const int p = bi;
        if (p != j) {
            for (int t = threadIdx.x; t < rfull; t += kNT) {
                const T a = W[int64_t(j) * ldw + t];
                W[int64_t(j) * ldw + t] = W[int64_t(p) * ldw + t];
                W[int64_t(p) * ldw + t] = a;
            }
            if (threadIdx.x == 0) {
                const int a = piv[j]; piv[j] = piv[p]; piv[p] = a;
                const T b = norm2[j]; norm2[j] = norm2[p]; norm2[p] = b;
            }
        }
        __syncthreads();
        // Householder vector from coordinates [j, r) of row j
        const T x0 = W[int64_t(j) * ldw + j];
        const T alpha = x0 >= T(0) ? -nrm : nrm;
        for (int t = j + threadIdx.x; t < r; t += kNT) v[t] = W[int64_t(j) * ldw + t];
        __syncthreads();
        if (threadIdx.x == 0) v[j] = x0 - alpha;
        __syncthreads();
        T vv = T(0);
        for (int t = j + threadIdx.x; t < r; t += kNT) vv += v[t] * v[t];
        vv = sum_block(vv);
        const T beta = vv > T(0) ? T(2) / vv : T(0);
        // pivot row becomes (alpha, 0, ..., 0) on [j, r)
        for (int t = j + threadIdx.x; t < r; t += kNT) W[int64_t(j) * ldw + t] = t == j ? alpha : T(0);
        // reflect the remaining rows and recompute their trailing norms
        for (int i = j + 1 + w; i < m; i += kNT / 32) {
            T *row = W + int64_t(i) * ldw;
            T dot = T(0);
            for (int t = j + l; t < r; t += 32) dot += v[t] * row[t];
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            const T f = beta * dot;
            T s = T(0);
            for (int t = j + l; t < r; t += 32) {
                const T y = row[t] - f * v[t];
                row[t] = y;
                if (t > j) s += y * y;
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (l == 0) norm2[i] = s;
        }
        if (threadIdx.x == 0) s_k = j + 1;
        __syncthreads();
    }
    __syncthreads();
    const int k = s_k;
    // in-sample relative residual ||R22||_F / ||W||_F (trailing norms of the
    // rows not taken)
    T rest = T(0);
    for (int i = k + threadIdx.x; i < m; i += kNT) rest += norm2[i];
    rest = sum_block(rest);
    if (in_err) *in_err = tot0 > T(0) ? sqrt(rest / tot0) : T(0);
    id_T<T>(m, k, W, ldw, Tout);
    __syncthreads();
    return k;
}

}  // namespace cta
}  // namespace krr

namespace krr {
namespace cta {
// Relative Frobenius error of the interpolative decomposition on held-out
// columns [c0, c1) of W (rows in pivot order, untouched by the QR):
// || W_r - T^T W_s || / || W ||.
template <class T>
__device__ T id_test_error(int m, int k, const T *W, int64_t ldw, const T *Tm, int c0, int c1) {
    const int nr = m - k;
    T err = T(0), tot = T(0);
    for (int e = threadIdx.x; e < m * (c1 - c0); e += kNT) {
        const int c = e / (c1 - c0), t = c0 + e % (c1 - c0);
        const T w = W[int64_t(c) * ldw + t];
        tot += w * w;
        if (c >= k) {
            T s = w;
            for (int a = 0; a < k; ++a) s -= Tm[int64_t(a) * nr + (c - k)] * W[int64_t(a) * ldw + t];
            err += s * s;
        }
    }
    err = sum_block(err);
    tot = sum_block(tot);
    return tot > T(0) ? sqrt(err / tot) : T(0);
}
}  // namespace cta
}  // namespace krr

namespace krr {
namespace cta {
// In-place inverse of the n x n matrix A (row-major) by Gauss-Jordan
// elimination with partial pivoting; ipiv is scratch (n ints).  Returns
// false on an exactly zero pivot.
template <class T>
__device__ bool gj_inverse(int n, T *A, int64_t lda, int *ipiv) {
    bool ok = true;
    __shared__ T s_piv;
    for (int j = 0; j < n; ++j) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + threadIdx.x; i < n; i += kNT) {
            const T v = tabs(A[int64_t(i) * lda + j]);
            if (v > best) { best = v; bi = i; }
        }
        argmax_block(best, bi);
        const int p = bi;
        if (p != j)
            for (int c = threadIdx.x; c < n; c += kNT) {
                const T t = A[int64_t(j) * lda + c];
                A[int64_t(j) * lda + c] = A[int64_t(p) * lda + c];
                A[int64_t(p) * lda + c] = t;
            }
        if (threadIdx.x == 0) {
            ipiv[j] = p;
            s_piv = A[int64_t(j) * lda + j];
        }
        __syncthreads();
        const T piv = s_piv;
        if (piv == T(0)) {
            ok = false;
            break;
        }
        // row j /= pivot, with A[j][j] replaced by 1 first
        const T inv = T(1) / piv;
        for (int c = threadIdx.x; c < n; c += kNT) {
            const T v = c == j ? T(1) : A[int64_t(j) * lda + c];
            A[int64_t(j) * lda + c] = v * inv;
        }
        __syncthreads();
        // eliminate column j from every other row (one warp per row)
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int i = w; i < n; i += kNT / 32) {
            if (i == j) continue;
            T *ri = A + int64_t(i) * lda;
            const T f = ri[j];
            if (f == T(0)) continue;
            __syncwarp();
            const T *rj = A + int64_t(j) * lda;
            for (int c = l; c < n; c += 32) ri[c] = (c == j ? T(0) : ri[c]) - f * rj[c];
        }
        __syncthreads();
    }
    __syncthreads();
    if (!ok) return false;
    // undo the row interchanges as column interchanges, last first
    for (int j = n - 1; j >= 0; --j) {
        const int p = ipiv[j];
        if (p != j)
            for (int r = threadIdx.x; r < n; r += kNT) {
                const T t = A[int64_t(r) * lda + j];
                A[int64_t(r) * lda + j] = A[int64_t(r) * lda + p];
                A[int64_t(r) * lda + p] = t;
            }
        __syncthreads();
    }
    return true;
}
}  // namespace cta
}  // namespace krr
