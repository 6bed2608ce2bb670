// Randomized HSS compression of K + lambda I (paper Section 3.1 and its
// ref. [2]: samples S = A R from the fused product plus selected entries
// of A), the ULV-type factorization and solve, iterative refinement with
// the exact fused product, and prediction (Algorithm 1 steps 2-4).
//
// Rows and columns are in two-means cluster order (Algorithm 1 step 0).
// Levels of the tree are processed bottom-up by node height; one CTA owns
// one node and works on global-memory (L2-resident) operands.
//
// Compression of a symmetric A with V = U (per node tau, rows I_tau):
//   leaf:   S_loc = A(I, I^c) R(I^c, :)  -- the off-diagonal-block sample,
//           which the fused product computes directly by skipping the
//           same-leaf pairs; R_loc = R(I, :)
//   parent: S_loc = [S_a(J_a) - B_ab Rhat_b ; S_b(J_b) - B_ab^T Rhat_a],
//           R_loc = [Rhat_a ; Rhat_b],  B_ab = A(J_a, J_b)
//   row ID of S_loc (pivoted QR of S_loc^T): skeleton J_tau, interpolation
//   matrix T (k x (m-k)), redundant rows ~= T^T x skeleton rows;
//   Rhat_tau = R_loc(J) + T R_loc(redundant).
// Adaptive sampling: a node whose rank exceeds r - p asks for more random
// columns; r doubles (up to r_max), the new columns are sampled and the
// sweep restarts.
//
// Factorization (per non-root node, local order permuted to skeleton s
// first, redundant r after; D is the node's diagonal block: K(I,I)+lambda I
// at a leaf, [Dt_a, B_ab; B_ab^T, Dt_b] at a parent):
//   the row/column operations E = [I 0; -T^T I] zero A(r, outside) exactly,
//   D'_rs = D_rs - T^T D_ss,  D'_rr = D_rr - T^T D_sr - D'_rs T,
//   LU of D'_rr,  Y = D'_rr^{-1} D'_rs,  Dt = D_ss - D'_rs^T Y  (to parent);
// the root's merged block is LU-factored.  The solve runs the same
// eliminations on the right-hand side up the tree and back-substitutes
// down.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "bigsteps.cuh"
#include "grouped.cuh"
#include "prep.cuh"

namespace krr {

int cluster(Ctx *c, const float *X, int64_t n, int d, int leaf, uint64_t seed, int32_t *perm_out,
            std::vector<int32_t> &tb, std::vector<int32_t> &te, std::vector<int32_t> &tl, std::vector<int32_t> &tr,
            std::vector<int32_t> &tp, std::vector<int32_t> &tv, const std::vector<int64_t> *segments, int method);

namespace {

constexpr int kHoldOut = 16;  // sample columns held out of each ID for its error test
constexpr double kTestFactor = 2.0;
constexpr int kBigNode = 384;  // levels whose largest node has at least this many rows use batched pivot steps  // held-out error allowed, relative to the in-sample error

// Per-node descriptor of one level (offsets are element offsets into the
// HSS arenas; -1 when unused).
struct NodeDesc {
    int m, k, is_leaf, leaf_begin;
    int ka, kb;          // children's ranks
    int child_a, child_b;  // node ids
    int64_t sloc;        // parent S_loc (m x r)
    int64_t skel, rhat;  // outputs (k x r, capacity m x r)
    int64_t w, rg;       // workspaces (m x r)
    int64_t tmat;        // T (k x (m-k)), capacity m*m
    int64_t piv;         // int arena, m
    int64_t rows;        // int arena, m: global row ids in local order
    int64_t jsk;         // int arena, m: skeleton global ids (first k)
    int64_t norm;        // workspace m
    int64_t bmat;        // B_ab (ka x kb) at parents
    // factorization (capacity m*m each)
    int64_t dmat, dtil, drs, drr, ymat;
    int64_t ipiv;        // int arena, m
    // solve workspaces (capacity m x nrhs_cap)
    int64_t zvec, btil, xloc;
};

template <class T>
struct Arena {
    Ctx *c = nullptr;
    DBuf<T> f;
    DBuf<int32_t> i;
};

// ------------------------------------------------------------ kernels
template <class T>
__device__ __forceinline__ T kern(const T *xa, const T *xb, int d, T inv2h2) {
    T s = T(0);
    for (int q = 0; q < d; ++q) {
        const T t = xa[q] - xb[q];
        s += t * t;
    }
    return exp(-s * inv2h2);
}

// B_ab = K(J_a, J_b) for every parent of the level.
template <class T>
__global__ void extract_b_kernel(const NodeDesc *nd, const T *X, int d, T inv2h2, T *F, const int32_t *I,
                                 const NodeDesc *all) {
    const NodeDesc &N = nd[blockIdx.x];
    if (N.is_leaf) return;
    const NodeDesc &A = all[N.child_a], &B = all[N.child_b];
    const int ka = A.k, kb = B.k;
    // gridDim.y CTAs share a node (the top levels have few, large nodes)
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < ka * kb; e += gridDim.y * blockDim.x) {
        const int a = e / kb, b = e % kb;
        const int ia = I[A.jsk + a], ib = I[B.jsk + b];
        F[N.bmat + e] = kern(X + int64_t(ia) * d, X + int64_t(ib) * d, d, inv2h2);
    }
}

// Parents: the children's skeleton samples stacked into S_loc, and the
// global ids of the local rows.  The subtraction of B R-hat follows as a
// grouped GEMM over the whole level.
template <class T>
__global__ void parent_sloc_kernel(const NodeDesc *nd, const NodeDesc *all, int r, T *F, int32_t *I) {
    const NodeDesc &N = nd[blockIdx.x];
    if (N.is_leaf) return;
    const NodeDesc &A = all[N.child_a], &B = all[N.child_b];
    const int ka = A.k, kb = B.k;
    T *Sl = F + N.sloc;
    // gridDim.y CTAs share a node (the top levels have few, large nodes)
    const int64_t t0 = int64_t(blockIdx.y) * blockDim.x + threadIdx.x, step = int64_t(gridDim.y) * blockDim.x;
    // four loads in flight per thread before its stores
    const int64_t tot = int64_t(ka + kb) * r, na = int64_t(ka) * r;
    for (int64_t e0 = t0; e0 < tot; e0 += 4 * step) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t e = e0 + u * step;
            if (e < tot) v[u] = e < na ? F[A.skel + e] : F[B.skel + (e - na)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e0 + u * step < tot) Sl[e0 + u * step] = v[u];
    }
    for (int64_t a = t0; a < ka; a += step) I[N.rows + a] = I[A.jsk + a];
    for (int64_t a = t0; a < kb; a += step) I[N.rows + ka + a] = I[B.jsk + a];
}

// Row ID of every node's S_loc (Householder QR with column pivoting of
// S_loc^T on a copy), its held-out test, the skeleton ids and samples, and
// R_loc gathered in pivot order (rg) with R-hat initialized to its first k
// rows; R-hat += T R_loc(redundant) follows as a grouped GEMM.
template <class T>
__global__ void __launch_bounds__(cta::kNT) id_kernel(NodeDesc *nd, const NodeDesc *all, const T *S, const T *R,
                                                      int64_t ldsr, int r, T *F, int32_t *I, T eps, T eps_abs,
                                                      int kmax, int *ranks, float *test_err, DevStatus *st,
                                                      T r11_cap) {
    NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    T *W = F + N.w;
    T *Rg = F + N.rg;
    int32_t *rows = I + N.rows;
    const T *Sorig = N.is_leaf ? S + int64_t(N.leaf_begin) * ldsr : F + N.sloc;
    const int64_t lds = N.is_leaf ? ldsr : r;
    for (int64_t e = threadIdx.x; e < int64_t(m) * r; e += blockDim.x) {
        const int a = int(e / r), t = int(e % r);
        W[e] = Sorig[int64_t(a) * lds + t];
    }
    if (N.is_leaf)
        for (int a = threadIdx.x; a < m; a += blockDim.x) rows[a] = N.leaf_begin + a;
    __syncthreads();
    int32_t *piv = I + N.piv;
    // the last kHoldOut sample columns are held out of the QR and measure
    // the decomposition's error on fresh random directions
    const int rid = r - kHoldOut;
    __shared__ T s_in_err;
    const int k = cta::row_id<T>(m, rid, r, W, r, eps, eps_abs, piv, F + N.norm, F + N.tmat, kmax, &s_in_err,
                                 r11_cap);
    const T terr = cta::id_test_error<T>(m, k, W, r, F + N.tmat, rid, r);
    __syncthreads();
    if (threadIdx.x == 0) {
        N.k = k;
        ranks[blockIdx.x] = k;
        test_err[2 * blockIdx.x] = float(terr);
        test_err[2 * blockIdx.x + 1] = float(s_in_err);
    }
    for (int a = threadIdx.x; a < k; a += blockDim.x) I[N.jsk + a] = rows[piv[a]];
    for (int64_t e = threadIdx.x; e < int64_t(k) * r; e += blockDim.x) {
        const int a = int(e / r), t = int(e % r);
        F[N.skel + e] = Sorig[int64_t(piv[a]) * lds + t];
    }
    // R_loc rows in pivot order: R(I) at a leaf, [Rhat_a; Rhat_b] at a parent
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    T *Rh = F + N.rhat;
    for (int64_t e = threadIdx.x; e < int64_t(m) * r; e += blockDim.x) {
        const int a = int(e / r), t = int(e % r);
        const int src = piv[a];
        T v;
        if (N.is_leaf) v = R[(int64_t(N.leaf_begin) + src) * ldsr + t];
        else if (src < A->k) v = F[A->rhat + int64_t(src) * r + t];
        else v = F[B->rhat + int64_t(src - A->k) * r + t];
        Rg[e] = v;
        if (a < k) Rh[e] = v;
    }
}

// Large-node path of the row ID, step 1: S_loc copied into W (ld r), row
// ids of leaves.  The QR then runs as batched pivot-step launches.
template <class T>
__global__ void __launch_bounds__(cta::kNT) id_prep_kernel(const NodeDesc *nd, const T *S, int64_t ldsr, int r, T *F,
                                                           int32_t *I) {
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const T *Sorig = N.is_leaf ? S + int64_t(N.leaf_begin) * ldsr : F + N.sloc;
    const int64_t lds = N.is_leaf ? ldsr : r;
    T *W = F + N.w;
    for (int64_t e = threadIdx.x; e < int64_t(m) * r; e += blockDim.x) W[e] = Sorig[(e / r) * lds + e % r];
    if (N.is_leaf)
        for (int a = threadIdx.x; a < m; a += blockDim.x) I[N.rows + a] = N.leaf_begin + a;
}

// Row ID from the Gram matrix.  With G = S S^T over the sample columns
// that enter the decomposition (rows of S_loc; G in the node's drr slot), a
// Cholesky factorization of G with diagonal pivoting picks at each step the
// row with the largest remaining squared norm, exactly the row a
// column-pivoted QR of S^T would pick, and its factor L is R^T of that QR
// (P G P^T = L L^T = R^T R).  So the rank rule (|R_jj| > eps |R_11| and
// > eps_abs), T = R11^{-1} R12 and the in-sample error
// sqrt(remaining diagonal / trace G) are those of the QR, from O(m^2) data
// instead of O(m r).  The kernels below run it blocked; these are their
// CTA-wide reductions for NT threads.
template <class T, int NT>
__device__ void argmax_nt(T &val, int &idx) {
    __shared__ T sv[NT / 32];
    __shared__ int si[NT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, val, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = val; si[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x < 32) {
        val = threadIdx.x < NT / 32 ? sv[threadIdx.x] : T(-1);
        idx = threadIdx.x < NT / 32 ? si[threadIdx.x] : 0x7fffffff;
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

template <class T, int NT>
__device__ T sum_nt(T v) {
    __shared__ T sh[NT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    for (int w = 0; w < NT / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Blocked form (LAPACK-style, right-looking between panels): panels of
// kPanel pivots run in one CTA per node (gram_panel_kernel), each followed
// by the update G -= L_p L_p^T of the panel's columns as one grouped GEMM
// over all nodes of the level.  Nothing is interchanged: rows keep their
// local index q, L is stored column-major by q (L(q, t) at w[t m + q]),
// a chosen row's remaining diagonal becomes -inf, and piv lists the chosen
// rows in pivot order (the rest follow in index order at the end).
constexpr int kPanel = 32;

template <class T>
struct GramState {
    int k, done;
    T r11, tot0;
};

template <class T, int NT>
__global__ void __launch_bounds__(NT) gram_init_kernel(const NodeDesc *nd, T *F, int32_t *I, GramState<T> *st) {
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const T *G = F + N.drr;
    T *d = F + N.norm;
    T tot = T(0);
    for (int i = threadIdx.x; i < m; i += NT) {
        if (N.is_leaf) I[N.rows + i] = N.leaf_begin + i;
        const T g = G[int64_t(i) * m + i];
        d[i] = g > T(0) ? g : T(0);
        tot += d[i];
    }
    tot = sum_nt<T, NT>(tot);
    if (threadIdx.x == 0) {
        st[blockIdx.x].k = 0;
        st[blockIdx.x].done = m == 0 ? 1 : 0;
        st[blockIdx.x].r11 = T(0);
        st[blockIdx.x].tot0 = tot;
    }
}

// Pivots [j0, j0 + kPanel) of every unfinished node: column j of L is
// (G(q, p_j) - sum_{t in [j0, j)} L(q, t) L(p_j, t)) / L(p_j, j) over the
// rows not yet chosen, G already updated by the earlier panels.  Stops at
// the rank rule or at jmax.  The remaining diagonal d lives in shared
// memory for the panel, and so do the panel's columns of L when they fit
// (ldl >= m rows; else they are read from global memory); row p_j of the
// panel is broadcast through shared memory.  Rows already chosen get 0 in
// the panel's later columns.  Three CTA barriers per pivot.
template <class T, int NT>
__global__ void __launch_bounds__(NT) gram_panel_kernel(const NodeDesc *nd, T *F, int32_t *I, GramState<T> *st,
                                                        int j0, int rid, int kmax, T eps, T eps_abs, T r11_cap,
                                                        int ldl) {
    extern __shared__ __align__(16) unsigned char gp_smem[];
    __shared__ T prow[kPanel];
    GramState<T> &S = st[blockIdx.x];
    if (S.done) return;
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const T *A = F + N.drr;
    T *Lc = F + N.w;
    T *dg = F + N.norm;
    int32_t *piv = I + N.piv;
    T *ds = reinterpret_cast<T *>(gp_smem);       // m entries
    T *Ls = ds + ((ldl > 0 ? ldl : m) + 3) / 4 * 4;  // kPanel x ldl (column t at Ls + t ldl)
    const bool in_sm = ldl >= m;
    const int jmax = min(min(m, rid), kmax);
    const int jend = min(j0 + kPanel, jmax);
    for (int q = threadIdx.x; q < m; q += NT) ds[q] = dg[q];
    __syncthreads();
    T r11 = S.r11;
    int j = j0;
    for (; j < jend; ++j) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int q = threadIdx.x; q < m; q += NT)
            if (ds[q] > best) { best = ds[q]; bi = q; }
        argmax_nt<T, NT>(best, bi);  // synchronizes
        const T nrm = sqrt(best > T(0) ? best : T(0));
        if (j == 0) r11 = nrm < r11_cap ? nrm : r11_cap;
        if (!(nrm > eps * r11) || !(nrm > eps_abs)) break;
        const int p = bi;
        const T inv = T(1) / nrm;
        const int nt = j - j0;
        if (threadIdx.x < nt) prow[threadIdx.x] = in_sm ? Ls[threadIdx.x * ldl + p] : Lc[int64_t(j0 + threadIdx.x) * m + p];
        __syncthreads();
        const T *gp = A + int64_t(p) * m;  // row p of the symmetric G: column p
        for (int q = threadIdx.x; q < m; q += NT) {
            T v;
            if (q == p) {
                v = nrm;
                ds[q] = -INFINITY;
            } else if (!(ds[q] >= T(0))) {
                v = T(0);  // already chosen
            } else {
                T sacc = gp[q];
                if (in_sm)
                    for (int t = 0; t < nt; ++t) sacc -= Ls[t * ldl + q] * prow[t];
                else
                    for (int t = 0; t < nt; ++t) sacc -= Lc[int64_t(j0 + t) * m + q] * prow[t];
                v = sacc * inv;
                const T dq = ds[q] - v * v;
                ds[q] = dq > T(0) ? dq : T(0);
            }
            if (in_sm) Ls[nt * ldl + q] = v;
            else Lc[int64_t(j) * m + q] = v;
        }
        if (threadIdx.x == 0) piv[j] = p;
        __syncthreads();
    }
    // the panel's columns of L and the remaining diagonal back to global memory
    if (in_sm)
        for (int t = 0; t < j - j0; ++t)
            for (int q = threadIdx.x; q < m; q += NT) Lc[int64_t(j0 + t) * m + q] = Ls[t * ldl + q];
    for (int q = threadIdx.x; q < m; q += NT) dg[q] = ds[q];
    if (threadIdx.x == 0) {
        S.r11 = r11;
        S.k = j;
        if (j < jend || j == jmax) S.done = 1;
    }
}

// Shared memory of gram_panel_kernel for nodes of up to mmax rows: the
// diagonal, and the panel's columns of L when all fit in 200 KB (ldl = mmax,
// else ldl = 0: L stays in global memory).
template <class T>
inline void gram_panel_smem(int mmax, int &ldl, size_t &bytes) {
    const size_t dbytes = size_t((mmax + 3) / 4 * 4) * sizeof(T);
    const size_t lbytes = size_t(kPanel) * mmax * sizeof(T);
    ldl = dbytes + lbytes <= size_t(200) * 1024 ? mmax : 0;
    bytes = dbytes + (ldl ? lbytes : 0);
}

// After the factorization, in three steps.  gram_prep_kernel: the unchosen
// rows appended to piv, the skeleton ids; gram_copy_kernel (several CTAs
// per node): skeleton samples, R_loc in pivot order and R-hat's first rows,
// L gathered into pivot order (m x k row-major in the dmat slot) and the
// right-hand side L21^T in T's place.  Then T =
// R11^{-1} R12 (R = L^T) by blocked back substitution: per block of
// kTrsmBlock rows from the bottom, the triangular diagonal block in one CTA
// per node (gram_trsm_diag_kernel) and the update of the rows above as a
// grouped GEMM.  gram_test_kernel: in-sample and held-out errors.
constexpr int kTrsmBlock = 64;

template <class T, int NT>
__global__ void __launch_bounds__(NT) gram_prep_kernel(const NodeDesc *nd, const GramState<T> *st, const T *F,
                                                       int32_t *I) {
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const int k = st[blockIdx.x].k;
    const T *d = F + N.norm;
    int32_t *piv = I + N.piv;
    int32_t *pos = I + N.ipiv;
    const int32_t *rows = I + N.rows;
    if (threadIdx.x == 0) {
        int a = k;
        for (int q = 0; q < m; ++q)
            if (d[q] >= T(0)) piv[a++] = q;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < m; a += NT) pos[piv[a]] = a;
    for (int a = threadIdx.x; a < k; a += NT) I[N.jsk + a] = rows[piv[a]];
}

// The node's data in pivot order, gridDim.y CTAs per node: skeleton
// samples, R_loc (and R-hat's first k rows), L in pivot order (Lp, lower
// part) and T's initial value L21^T, read straight from L through the
// pivot order (T(a, c) = L(piv[k + c], a)).
template <class T>
__global__ void __launch_bounds__(256) gram_copy_kernel(const NodeDesc *nd, const NodeDesc *all,
                                                        const GramState<T> *st, const T *S, const T *R, int64_t ldsr,
                                                        int r, T *F, const int32_t *I) {
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const int k = st[blockIdx.x].k;
    const T *Lc = F + N.w;
    const int32_t *piv = I + N.piv;
    const int32_t *pos = I + N.ipiv;
    const int64_t t0 = int64_t(blockIdx.y) * blockDim.x + threadIdx.x, step = int64_t(gridDim.y) * blockDim.x;
    // Each thread gathers four elements before it stores any (a store
    // between two loads would order the second load after it), so four
    // loads are in flight per thread.
    auto copy4 = [&](int64_t total, auto load, auto store) {
        for (int64_t e0 = t0; e0 < total; e0 += 4 * step) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + u * step < total) v[u] = load(e0 + u * step);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e0 + u * step < total) store(e0 + u * step, v[u]);
        }
    };
    const T *Sorig = N.is_leaf ? S + int64_t(N.leaf_begin) * ldsr : F + N.sloc;
    const int64_t lds = N.is_leaf ? ldsr : r;
    T *Sk = F + N.skel;
    copy4(int64_t(k) * r, [&](int64_t e) { return Sorig[int64_t(piv[e / r]) * lds + e % r]; },
          [&](int64_t e, T v) { Sk[e] = v; });
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    T *Rg = F + N.rg;
    T *Rh = F + N.rhat;
    copy4(int64_t(m) * r,
          [&](int64_t e) {
              const int a = int(e / r), t = int(e % r);
              const int src = piv[a];
              if (N.is_leaf) return R[(int64_t(N.leaf_begin) + src) * ldsr + t];
              if (src < A->k) return F[A->rhat + int64_t(src) * r + t];
              return F[B->rhat + int64_t(src - A->k) * r + t];
          },
          [&](int64_t e, T v) {
              Rg[e] = v;
              if (e / r < k) Rh[e] = v;
          });
    T *Lp = F + N.dmat;
    copy4(int64_t(m) * k,  // reads of Lc coalesced over q
          [&](int64_t e) {
              const int b = int(e / m), a = pos[int(e % m)];
              return (b <= a) ? Lc[e] : T(0);
          },
          [&](int64_t e, T v) { Lp[int64_t(pos[int(e % m)]) * k + e / m] = v; });
    T *Tm = F + N.tmat;
    const int nr = m - k;
    if (nr > 0)
        copy4(int64_t(k) * nr, [&](int64_t e) { return Lc[(e / nr) * m + piv[k + int(e % nr)]]; },
              [&](int64_t e, T v) { Tm[e] = v; });
}

// Rows [a0, min(a1, k)) of T: back substitution with the diagonal block of
// L11^T.  The columns of T are independent: gridDim.y CTAs of 128 threads
// per node, one column per thread held in registers, the diagonal block of
// L staged in shared memory (zero outside the block, so the fixed-size
// loops add exact zeros past its end).
constexpr int kTrsmCols = 128;

template <class T>
__global__ void __launch_bounds__(kTrsmCols) gram_trsm_diag_kernel(const NodeDesc *nd, const GramState<T> *st, T *F,
                                                                   int a0, int a1) {
    const NodeDesc &N = nd[blockIdx.x];
    const int k = st[blockIdx.x].k;
    const int hi = min(a1, k);
    const int nr = N.m - k;
    const int c0 = int(blockIdx.y) * kTrsmCols;
    if (hi <= a0 || c0 >= nr) return;
    const int nb = hi - a0;
    __shared__ T Ls[kTrsmBlock][kTrsmBlock + 1];  // Ls[b][a] = L(a0 + b, a0 + a), b >= a
    const T *Lp = F + N.dmat;
    for (int e = threadIdx.x; e < kTrsmBlock * kTrsmBlock; e += kTrsmCols) {
        const int b = e / kTrsmBlock, a = e % kTrsmBlock;
        Ls[b][a] = (a <= b && b < nb) ? Lp[int64_t(a0 + b) * k + a0 + a] : T(0);
    }
    __syncthreads();
    const int c = c0 + int(threadIdx.x);
    if (c >= nr) return;
    T *Tm = F + N.tmat;
    T x[kTrsmBlock];
#pragma unroll
    for (int a = 0; a < kTrsmBlock; ++a) x[a] = a < nb ? Tm[int64_t(a0 + a) * nr + c] : T(0);
#pragma unroll
    for (int a = kTrsmBlock - 1; a >= 0; --a) {
        if (a < nb) {
            T sacc = x[a];
#pragma unroll
            for (int b = a + 1; b < kTrsmBlock; ++b) sacc -= Ls[b][a] * x[b];
            x[a] = sacc / Ls[a][a];
        }
    }
#pragma unroll
    for (int a = 0; a < kTrsmBlock; ++a)
        if (a < nb) Tm[int64_t(a0 + a) * nr + c] = x[a];
}

template <class T, int NT>
__global__ void __launch_bounds__(NT) gram_test_kernel(NodeDesc *nd, const GramState<T> *st, const T *S,
                                                       int64_t ldsr, int r, T *F, const int32_t *I, int *ranks,
                                                       float *test_err) {
    NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const int rid = r - kHoldOut;
    const int k = st[blockIdx.x].k;
    const T tot0 = st[blockIdx.x].tot0;
    const T *d = F + N.norm;
    const int32_t *piv = I + N.piv;
    T rest = T(0);
    for (int q = threadIdx.x; q < m; q += NT) rest += d[q] >= T(0) ? d[q] : T(0);
    rest = sum_nt<T, NT>(rest);
    const T *Sorig = N.is_leaf ? S + int64_t(N.leaf_begin) * ldsr : F + N.sloc;
    const int64_t lds = N.is_leaf ? ldsr : r;
    const T *Sk = F + N.skel;
    const T *Tm = F + N.tmat;
    const int nr = m - k;
    const int nh = r - rid;
    T err = T(0), tot = T(0);
    for (int e = threadIdx.x; e < nr * nh; e += NT) {
        const int c = e % nr, t = rid + e / nr;
        const T v = Sorig[int64_t(piv[k + c]) * lds + t];
        tot += v * v;
        T sacc = v;
        for (int a = 0; a < k; ++a) sacc -= Tm[int64_t(a) * nr + c] * Sk[int64_t(a) * r + t];
        err += sacc * sacc;
    }
    for (int e = threadIdx.x; e < k * nh; e += NT) {
        const T v = Sk[int64_t(e / nh) * r + rid + e % nh];
        tot += v * v;
    }
    err = sum_nt<T, NT>(err);
    tot = sum_nt<T, NT>(tot);
    if (threadIdx.x == 0) {
        N.k = k;
        ranks[blockIdx.x] = k;
        test_err[2 * blockIdx.x] = float(tot > T(0) ? sqrt(err / tot) : T(0));
        test_err[2 * blockIdx.x + 1] = float(tot0 > T(0) ? sqrt(rest / tot0) : T(0));
    }
}

// Nodes that stay whole: rank 0, local rows in their natural order.
__global__ void noid_kernel(const NodeDesc *nd, int32_t *I) {
    const NodeDesc &N = nd[blockIdx.x];
    for (int a = threadIdx.x; a < N.m; a += blockDim.x) {
        I[N.piv + a] = a;
        if (N.is_leaf) I[N.rows + a] = N.leaf_begin + a;
    }
}

// Large-node path, last step: T from the QR, in-sample and held-out errors,
// skeleton ids and samples, R_loc in pivot order and R-hat's first rows.
template <class T>
__global__ void __launch_bounds__(cta::kNT) id_post_kernel(NodeDesc *nd, const NodeDesc *all, const big::QrState *qs,
                                                           const T *S, const T *R, int64_t ldsr, int r, T *F,
                                                           int32_t *I, int *ranks, float *test_err) {
    NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const int k = qs[blockIdx.x].k;
    T *W = F + N.w;
    const int rid = r - kHoldOut;
    cta::id_T<T>(m, k, W, r, F + N.tmat);
    __syncthreads();
    T rest = T(0);
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) rest += F[N.norm + i];
    rest = cta::sum_block(rest);
    const double tot0 = qs[blockIdx.x].tot0;
    const T in_err = tot0 > 0 ? T(sqrt(double(rest) / tot0)) : T(0);
    const T terr = cta::id_test_error<T>(m, k, W, r, F + N.tmat, rid, r);
    if (threadIdx.x == 0) {
        N.k = k;
        ranks[blockIdx.x] = k;
        test_err[2 * blockIdx.x] = float(terr);
        test_err[2 * blockIdx.x + 1] = float(in_err);
    }
    const int32_t *piv = I + N.piv;
    const int32_t *rows = I + N.rows;
    const T *Sorig = N.is_leaf ? S + int64_t(N.leaf_begin) * ldsr : F + N.sloc;
    const int64_t lds = N.is_leaf ? ldsr : r;
    for (int a = threadIdx.x; a < k; a += blockDim.x) I[N.jsk + a] = rows[piv[a]];
    for (int64_t e = threadIdx.x; e < int64_t(k) * r; e += blockDim.x)
        F[N.skel + e] = Sorig[int64_t(piv[e / r]) * lds + e % r];
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    T *Rg = F + N.rg;
    T *Rh = F + N.rhat;
    __syncthreads();  // the Householder vector lived in rg
    for (int64_t e = threadIdx.x; e < int64_t(m) * r; e += blockDim.x) {
        const int a = int(e / r), t = int(e % r);
        const int src = piv[a];
        T v;
        if (N.is_leaf) v = R[(int64_t(N.leaf_begin) + src) * ldsr + t];
        else if (src < A->k) v = F[A->rhat + int64_t(src) * r + t];
        else v = F[B->rhat + int64_t(src - A->k) * r + t];
        Rg[e] = v;
        if (a < k) Rh[e] = v;
    }
}

// Diagonal block of a node in skeleton-first order: K(I,I) + lambda I at a
// leaf, [Dt_a, B; B^T, Dt_b] at a parent.  Writes D_ss -> dtil, D_rs ->
// dmat (kept) and drs (to be updated), D_rr -> drr; the root's whole
// block (local order) -> drr.
template <class T>
__global__ void __launch_bounds__(cta::kNT) factor_build_kernel(const NodeDesc *nd, const NodeDesc *all, const T *X,
                                                                int d, T inv2h2, T lambda, T *F, const int32_t *I,
                                                                int is_root) {
    const NodeDesc &N = nd[blockIdx.x];
    const int m = N.m;
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    auto dval = [&](int a, int b) -> T {
        if (N.is_leaf) {
            if (a == b) return T(1) + lambda;
            return kern(X + (N.leaf_begin + int64_t(a)) * d, X + (N.leaf_begin + int64_t(b)) * d, d, inv2h2);
        }
        const int ka = A->k, kb = B->k;
        if (a < ka && b < ka) return F[A->dtil + int64_t(a) * ka + b];
        if (a >= ka && b >= ka) return F[B->dtil + int64_t(a - ka) * kb + (b - ka)];
        if (a < ka) return F[N.bmat + int64_t(a) * kb + (b - ka)];
        return F[N.bmat + int64_t(b) * kb + (a - ka)];
    };
    // gridDim.y CTAs share a node (the top levels have few, large nodes)
    const int64_t t0 = int64_t(blockIdx.y) * blockDim.x + threadIdx.x, step = int64_t(gridDim.y) * blockDim.x;
    if (is_root) {
        for (int64_t e = t0; e < int64_t(m) * m; e += step) F[N.drr + e] = dval(int(e / m), int(e % m));
        return;
    }
    const int k = N.k, nr = m - k;
    const int32_t *piv = I + N.piv;
    for (int64_t e = t0; e < int64_t(k) * k; e += step)
        F[N.dtil + e] = dval(piv[e / k], piv[e % k]);
    for (int64_t e = t0; e < int64_t(nr) * k; e += step) {
        const T v = dval(piv[k + e / k], piv[e % k]);
        F[N.dmat + e] = v;
        F[N.drs + e] = v;
    }
    for (int64_t e = t0; e < int64_t(nr) * nr; e += step)
        F[N.drr + e] = dval(piv[k + e / nr], piv[k + e % nr]);
}

// drr <- drr^{-1} (redundant block, or the root's whole block).
template <class T>
__global__ void __launch_bounds__(cta::kNT) invert_kernel(const NodeDesc *nd, T *F, int32_t *I, int is_root,
                                                          DevStatus *st) {
    const NodeDesc &N = nd[blockIdx.x];
    const int n = is_root ? N.m : N.m - N.k;
    if (n <= 0) return;
    if (!cta::gj_inverse<T>(n, F + N.drr, n, I + N.ipiv) && threadIdx.x == 0) dev_fail(st, KRR_ERR_SINGULAR, 201);
}

// Up-sweep, step 1 (one CTA per node): the node's local right-hand side
// (rows of y at a leaf, [btil_a; btil_b] at a parent) split in pivot order:
// skeleton rows -> btil (k x nrhs), redundant rows -> xloc (nr x nrhs).
// The root's whole block goes to zvec.  The eliminations follow as
// grouped GEMMs over the level:
//   xloc -= T^T btil ; zvec = D'_rr^{-1} xloc ; btil -= D'_rs^T zvec
// and at the root xloc = D^{-1} zvec.  The bodies below take the node and
// the part (y of ny CTAs) a CTA handles, so the kernels (one CTA per part)
// and the one-launch sweep share them; vectors another CTA wrote earlier in
// the sweep are read through L2 (__ldcg), never a stale L1 line.
template <class T>
__device__ __forceinline__ void solve_gather_body(const NodeDesc &N, const NodeDesc *all, const T *yperm,
                                                  int64_t ldy, int nrhs, T *F, const int32_t *I, int is_root, int y,
                                                  int ny) {
    const int m = N.m, k = is_root ? 0 : N.k;
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    const int32_t *piv = I + N.piv;
    for (int64_t e = int64_t(y) * blockDim.x + threadIdx.x; e < int64_t(m) * nrhs; e += int64_t(ny) * blockDim.x) {
        const int a = int(e / nrhs), c = int(e % nrhs);
        const int src = is_root ? a : piv[a];
        T v;
        if (N.is_leaf) v = yperm[(N.leaf_begin + int64_t(src)) * ldy + c];
        else if (src < A->k) v = __ldcg(F + A->btil + int64_t(src) * nrhs + c);
        else v = __ldcg(F + B->btil + int64_t(src - A->k) * nrhs + c);
        if (is_root) F[N.zvec + e] = v;
        else if (a < k) F[N.btil + int64_t(a) * nrhs + c] = v;
        else F[N.xloc + int64_t(a - k) * nrhs + c] = v;
    }
}

template <class T>
__global__ void __launch_bounds__(cta::kNT) solve_gather_kernel(const NodeDesc *nd, const NodeDesc *all,
                                                                const T *yperm, int64_t ldy, int nrhs, T *F,
                                                                const int32_t *I, int is_root) {
    solve_gather_body<T>(nd[blockIdx.x], all, yperm, ldy, nrhs, F, I, is_root, blockIdx.y, gridDim.y);
}

// Down-sweep, last step (one CTA per node): after
//   zvec -= Y btil  (x'_r) ;  btil -= T zvec  (x_s)
// the local x in the node's original row order -> xloc; leaves write
// their rows of the solution.
template <class T>
__device__ __forceinline__ void solve_place_body(const NodeDesc &N, int nrhs, T *F, const int32_t *I, T *xperm,
                                                 int64_t ldx, int y, int ny) {
    const int m = N.m, k = N.k;
    const int32_t *piv = I + N.piv;
    for (int64_t e = int64_t(y) * blockDim.x + threadIdx.x; e < int64_t(m) * nrhs; e += int64_t(ny) * blockDim.x) {
        const int a = int(e / nrhs), c = int(e % nrhs);
        const T v = a < k ? __ldcg(F + N.btil + int64_t(a) * nrhs + c) : __ldcg(F + N.zvec + int64_t(a - k) * nrhs + c);
        const int dst = piv[a];
        if (N.is_leaf) xperm[(N.leaf_begin + int64_t(dst)) * ldx + c] = v;
        else F[N.xloc + int64_t(dst) * nrhs + c] = v;
    }
}

template <class T>
__global__ void __launch_bounds__(cta::kNT) solve_place_kernel(const NodeDesc *nd, int nrhs, T *F, const int32_t *I,
                                                               T *xperm, int64_t ldx) {
    solve_place_body<T>(nd[blockIdx.x], nrhs, F, I, xperm, ldx, blockIdx.y, gridDim.y);
}

// Single-leaf tree: the root's solve is the answer.
template <class T>
__device__ __forceinline__ void root_leaf_out_body(const NodeDesc &N, int nrhs, const T *F, T *xperm, int64_t ldx,
                                                   int y, int ny) {
    for (int64_t e = int64_t(y) * blockDim.x + threadIdx.x; e < int64_t(N.m) * nrhs; e += int64_t(ny) * blockDim.x) {
        const int a = int(e / nrhs), c = int(e % nrhs);
        xperm[(N.leaf_begin + int64_t(a)) * ldx + c] = __ldcg(F + N.xloc + e);
    }
}

template <class T>
__global__ void root_leaf_out_kernel(const NodeDesc *nd, int nrhs, const T *F, T *xperm, int64_t ldx) {
    root_leaf_out_body<T>(nd[0], nrhs, F, xperm, ldx, 0, 1);
}

// Hand the parent's local x to its children (x'_s slots).
template <class T>
__device__ __forceinline__ void scatter_down_body(const NodeDesc &N, const NodeDesc *all, int nrhs, T *F, int y,
                                                  int ny) {
    if (N.is_leaf) return;
    const NodeDesc &A = all[N.child_a], &B = all[N.child_b];
    const T *x = F + N.xloc;
    const int64_t e0 = int64_t(y) * blockDim.x + threadIdx.x, step = int64_t(ny) * blockDim.x;
    for (int64_t e = e0; e < int64_t(A.k) * nrhs; e += step) F[A.btil + e] = __ldcg(x + e);
    for (int64_t e = e0; e < int64_t(B.k) * nrhs; e += step) F[B.btil + e] = __ldcg(x + int64_t(A.k) * nrhs + e);
}

template <class T>
__global__ void scatter_down_kernel(const NodeDesc *nd, const NodeDesc *all, int nrhs, T *F) {
    scatter_down_body<T>(nd[blockIdx.x], all, nrhs, F, blockIdx.y, gridDim.y);
}

// ------------------------------------- small nodes: one CTA per node step
// A node with m <= kFuseMax rows takes its whole up-sweep step (gather,
// x_r -= T^T b_s, z = D'_rr^{-1} x_r, b_s -= D'_rs^T z) or down-sweep step
// (z -= Y b, b -= T z, placement into the children's or the solution's
// rows) in one CTA of 256 threads, its vectors (16 columns) in shared
// memory, instead of one grid-wide phase per product.
constexpr int kFuseMax = 128;
constexpr int kFuseRhs = 16;

// out(i, :) += sign sum_j A[j lda + i] v(j, :), i < M, j < K (A stored K x M;
// v, out in shared memory, 16 columns).  Each warp takes 32 x 32 blocks of
// A: lane l reads column i0 + l of 32 consecutive rows (each row segment
// one coalesced 128-byte read, all 32 in flight at once) and sums them into
// output row i0 + l; parts added with shared-memory atomics.
template <class T>
__device__ void cta_gemv_t(const T *A, int64_t lda, int M, int K, const T *v, T *out, T sign) {
    if (M <= 0 || K <= 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = (K + 31) / 32, nitems = ((M + 31) / 32) * nkc;
    for (int item = warp; item < nitems; item += int(blockDim.x >> 5)) {
        const int i = (item / nkc) * 32 + lane, j0 = (item % nkc) * 32, jn = min(32, K - j0);
        T a[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) a[jj] = (i < M && jj < jn) ? A[int64_t(j0 + jj) * lda + i] : T(0);
        T acc[kFuseRhs];
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) acc[c] = T(0);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
            if (jj < jn)  // rows of v past K are not part of it (uniform over the warp)
#pragma unroll
                for (int c = 0; c < kFuseRhs; ++c) acc[c] += a[jj] * v[(j0 + jj) * kFuseRhs + c];
        if (i < M)
#pragma unroll
            for (int c = 0; c < kFuseRhs; ++c) atomicAdd(out + i * kFuseRhs + c, sign * acc[c]);
    }
}

// out(i, :) += sign sum_j A[i lda + j] v(j, :) (A stored M x K): each warp
// takes 32-row x 32-column blocks of A, read along rows (coalesced) into
// its own 32 x 33 tile and read back transposed; parts added with
// shared-memory atomics.
template <class T>
__device__ void cta_gemv_n(const T *A, int64_t lda, int M, int K, const T *v, T *out, T sign, T *tiles) {
    if (M <= 0 || K <= 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *tw = tiles + warp * 32 * 33;
    const int nkc = (K + 31) / 32, nitems = ((M + 31) / 32) * nkc;
    for (int item = warp; item < nitems; item += int(blockDim.x >> 5)) {
        const int r0 = (item / nkc) * 32, k0 = (item % nkc) * 32, kn = min(32, K - k0);
        // all 32 loads issued before the first shared-memory store (a store
        // through the generic pointer would otherwise order each load after
        // the previous store)
        T a[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
            a[rr] = (r0 + rr < M && lane < kn) ? A[int64_t(r0 + rr) * lda + k0 + lane] : T(0);
        __syncwarp();
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) tw[rr * 33 + lane] = a[rr];
        __syncwarp();
        T acc[kFuseRhs];
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) acc[c] = T(0);
        for (int kk = 0; kk < kn; ++kk) {
            const T a = tw[lane * 33 + kk];
#pragma unroll
            for (int c = 0; c < kFuseRhs; ++c) acc[c] += a * v[(k0 + kk) * kFuseRhs + c];
        }
        if (r0 + lane < M)
#pragma unroll
            for (int c = 0; c < kFuseRhs; ++c) atomicAdd(out + (r0 + lane) * kFuseRhs + c, sign * acc[c]);
    }
}

template <class T>
constexpr size_t fused_smem() {
    return sizeof(T) * (size_t(2) * kFuseMax * kFuseRhs + size_t(8) * 32 * 33);
}

// Up-sweep step of a small node (see solve_gather_body for the steps).
template <class T>
__device__ void fused_up_body(const NodeDesc &N, const NodeDesc *all, const T *yperm, int nrhs, T *F,
                              const int32_t *I, unsigned char *smem) {
    T *L = reinterpret_cast<T *>(smem);    // m x 16: local rhs in pivot order, skeleton rows first
    T *Z = L + kFuseMax * kFuseRhs;        // nr x 16
    T *tiles = Z + kFuseMax * kFuseRhs;    // per-warp 32 x 33
    const int m = N.m, k = N.k, nr = m - k;
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    const int32_t *piv = I + N.piv;
    __syncthreads();  // shared memory may still be read by the CTA's previous item
    for (int a = threadIdx.x; a < m; a += blockDim.x) {  // one row per thread, its loads all in flight
        const int src = piv[a];
        const T *row = N.is_leaf ? yperm + (N.leaf_begin + int64_t(src)) * nrhs
                       : src < A->k ? F + A->btil + int64_t(src) * nrhs
                                    : F + B->btil + int64_t(src - A->k) * nrhs;
        T v[kFuseRhs];
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) v[c] = c < nrhs ? __ldcg(row + c) : T(0);
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) L[a * kFuseRhs + c] = v[c];
    }
    for (int e = threadIdx.x; e < nr * kFuseRhs; e += blockDim.x) Z[e] = T(0);
    __syncthreads();
    cta_gemv_t<T>(F + N.tmat, nr, nr, k, L, L + k * kFuseRhs, T(-1));  // x_r -= T^T b_s
    __syncthreads();
    cta_gemv_n<T>(F + N.drr, nr, nr, nr, L + k * kFuseRhs, Z, T(1), tiles);  // z = D'_rr^{-1} x_r
    __syncthreads();
    cta_gemv_t<T>(F + N.drs, k, k, nr, Z, L, T(-1));  // b_s -= D'_rs^T z
    __syncthreads();
    for (int e = threadIdx.x; e < k * nrhs; e += blockDim.x) F[N.btil + e] = L[(e / nrhs) * kFuseRhs + e % nrhs];
    for (int e = threadIdx.x; e < nr * nrhs; e += blockDim.x) F[N.zvec + e] = Z[(e / nrhs) * kFuseRhs + e % nrhs];
    __syncthreads();
}

// Down-sweep step of a small node (its b set by its parent): z -= Y b,
// b -= T z, then the local x in original row order goes to the children's
// b slots (parent) or to the solution's rows (leaf).
template <class T>
__device__ void fused_down_body(const NodeDesc &N, const NodeDesc *all, int nrhs, T *F, const int32_t *I,
                                T *xperm, unsigned char *smem) {
    T *L = reinterpret_cast<T *>(smem);    // k x 16
    T *Z = L + kFuseMax * kFuseRhs;        // nr x 16
    T *tiles = Z + kFuseMax * kFuseRhs;
    const int m = N.m, k = N.k, nr = m - k;
    __syncthreads();
    for (int a = threadIdx.x; a < m; a += blockDim.x) {  // b rows then z rows, one per thread
        const T *row = a < k ? F + N.btil + int64_t(a) * nrhs : F + N.zvec + int64_t(a - k) * nrhs;
        T *dst = a < k ? L + a * kFuseRhs : Z + (a - k) * kFuseRhs;
        T v[kFuseRhs];
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) v[c] = c < nrhs ? __ldcg(row + c) : T(0);
#pragma unroll
        for (int c = 0; c < kFuseRhs; ++c) dst[c] = v[c];
    }
    __syncthreads();
    cta_gemv_n<T>(F + N.ymat, k, nr, k, L, Z, T(-1), tiles);  // z -= Y b
    __syncthreads();
    cta_gemv_n<T>(F + N.tmat, nr, k, nr, Z, L, T(-1), tiles);  // b -= T z
    __syncthreads();
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    const NodeDesc *B = N.is_leaf ? nullptr : &all[N.child_b];
    const int32_t *piv = I + N.piv;
    for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
        const int a = e / nrhs, c = e % nrhs;
        const T v = a < k ? L[a * kFuseRhs + c] : Z[(a - k) * kFuseRhs + c];
        const int dst = piv[a];
        if (N.is_leaf) xperm[(N.leaf_begin + int64_t(dst)) * nrhs + c] = v;
        else if (dst < A->k) F[A->btil + int64_t(dst) * nrhs + c] = v;
        else F[B->btil + int64_t(dst - A->k) * nrhs + c] = v;
    }
    __syncthreads();
}

// ---------------------------------------------- ULV solve in one launch
// The whole sweep (up the tree, the root, down the tree) as one persistent
// cooperative launch: a list of phases (a level's gathers, one of its
// grouped skinny products, its placements, its hand-downs), each spread
// over every CTA, separated by a grid-wide barrier.  The launch replaces
// about a hundred dependent kernel launches per solve.
enum UlvKind { kUlvGather = 0, kUlvGemm = 1, kUlvPlace = 2, kUlvScatter = 3, kUlvRootLeaf = 4 };

template <class T>
struct UlvPhase {
    const NodeDesc *fl;        // small nodes whose whole step runs first in this phase (fdir 1 up, 2 down)
    int nf, fdir;
    int kind, is_root;
    int nn, per_node;          // node phases: nn nodes x per_node parts
    const NodeDesc *dl;
    const GemmProb<T> *probs;  // product phases
    const int32_t *tp;
    int np, tiles;
    const ZeroJob<T> *z;       // gather phases: regions cleared for the level's split products
    int nz, zparts;
    int items;                 // work items of the phase
};

// Grid-wide barrier over the CTAs of a cooperative launch (all resident):
// the last CTA to arrive resets the count and advances the generation.
// The wait is bounded: past `budget` SM cycles the status latches
// KRR_ERR_TIMEOUT and the CTA leaves the sweep.
struct GridBar {
    unsigned count, gen;
};

__device__ bool grid_barrier(GridBar *b, unsigned nblocks, long long budget, DevStatus *st) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &b->gen;
        const unsigned g = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&b->count, 1u) + 1u == nblocks) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > budget) {
                    dev_fail(st, KRR_ERR_TIMEOUT, 301);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T>
__global__ void __launch_bounds__(256) ulv_sweep_kernel(const UlvPhase<T> *phases, int nph, const NodeDesc *all,
                                                        const T *yperm, T *xperm, int nrhs, T *F, const int32_t *I,
                                                        GridBar *bar, long long budget, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char ulv_smem[];
    for (int p = 0; p < nph; ++p) {
        const UlvPhase<T> &P = phases[p];
        const int nodes = P.nn * P.per_node;
        for (int i2 = blockIdx.x; i2 < P.items; i2 += gridDim.x) {
            if (i2 < P.nf) {
                if (P.fdir == 1) fused_up_body<T>(P.fl[i2], all, yperm, nrhs, F, I, ulv_smem);
                else fused_down_body<T>(P.fl[i2], all, nrhs, F, I, xperm, ulv_smem);
                continue;
            }
            const int it = i2 - P.nf;
            if (P.kind == kUlvGemm) {
                skinny_tile<T>(P.probs, P.np, it, ulv_smem, P.tp);
            } else if (it < nodes) {
                const NodeDesc &N = P.dl[it / P.per_node];
                const int y = it % P.per_node;
                if (P.kind == kUlvGather) solve_gather_body<T>(N, all, yperm, nrhs, nrhs, F, I, P.is_root, y, P.per_node);
                else if (P.kind == kUlvPlace) solve_place_body<T>(N, nrhs, F, I, xperm, nrhs, y, P.per_node);
                else if (P.kind == kUlvScatter) scatter_down_body<T>(N, all, nrhs, F, y, P.per_node);
                else root_leaf_out_body<T>(N, nrhs, F, xperm, nrhs, y, P.per_node);
            } else {  // clearing of a split product's output (gather phases)
                const int q = it - nodes;
                const ZeroJob<T> z = P.z[q / P.zparts];
                for (int64_t e = int64_t(q % P.zparts) * blockDim.x + threadIdx.x; e < int64_t(z.M) * z.N;
                     e += int64_t(P.zparts) * blockDim.x)
                    z.C[(e / z.N) * z.ldc + e % z.N] = T(0);
            }
        }
        if (p + 1 < nph && !grid_barrier(bar, gridDim.x, budget, st)) return;
    }
}

__global__ void leaf_id_kernel(int64_t n, const int32_t *begin, const int32_t *end, const int32_t *isleaf, int nn,
                               int32_t *leaf_of) {
    const int v = blockIdx.x;
    if (v >= nn || !isleaf[v]) return;
    for (int64_t i = begin[v] + threadIdx.x; i < end[v]; i += blockDim.x) leaf_of[i] = v;
}

// out(i, c) = hi(v) and lo(v): a value split into two FP16-exact parts
// (stored as float), so a tensor-core product with [hi | lo] recovers the
// FP32 precision of v.
__global__ void split16_kernel(const double *v, int64_t n, int nr, int64_t ldv, float *out, int64_t ldo) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * nr) return;
    const int64_t i = e / nr;
    const int c = int(e % nr);
    const double x = v[i * ldv + c];
    const float hi = __half2float(__double2half(x));
    const float lo = __half2float(__double2half(x - double(hi)));
    out[i * ldo + c] = hi;
    out[i * ldo + nr + c] = lo;
}

// res = y - (S_hi + S_lo) - lambda * a  (mixed) or y - S - lambda a (FP64);
// also the per-column squared norms of res and y.
template <class TS>
__global__ void residual_kernel(const double *y, int64_t ldy, const TS *S, int64_t lds, int split, const double *a,
                                int64_t lda, int64_t n, int nr, double lambda, double *res, int64_t ldr,
                                double *norms) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * nr) return;
    const int64_t i = e / nr;
    const int c = int(e % nr);
    double ka = double(S[i * lds + c]);
    if (split) ka += double(S[i * lds + nr + c]);
    const double yy = y[i * ldy + c];
    const double rr = yy - ka - lambda * a[i * lda + c];
    res[i * ldr + c] = rr;
    atomicAdd(&norms[2 * c], rr * rr);
    atomicAdd(&norms[2 * c + 1], yy * yy);
}

// out = S (+ S_lo) + lambda * V  (lambda only when V's rows are the rows of out)
template <class TS>
__global__ void combine_kernel(const TS *S, int64_t lds, int split, const double *V, int64_t ldv, double lambda,
                               int64_t n, int nr, double *out, int64_t ldo) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * nr) return;
    const int64_t i = e / nr;
    const int c = int(e % nr);
    double v = double(S[i * lds + c]);
    if (split) v += double(S[i * lds + nr + c]);
    if (lambda != 0.0) v += lambda * V[i * ldv + c];
    out[i * ldo + c] = v;
}

// dots[i][c] += sum_rows A_i(row, c) * B(row, c) for blocks A_i = A + i * bstride
// dots[i][c] += sum_row A_i(row, c) B(row, c) for the nb blocks A_i = A +
// i bstride (n x nr, row-major), blockIdx.y = i, blockIdx.z = a group of 16
// columns: each thread sums its rows in registers, the CTA reduces by warp
// shuffles, and one atomic add per column per CTA goes to memory.
__global__ void __launch_bounds__(256) multidot_kernel(const double *A, int64_t bstride, int nb, const double *B,
                                                       int64_t n, int nr, double *dots) {
    __shared__ double part[8][16];
    const int i = blockIdx.y, c0 = 16 * blockIdx.z;
    const int nc = min(16, nr - c0);
    const double *Ai = A + int64_t(i) * bstride;
    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;
    for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < n; row += int64_t(gridDim.x) * blockDim.x) {
        const double *a = Ai + row * nr + c0;
        const double *b = B + row * nr + c0;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < nc) acc[c] += a[c] * b[c];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double v = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) v += part[w][threadIdx.x];
        atomicAdd(&dots[i * nr + c0 + threadIdx.x], v);
    }
}

// W(row, c) += sign sum_i coef[i][c] * A_i(row, c)
__global__ void combo_kernel(double *W, const double *A, int64_t bstride, int nb, const double *coef, double sign,
                             int64_t n, int nr) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * nr) return;
    const int c = int(e % nr);
    double s = W[e];
    for (int i = 0; i < nb; ++i) s += (sign * coef[i * nr + c]) * A[int64_t(i) * bstride + e];
    W[e] = s;
}

// A(row, c) = B(row, c) * scale[c]
__global__ void colscale_kernel(double *A, const double *B, const double *scale, int64_t n, int nr) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n * nr) A[e] = B[e] * scale[e % nr];
}

// A(row, c) = B(row, c) / |B(:, c)| from the squared norms (0 for a zero
// column): the next Krylov vector, normalized on the device.
__global__ void colnorm_kernel(double *A, const double *B, const double *normsq, int64_t n, int nr) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * nr) return;
    const double h = sqrt(fmax(normsq[e % nr], 0.0));
    A[e] = B[e] * (h > 0 ? 1.0 / h : 0.0);
}

template <class Tin, class Tout>
__global__ void convert_kernel(const Tin *a, int64_t n, Tout *b) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n) b[e] = Tout(a[e]);
}

// X(i, :) *= s[grp[i]]  (a problem's coordinates divided by its width)
template <class T>
__global__ void scale_rows_kernel(T *X, int64_t n, int d, const int32_t *grp, const double *s) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n * d) X[e] = T(double(X[e]) * s[grp[e / d]]);
}

// dst(i, c) = src(i, c) for c < cols (strided FP32 -> FP64 columns)
__global__ void widen_cols_kernel(const float *src, int64_t lds, int64_t n, int cols, double *dst, int64_t ldd) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * cols) return;
    const int64_t i = e / cols;
    const int c = int(e % cols);
    dst[i * ldd + c] = double(src[i * lds + c]);
}

__global__ void axpy_kernel(double *a, const double *b, int64_t n) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n) a[e] += b[e];
}

}  // namespace

// ------------------------------------------------------------------ host
struct HssImpl {
    Ctx *c = nullptr;
    krr_options opt{};
    int64_t n = 0;
    int d = 0;
    // tree (postorder)
    std::vector<int32_t> tb, te, tl, tr, tp, tv;
    std::vector<int> height;
    int root = -1, H = 0;
    std::vector<std::vector<int>> by_height;  // node ids per height (root excluded from IDs)
    DBuf<int32_t> perm, leaf_of;
    DBuf<float> Xp32;     // permuted X (FP32)
    DBuf<double> Xp64;    // permuted X (FP64, plain path)
    DBuf<__half> XA, XB;  // augmented operands (mixed path)
    int kpad = 0;
    int64_t ldrt = 0;
    // samples
    int r = 0, r_cap = 0, rounds = 0;
    DBuf<float> R32, S32;
    DBuf<double> R64, S64;
    DBuf<__half> RT;
    // per-node data
    std::vector<NodeDesc> desc;  // host copy (k filled after IDs)
    DBuf<NodeDesc> ddesc;        // device copy of all nodes
    DBuf<float> F32;
    DBuf<double> F64;
    DBuf<int32_t> IA;
    int nrhs_cap = 0;
    int64_t arena_f = 0, arena_i = 0;  // elements of F32/F64 and IA in use
    bool factored = false;
    // cached solve plan (rebuilt when the factorization or nrhs changes)
    struct LevelPlan {
        DBuf<NodeDesc> dl;
        GemmPlan<float, 16> f2, f3, f4, f1, fd1, fd2;
        GemmPlan<double, 16> e2, e3, e4, e1, ed1, ed2;
        // the one-launch sweep: small nodes (one CTA per node step) and the
        // rest, whose products (sf / se: up-sweep 0-3 and down-sweep 4-5 as
        // above) and clearing jobs (ZeroJob<T>) run as grid-wide phases
        DBuf<NodeDesc> dl_small, dl_big;
        int n_small = 0, n_big = 0;
        GemmPlan<float, 16> sf[6];
        GemmPlan<double, 16> se[6];
        DBuf<unsigned char> zall;
        int nzall = 0, zmax_all = 0;
    };
    std::vector<LevelPlan> plan;
    int plan_nrhs = -1;
    // the one-launch ULV sweep: its phase list (UlvPhase<T>), barrier,
    // grid (CTAs resident at once; 0 = use the captured graph instead)
    DBuf<unsigned char> ulv_ph;
    int ulv_nph = 0, ulv_grid = -1;
    DBuf<unsigned> ulv_bar;
    DBuf<float> ws_bf, ws_xf, ws_rs, ws_sm;
    DBuf<__half> ws_rt;
    int ws_nrhs = -1;
    double lambda = 0;
    // Many independent problems in one block-diagonal system: problem p
    // owns rows [boff[p], boff[p+1]) (original and cluster order alike),
    // its coordinates are stored divided by its width bh[p] and every
    // kernel evaluation uses width 1.  nprob == 0: a single problem.
    int nprob = 0;
    std::vector<int64_t> boff;
    std::vector<double> bh;
    DBuf<int32_t> bgrp, tl_lo, tl_hi;
    DBuf<int64_t> dboff, tl_off;
    int64_t tl_tiles = 0;
    BlockDiag bd_train() const {
        BlockDiag b;
        b.grp_a = b.grp_b = bgrp.get();
        b.off_b = dboff.get();
        b.tl_lo = tl_lo.get();
        b.tl_hi = tl_hi.get();
        b.tl_off = tl_off.get();
        b.tiles = tl_tiles;
        return b;
    }
    const BlockDiag *bd_or_null(const BlockDiag &b) const { return nprob > 0 ? &b : nullptr; }
    // nodes whose rows are whole problems (a problem's root, the nodes that
    // join problems): their off-diagonal blocks are zero, so they take rank
    // 0 without an ID and are eliminated whole
    std::vector<char> top;
    bool is_top(int v) const { return !top.empty() && top[v]; }
    // IDs from the Gram matrix need eps^2 well above its rounding; tighter
    // tolerances take the QR of the samples
    bool use_gram() const { return opt.eps_c >= (f32() ? 1e-2 : 1e-5); }
    // KRR_LAMBDA_TOL: a decomposition stops only below eps_c * min(|R_11|,
    // lambda sqrt(rid)), i.e. also once the next singular value of the
    // block (a pivot is about sigma sqrt(rid) in sample units) is below
    // eps_c lambda; otherwise no cap
    double r11_cap(int rid) const {
        return (opt.flags & KRR_LAMBDA_TOL) ? lambda * std::sqrt(double(rid)) : INFINITY;
    }
    int max_rank = 0, refine_steps = 0;
    bool truncated = false;
    double max_test_err = 0;
    double t_cluster = 0, t_sample = 0, t_compress = 0, t_factor = 0, t_solve = 0;
    // tc(): kernel products on tensor cores (KRR_MIXED, KRR_MIXED_F64);
    // f32(): decompositions, factorization and ULV solve in FP32 (KRR_MIXED)
    bool tc() const { return opt.precision != KRR_FP64; }
    bool f32() const { return opt.precision == KRR_MIXED; }
    // The ULV solve as a captured CUDA graph, replayed on the context's
    // stream (valid for one plan, one pair of fixed buffers, one nrhs).
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t ulv_exec = nullptr;
    const void *g_y = nullptr, *g_x = nullptr;
    int g_nrhs = -1;
    long long g_kernels = 0;
    DBuf<double> ws_b64, ws_x64;
    void drop_graph() {
        if (ulv_exec) cudaGraphExecDestroy(ulv_exec);
        ulv_exec = nullptr;
        g_nrhs = -1;
    }
    ~HssImpl() {
        drop_graph();
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Read (and clear) the context's device status word; an error latched by a
// kernel (a wait past its limit, a zero pivot, an input out of range)
// fails the call.  Synchronizes.
// Tile list of a block-diagonal product (rows of A and columns of B split
// into the same problems, offsets offa / offb): row tile rt meets column
// tiles [lo, hi], the column range of the problems its rows belong to.
int make_tile_list(Ctx *c, const std::vector<int64_t> &offa, const std::vector<int64_t> &offb, DBuf<int32_t> &lo,
                   DBuf<int32_t> &hi, DBuf<int64_t> &off, int64_t &total) {
    const int P = int(offa.size()) - 1;
    const int64_t ma = offa[P];
    const int64_t nrt = cdiv(ma, kTcTile);
    std::vector<int32_t> hl(nrt), hh(nrt);
    std::vector<int64_t> ho(nrt + 1);
    total = 0;
    int p = 0;
    for (int64_t rt = 0; rt < nrt; ++rt) {
        const int64_t r0 = rt * kTcTile, r1 = std::min(r0 + kTcTile, ma) - 1;
        while (offa[p + 1] <= r0) ++p;
        int q = p;
        while (offa[q + 1] <= r1) ++q;
        const int64_t c0 = offb[p], c1 = offb[q + 1];
        if (c1 <= c0) return fail(KRR_ERR_INVALID_ARG, "block-diagonal product: a problem has no columns");
        hl[rt] = int32_t(c0 / kTcTile);
        hh[rt] = int32_t((c1 - 1) / kTcTile);
        ho[rt] = total;
        total += hh[rt] - hl[rt] + 1;
    }
    ho[nrt] = total;
    if (!lo.reset(c, nrt) || !hi.reset(c, nrt) || !off.reset(c, nrt + 1))
        return fail(KRR_ERR_OOM, "block-diagonal product: out of memory");
    KRR_CUDA(cudaMemcpyAsync(lo.get(), hl.data(), nrt * 4, cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaMemcpyAsync(hi.get(), hh.data(), nrt * 4, cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaMemcpyAsync(off.get(), ho.data(), (nrt + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

// Problem id of every row for row offsets off (device int32[off.back()]).
int make_groups(Ctx *c, const std::vector<int64_t> &off, DBuf<int32_t> &grp) {
    const int64_t n = off.back();
    std::vector<int32_t> h(n);
    for (size_t p = 0; p + 1 < off.size(); ++p)
        for (int64_t i = off[p]; i < off[p + 1]; ++i) h[i] = int32_t(p);
    if (!grp.reset(c, n)) return fail(KRR_ERR_OOM, "block-diagonal product: out of memory");
    KRR_CUDA(cudaMemcpyAsync(grp.get(), h.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

// Divide each problem's rows of X (device rows x d, in place) by its width.
template <class T>
int scale_by_width(Ctx *c, T *X, int64_t rows, int d, const int32_t *grp, const std::vector<double> &h) {
    std::vector<double> inv(h.size());
    for (size_t p = 0; p < h.size(); ++p) inv[p] = 1.0 / h[p];
    DBuf<double> dinv(c, inv.size());
    if (!dinv.get()) return fail(KRR_ERR_OOM, "block-diagonal product: out of memory");
    KRR_CUDA(cudaMemcpyAsync(dinv.get(), inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, c->stream));
    if (rows > 0)
        { scale_rows_kernel<T><<<unsigned(cdiv(rows * d, 256)), 256, 0, c->stream>>>(X, rows, d, grp, dinv.get()); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

int take_status(Ctx *c, const char *what) {
    DevStatus st{};
    KRR_CUDA(cudaMemcpyAsync(&st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    if (st.code != 0) {
        KRR_CUDA(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->stream));
        return fail(st.code, std::string(what) + ": device error (site " + std::to_string(st.where) + ")");
    }
    return KRR_OK;
}

// KRR_TRACE=1 in the environment: synchronize and print the time of every
// phase of every level (a diagnostic; it serializes the stream).
struct Tracer {
    bool on;
    double t;
    Ctx *c;
    explicit Tracer(Ctx *ctx) : on(std::getenv("KRR_TRACE") != nullptr), t(0), c(ctx) {
        if (on) {
            cudaStreamSynchronize(c->stream);
            t = now_ms();
        }
    }
    void mark(const char *what, int h, int nn, int mmax) {
        if (!on) return;
        cudaStreamSynchronize(c->stream);
        const double t1 = now_ms();
        std::fprintf(stderr, "[krr] %-14s h=%2d nodes=%4d mmax=%5d %9.3f ms\n", what, h, nn, mmax, t1 - t);
        t = t1;
    }
};

template <class T>
T *farena(HssImpl *H);
template <>
float *farena<float>(HssImpl *H) { return H->F32.get(); }
template <>
double *farena<double>(HssImpl *H) { return H->F64.get(); }

// Lay out the arena slots of the nodes at height h, whose m is exact once
// their children's ranks are known, after the slots already taken (running
// offsets fo, io in elements).  Capacities depend on m, r and nrhs_cap.
void layout_level(HssImpl *H, int h, int nrhs_cap, int64_t &fo, int64_t &io) {
    const int64_t r = H->r;
    for (int v : H->by_height[h]) {
        NodeDesc &N = H->desc[v];
        const int64_t m = N.m;
        auto take = [&](int64_t cnt) { const int64_t o = fo; fo += (cnt + 63) & ~int64_t(63); return o; };
        auto itake = [&](int64_t cnt) { const int64_t o = io; io += (cnt + 15) & ~int64_t(15); return o; };
        // whole-problem nodes take no ID: no sample slots beyond S_loc
        const int64_t rs = H->is_top(v) ? 0 : r;
        N.sloc = N.is_leaf ? -1 : take(m * r);
        N.skel = take(m * rs);
        N.rhat = take(m * rs);
        N.w = take(m * (H->use_gram() ? std::min(m, rs) : rs));
        N.rg = take(m * rs);
        N.tmat = take(m * m);
        N.norm = take(m);
        N.bmat = N.is_leaf ? -1 : take(int64_t(N.ka) * N.kb);
        N.dmat = take(m * m);
        N.dtil = take(m * m);
        N.drs = take(m * m);
        N.drr = take(m * m);
        N.ymat = take(m * m);
        N.zvec = take(m * nrhs_cap);
        N.btil = take(m * nrhs_cap);
        N.xloc = take(m * nrhs_cap);
        N.piv = itake(m);
        N.rows = itake(m);
        N.jsk = itake(m);
        N.ipiv = itake(m);
    }
}

// Grow an arena to hold at least `need` elements, keeping its first `used`
// elements (1.5x growth, so a sweep reallocates a few times at most).
template <class T>
int grow_arena(Ctx *c, DBuf<T> &a, int64_t used, int64_t need) {
    if (int64_t(a.n) >= need) return KRR_OK;
    const int64_t cap = std::max(need, int64_t(a.n) + int64_t(a.n) / 2);
    DBuf<T> b(c, size_t(cap));
    if (!b.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
    if (used > 0 && a.get())
        KRR_CUDA(cudaMemcpyAsync(b.get(), a.get(), size_t(used) * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    a = std::move(b);
    return KRR_OK;
}

template <class T>
int sample_columns(HssImpl *H, int c0, int c1) {
    Ctx *c = H->c;
    const int dr = c1 - c0;
    const BlockDiag bd = H->bd_train();
    if (H->tc()) {
        KRR_TRY(random_block(c, H->n, dr, c0, H->opt.seed, KRR_MIXED, H->R32.get() + c0, H->r_cap));
        KRR_TRY(transpose_half(c, H->R32.get() + c0, H->n, dr, H->r_cap, H->RT.get() + int64_t(c0) * H->ldrt,
                               int(round_up(dr, 64)), H->ldrt));
        KRR_TRY(sample_mixed_prepared(c, H->XA.get(), H->n, H->XB.get(), H->n, H->d,
                                      H->RT.get() + int64_t(c0) * H->ldrt, dr, H->ldrt, H->leaf_of.get(),
                                      H->leaf_of.get(), H->S32.get() + c0, H->r_cap, false, H->bd_or_null(bd)));
        if (!H->f32()) {  // FP64 decompositions: the new columns widened (R is FP16-exact)
            const dim3 g(unsigned(cdiv(H->n * dr, 256)));
            { widen_cols_kernel<<<g, 256, 0, c->stream>>>(H->R32.get() + c0, H->r_cap, H->n, dr, H->R64.get() + c0,
                                                         H->r_cap); ::krr::count_launch(); }
            { widen_cols_kernel<<<g, 256, 0, c->stream>>>(H->S32.get() + c0, H->r_cap, H->n, dr, H->S64.get() + c0,
                                                         H->r_cap); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        }
    } else {
        KRR_TRY(random_block(c, H->n, dr, c0, H->opt.seed, KRR_FP64, H->R64.get() + c0, H->r_cap));
        KRR_TRY(launch_sample_f64(c, H->Xp64.get(), H->n, H->Xp64.get(), H->n, H->d, H->opt.h,
                                  H->R64.get() + c0, dr, H->r_cap, H->leaf_of.get(), H->leaf_of.get(),
                                  H->S64.get() + c0, H->r_cap, H->bd_or_null(bd)));
    }
    return KRR_OK;
}

// One bottom-up ID sweep with the current r.  Returns KRR_OK and sets
// `need_more` when some node's rank exceeds r - p.
template <class T>
int id_sweep(HssImpl *H, bool &need_more, bool keep_going = false) {
    Ctx *c = H->c;
    need_more = false;
    const T *S = H->f32() ? reinterpret_cast<const T *>(H->S32.get()) : reinterpret_cast<const T *>(H->S64.get());
    const T *R = H->f32() ? reinterpret_cast<const T *>(H->R32.get()) : reinterpret_cast<const T *>(H->R64.get());
    const T inv2h2 = T(1.0 / (2.0 * H->opt.h * H->opt.h));
    const T *X = H->f32() ? reinterpret_cast<const T *>(H->Xp32.get()) : reinterpret_cast<const T *>(H->Xp64.get());
    const int kmax = H->r - kHoldOut - H->opt.p + 1;  // one past the budget: a rank there means "need more"
    // The arena is laid out level by level: a parent's m (the sum of its
    // children's ranks) is exact when its level comes, so every slot has its
    // final size and the arena grows as the sweep goes up.
    int64_t fo = 0, io = 0;
    T *F = nullptr;
    auto arena = [&](int h) -> int {
        layout_level(H, h, H->nrhs_cap, fo, io);
        if (H->f32()) {
            KRR_TRY(grow_arena(c, H->F32, H->arena_f, fo));
            F = reinterpret_cast<T *>(H->F32.get());
        } else {
            KRR_TRY(grow_arena(c, H->F64, H->arena_f, fo));
            F = reinterpret_cast<T *>(H->F64.get());
        }
        KRR_TRY(grow_arena(c, H->IA, H->arena_i, io));
        H->arena_f = fo;
        H->arena_i = io;
        return KRR_OK;
    };
    H->arena_f = H->arena_i = 0;
    if (!H->ddesc.get() && !H->ddesc.reset(c, H->desc.size())) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
    DBuf<int> dranks(c, H->desc.size());
    DBuf<float> derr(c, 2 * H->desc.size());
    if (!dranks.get() || !derr.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
    H->max_test_err = 0;
    std::vector<NodeDesc> lvdesc;
    H->max_rank = 0;
    Tracer tr(c);
    for (int h = 0; h <= H->H; ++h) {
        std::vector<int> &lv = H->by_height[h];
        // exact m for parents now that children are done
        for (int v : lv) {
            NodeDesc &N = H->desc[v];
            if (!N.is_leaf) {
                N.ka = H->desc[N.child_a].k;
                N.kb = H->desc[N.child_b].k;
                N.m = N.ka + N.kb;
            }
        }
        int nn = int(lv.size());
        if (nn == 0) continue;
        KRR_TRY(arena(h));
        KRR_CUDA(cudaMemcpyAsync(H->ddesc.get(), H->desc.data(), H->desc.size() * sizeof(NodeDesc),
                                 cudaMemcpyHostToDevice, c->stream));
        lvdesc.resize(nn);
        for (int a = 0; a < nn; ++a) lvdesc[a] = H->desc[lv[a]];
        DBuf<NodeDesc> dl(c, nn);
        if (!dl.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
        KRR_CUDA(cudaMemcpyAsync(dl.get(), lvdesc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, c->stream));
        const bool is_root_level = (h == H->H);
        // the nodes of this level that get an ID (all but the whole-problem ones)
        std::vector<int> lid;
        for (int v : lv)
            if (!H->is_top(v)) lid.push_back(v);
        // CTAs per node for the per-node copy kernels: about four waves of
        // the SMs over the level
        const unsigned per_node = unsigned(std::max(1, std::min(64, 4 * c->num_sms / std::max(nn, 1))));
        if (h > 0) {
            { extract_b_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(dl.get(), X, H->d, inv2h2, F,
                                                                                  H->IA.get(), H->ddesc.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        }
        int mmax = 0;
        for (int v : lid) mmax = std::max(mmax, H->desc[v].m);
        tr.mark("extract_b", h, nn, mmax);
        if (is_root_level) break;  // the root needs B only
        const int r = H->r;
        if (h > 0) {
            { parent_sloc_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(dl.get(), H->ddesc.get(), r, F,
                                                                                     H->IA.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            // S_a(J_a) - B_ab Rhat_b ;  S_b(J_b) - B_ab^T Rhat_a
            GemmBatch<T> gb;
            for (int v : lid) {
                const NodeDesc &N = H->desc[v];
                const NodeDesc &A = H->desc[N.child_a], &B = H->desc[N.child_b];
                T *Sl = F + N.sloc;
                gb.add(A.k, r, B.k, T(-1), F + N.bmat, B.k, false, F + B.rhat, r, false, T(1), Sl, r);
                gb.add(B.k, r, A.k, T(-1), F + N.bmat, B.k, true, F + A.rhat, r, false, T(1), Sl + int64_t(A.k) * r, r);
            }
            KRR_TRY(gb.launch(c));
            tr.mark("parent_sloc", h, nn, mmax);
        }
        if (int(lid.size()) != nn) {
            // whole-problem nodes: rank 0 without an ID; the rest of the level continues alone
            std::vector<NodeDesc> tops;
            for (int v : lv)
                if (H->is_top(v)) {
                    H->desc[v].k = 0;
                    tops.push_back(H->desc[v]);
                }
            DBuf<NodeDesc> dt(c, tops.size());
            if (!dt.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
            KRR_CUDA(cudaMemcpyAsync(dt.get(), tops.data(), tops.size() * sizeof(NodeDesc), cudaMemcpyHostToDevice,
                                     c->stream));
            { noid_kernel<<<unsigned(tops.size()), 128, 0, c->stream>>>(dt.get(), H->IA.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            nn = int(lid.size());
            if (nn == 0) continue;
            lvdesc.resize(nn);
            for (int a = 0; a < nn; ++a) lvdesc[a] = H->desc[lid[a]];
            KRR_CUDA(cudaMemcpyAsync(dl.get(), lvdesc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice,
                                     c->stream));
        }
        // The Gram form needs eps^2 well above the rounding of the Gram
        // matrix; tighter tolerances take the QR of the samples.
        const bool gram = H->use_gram();
        if (mmax == 0) {
            // every node of the level is empty (its children have rank 0)
            KRR_CUDA(cudaMemsetAsync(dranks.get(), 0, nn * sizeof(int), c->stream));
            KRR_CUDA(cudaMemsetAsync(derr.get(), 0, 2 * nn * sizeof(float), c->stream));
        } else if (gram) {
            // G = S_loc S_loc^T over the columns that enter the decomposition
            const int rid = r - kHoldOut;
            GemmBatch<T> gg;
            for (int a = 0; a < nn; ++a) {
                const NodeDesc &N = lvdesc[a];
                const T *So = N.is_leaf ? S + int64_t(N.leaf_begin) * H->r_cap : F + N.sloc;
                const int64_t lds = N.is_leaf ? H->r_cap : r;
                gg.add(N.m, N.m, rid, T(1), So, lds, false, So, lds, true, T(0), F + N.drr, N.m);
            }
            KRR_TRY(gg.launch(c));
            tr.mark("id_gram", h, nn, mmax);
            DBuf<GramState<T>> gs(c, nn);
            if (!gs.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
            const bool wide = mmax > 256;
            if (wide) { gram_init_kernel<T, 1024><<<nn, 1024, 0, c->stream>>>(dl.get(), F, H->IA.get(), gs.get()); ::krr::count_launch(); }
            else { gram_init_kernel<T, 256><<<nn, 256, 0, c->stream>>>(dl.get(), F, H->IA.get(), gs.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            const int jmax = std::min(std::min(mmax, rid), kmax);
            std::vector<GramState<T>> hs(nn);
            int ldl = 0;
            size_t psm = 0;
            gram_panel_smem<T>(mmax, ldl, psm);
            {
                static SmemLimitOnce lim1024, lim256;
                if (wide) KRR_CUDA(raise_smem_limit(lim1024, c->device, gram_panel_kernel<T, 1024>, int(psm)));
                else KRR_CUDA(raise_smem_limit(lim256, c->device, gram_panel_kernel<T, 256>, int(psm)));
            }
            // the trailing updates of every panel, uploaded once; a node that
            // has finished skips its updates on the device (its done flag)
            GemmSeq<T> pseq;
            for (int j0 = 0; j0 + kPanel < jmax; j0 += kPanel) {
                GemmBatch<T> gt;
                for (int a = 0; a < nn; ++a) {
                    const NodeDesc &N = lvdesc[a];
                    if (N.m <= j0) continue;  // rank at most m: finished by then
                    const T *Lp = F + N.w + int64_t(j0) * N.m;
                    gt.add(N.m, N.m, kPanel, T(-1), Lp, N.m, true, Lp, N.m, false, T(1), F + N.drr, N.m);
                    gt.v.back().skip = &gs.get()[a].done;
                }
                pseq.add_step(gt);
            }
            KRR_TRY(pseq.upload(c));
            for (int j0 = 0, np = 0; j0 < jmax; j0 += kPanel, ++np) {
                if (wide) { gram_panel_kernel<T, 1024><<<nn, 1024, psm, c->stream>>>(dl.get(), F, H->IA.get(), gs.get(), j0, rid, kmax, T(H->opt.eps_c), T(H->opt.eps_abs), T(H->r11_cap(rid)), ldl); ::krr::count_launch(); }
                else { gram_panel_kernel<T, 256><<<nn, 256, psm, c->stream>>>(dl.get(), F, H->IA.get(), gs.get(), j0, rid, kmax, T(H->opt.eps_c), T(H->opt.eps_abs), T(H->r11_cap(rid)), ldl); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
                if (j0 + kPanel >= jmax) break;
                // the host reads which nodes finished every fourth panel only
                if (np % 4 == 3) {
                    KRR_CUDA(cudaMemcpyAsync(hs.data(), gs.get(), nn * sizeof(GramState<T>), cudaMemcpyDeviceToHost,
                                             c->stream));
                    KRR_CUDA(cudaStreamSynchronize(c->stream));
                    bool any = false;
                    for (int a = 0; a < nn; ++a) any = any || !hs[a].done;
                    if (!any) break;
                }
                // update of the nodes still running: G -= L_p L_p^T (L_p: m x kPanel, column-major)
                KRR_TRY(pseq.launch(c, np));
            }
            tr.mark("id_panels", h, nn, mmax);
            KRR_CUDA(cudaMemcpyAsync(hs.data(), gs.get(), nn * sizeof(GramState<T>), cudaMemcpyDeviceToHost,
                                     c->stream));
            KRR_CUDA(cudaStreamSynchronize(c->stream));
            { gram_prep_kernel<T, 256><<<nn, 256, 0, c->stream>>>(dl.get(), gs.get(), F, H->IA.get()); ::krr::count_launch(); }
            { gram_copy_kernel<T><<<dim3(nn, per_node), 256, 0, c->stream>>>(dl.get(), H->ddesc.get(), gs.get(), S, R,
                                                                             H->r_cap, r, F, H->IA.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            int kmx = 0, nrmx = 0;
            for (int a = 0; a < nn; ++a) {
                kmx = std::max(kmx, hs[a].k);
                nrmx = std::max(nrmx, lvdesc[a].m - hs[a].k);
            }
            const unsigned tcb = unsigned(std::max<int64_t>(1, cdiv(nrmx, kTrsmCols)));
            // the update products of every block step, uploaded once
            GemmSeq<T> useq;
            for (int a1 = int(round_up(kmx, kTrsmBlock)); a1 > kTrsmBlock; a1 -= kTrsmBlock) {
                const int a0 = a1 - kTrsmBlock;
                // rows [0, a0) of T -= (L(a0:a1, 0:a0))^T T(a0:a1, :)
                GemmBatch<T> gu;
                for (int a = 0; a < nn; ++a) {
                    const NodeDesc &N = lvdesc[a];
                    const int k = hs[a].k, nr = N.m - k;
                    const int hi = std::min(a1, k);
                    if (hi <= a0 || nr <= 0) continue;
                    gu.add(a0, nr, hi - a0, T(-1), F + N.dmat + int64_t(a0) * k, k, true,
                           F + N.tmat + int64_t(a0) * nr, nr, false, T(1), F + N.tmat, nr);
                }
                useq.add_step(gu);
            }
            KRR_TRY(useq.upload(c));
            int step = 0;
            for (int a1 = int(round_up(kmx, kTrsmBlock)); a1 > 0; a1 -= kTrsmBlock, ++step) {
                const int a0 = a1 - kTrsmBlock;
                { gram_trsm_diag_kernel<T><<<dim3(nn, tcb), kTrsmCols, 0, c->stream>>>(dl.get(), gs.get(), F, a0, a1); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
                if (a0 == 0) break;
                KRR_TRY(useq.launch(c, step));
            }
            tr.mark("id_trsm", h, nn, mmax);
            if (wide) { gram_test_kernel<T, 1024><<<nn, 1024, 0, c->stream>>>(dl.get(), gs.get(), S, H->r_cap, r, F, H->IA.get(), dranks.get(), derr.get()); ::krr::count_launch(); }
            else { gram_test_kernel<T, 256><<<nn, 256, 0, c->stream>>>(dl.get(), gs.get(), S, H->r_cap, r, F, H->IA.get(), dranks.get(), derr.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        } else if (mmax < kBigNode && nn >= c->num_sms) {
            const size_t smem = size_t(r) * sizeof(T);
            static SmemLimitOnce smem_limit;
            KRR_CUDA(raise_smem_limit(smem_limit, c->device, id_kernel<T>, 96 * 1024));
            { id_kernel<T><<<nn, cta::kNT, smem, c->stream>>>(dl.get(), H->ddesc.get(), S, R, H->r_cap, r, F,
                                                              H->IA.get(), T(H->opt.eps_c), T(H->opt.eps_abs), kmax,
                                                              dranks.get(), derr.get(), c->status,
                                                              T(H->r11_cap(r - kHoldOut))); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        } else {
            // large nodes: the pivoted QR as batched pivot-step launches
            { id_prep_kernel<T><<<nn, cta::kNT, 0, c->stream>>>(dl.get(), S, H->r_cap, r, F, H->IA.get()); ::krr::count_launch(); }
            std::vector<big::QrItem> qi(nn);
            for (int a = 0; a < nn; ++a) {
                const NodeDesc &N = lvdesc[a];
                qi[a] = big::QrItem{N.w, N.norm, N.rg, N.piv, N.m, r - kHoldOut, r, kmax};
            }
            DBuf<big::QrItem> dqi(c, nn);
            DBuf<big::QrState> dqs(c, nn);
            if (!dqi.get() || !dqs.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
            KRR_CUDA(cudaMemcpyAsync(dqi.get(), qi.data(), nn * sizeof(big::QrItem), cudaMemcpyHostToDevice, c->stream));
            KRR_CUDA(cudaMemsetAsync(dqs.get(), 0, nn * sizeof(big::QrState), c->stream));
            const dim3 g(unsigned(cdiv(mmax, big::kRowsPerBlock)), unsigned(nn));
            { big::qr_init_kernel<T><<<g, 256, 0, c->stream>>>(dqi.get(), dqs.get(), F, H->IA.get()); ::krr::count_launch(); }
            const int jmax = std::min(std::min(mmax, r - kHoldOut), kmax);
            std::vector<big::QrState> hs(nn);
            for (int j = 0; j < jmax; ++j) {
                { big::qr_pivot_kernel<T><<<nn, 256, 0, c->stream>>>(dqi.get(), dqs.get(), F, H->IA.get(), j,
                                                                     H->opt.eps_c, H->opt.eps_abs, H->r11_cap(r - kHoldOut)); ::krr::count_launch(); }
                { big::qr_apply_kernel<T><<<g, 256, 0, c->stream>>>(dqi.get(), dqs.get(), F, j); ::krr::count_launch(); }
                if ((j & 15) == 15) {  // stop early once every node has found its rank
                    KRR_CUDA(cudaMemcpyAsync(hs.data(), dqs.get(), nn * sizeof(big::QrState), cudaMemcpyDeviceToHost,
                                             c->stream));
                    KRR_CUDA(cudaStreamSynchronize(c->stream));
                    bool all = true;
                    for (const big::QrState &q : hs) all = all && q.done;
                    if (all) break;
                }
            }
            // nodes still running at jmax stop there
            { big::qr_pivot_kernel<T><<<nn, 256, 0, c->stream>>>(dqi.get(), dqs.get(), F, H->IA.get(), jmax,
                                                                 H->opt.eps_c, H->opt.eps_abs, H->r11_cap(r - kHoldOut)); ::krr::count_launch(); }
            { id_post_kernel<T><<<nn, cta::kNT, 0, c->stream>>>(dl.get(), H->ddesc.get(), dqs.get(), S, R, H->r_cap,
                                                                r, F, H->IA.get(), dranks.get(), derr.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        }
        tr.mark("id", h, nn, mmax);
        std::vector<int> hr(nn);
        std::vector<float> he(2 * nn);
        KRR_CUDA(cudaMemcpyAsync(hr.data(), dranks.get(), nn * 4, cudaMemcpyDeviceToHost, c->stream));
        KRR_CUDA(cudaMemcpyAsync(he.data(), derr.get(), 2 * nn * 4, cudaMemcpyDeviceToHost, c->stream));
        KRR_CUDA(cudaStreamSynchronize(c->stream));
        for (int a = 0; a < nn; ++a) {
            H->desc[lid[a]].k = hr[a];
            H->max_rank = std::max(H->max_rank, hr[a]);
            const double e_test = he[2 * a], e_in = he[2 * a + 1];
            H->max_test_err = std::max(H->max_test_err, e_test);
            if (hr[a] > H->r - kHoldOut - H->opt.p) need_more = true;
            // under-sampled: the decomposition fits the sampled directions
            // markedly better than fresh ones
            if (e_test > kTestFactor * std::max(e_in, H->opt.eps_c)) need_more = true;
        }
        // a level that asks for more samples ends the sweep, unless this is
        // the last round allowed (ranks then stay at the budget)
        if (need_more && !keep_going) return KRR_OK;
        {
            // R-hat += T R_loc(redundant)
            GemmBatch<T> gb;
            for (int v : lid) {
                const NodeDesc &N = H->desc[v];
                const int k = N.k, nr = N.m - N.k;
                gb.add(k, H->r, nr, T(1), F + N.tmat, nr, false, F + N.rg + int64_t(k) * H->r, H->r, false, T(1),
                       F + N.rhat, H->r);
            }
            KRR_TRY(gb.launch(c));
            tr.mark("rhat", h, nn, 0);
        }
    }
    return KRR_OK;
}

template <class T>
int compress(HssImpl *H) {
    Ctx *c = H->c;
    const double t0 = now_ms();
    double ts = 0;
    int c0 = 0;
    H->rounds = 0;
    // the QR needs at least one column beyond the held-out and oversampling columns
    while (H->r - kHoldOut - H->opt.p < 1) {
        if (H->r >= H->opt.r_max) return fail(KRR_ERR_INVALID_ARG, "hss_compress: r_max too small for p");
        H->r = int(std::min<int64_t>(H->opt.r_max, 2 * int64_t(H->r)));
    }
    while (true) {
        const double s0 = now_ms();
        KRR_TRY(sample_columns<T>(H, c0, H->r));
        KRR_TRY(take_status(c, "hss_compress"));
        KRR_CUDA(cudaStreamSynchronize(c->stream));
        ts += now_ms() - s0;
        ++H->rounds;
        bool more = false;
        const bool last = H->r >= H->opt.r_max && (H->opt.flags & KRR_TRUNCATE_AT_RMAX);
        KRR_TRY(id_sweep<T>(H, more, last));
        if (last) {
            H->truncated = more;
            break;
        }
        if (!more) break;
        if (H->r >= H->opt.r_max) return fail(KRR_ERR_RANK_BUDGET, "hss_compress: ranks not revealed within r_max");
        c0 = H->r;
        H->r = int(std::min<int64_t>(H->opt.r_max, 2 * int64_t(H->r)));
    }
    H->t_sample = ts;
    H->t_compress = now_ms() - t0;
    return KRR_OK;
}

template <class T>
int factor(HssImpl *H) {
    Ctx *c = H->c;
    const double t0 = now_ms();
    T *F = farena<T>(H);
    const T inv2h2 = T(1.0 / (2.0 * H->opt.h * H->opt.h));
    const T *X = H->f32() ? reinterpret_cast<const T *>(H->Xp32.get()) : reinterpret_cast<const T *>(H->Xp64.get());
    KRR_CUDA(cudaMemcpyAsync(H->ddesc.get(), H->desc.data(), H->desc.size() * sizeof(NodeDesc),
                             cudaMemcpyHostToDevice, c->stream));
    Tracer tr(c);
    for (int h = 0; h <= H->H; ++h) {
        std::vector<int> &lv = H->by_height[h];
        const int nn = int(lv.size());
        if (!nn) continue;
        const int is_root = h == H->H ? 1 : 0;
        int mmax = 0;
        for (int v : lv) mmax = std::max(mmax, H->desc[v].m);
        std::vector<NodeDesc> ld(nn);
        for (int a = 0; a < nn; ++a) ld[a] = H->desc[lv[a]];
        DBuf<NodeDesc> dl(c, nn);
        if (!dl.get()) return fail(KRR_ERR_OOM, "hss_factor: out of memory");
        KRR_CUDA(cudaMemcpyAsync(dl.get(), ld.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, c->stream));
        const unsigned per_node = unsigned(std::max(1, std::min(64, 4 * c->num_sms / nn)));
        { factor_build_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(dl.get(), H->ddesc.get(), X, H->d, inv2h2,
                                                                 T(H->lambda), F, H->IA.get(), is_root); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        if (!is_root) {
            // D'_rs = D_rs - T^T D_ss ; D'_rr = D_rr - T^T D_sr - D'_rs T
            GemmBatch<T> g1, g2, g3;
            for (const NodeDesc &N : ld) {
                const int k = N.k, nr = N.m - N.k;
                g1.add(nr, k, k, T(-1), F + N.tmat, nr, true, F + N.dtil, k, false, T(1), F + N.drs, k);
                g2.add(nr, nr, k, T(-1), F + N.tmat, nr, true, F + N.dmat, k, true, T(1), F + N.drr, nr);
                g3.add(nr, nr, k, T(-1), F + N.drs, k, false, F + N.tmat, nr, false, T(1), F + N.drr, nr);
            }
            tr.mark("f_build", h, nn, mmax);
            KRR_TRY(g1.launch(c));
            KRR_TRY(g2.launch(c));
            KRR_TRY(g3.launch(c));
            tr.mark("f_gemm123", h, nn, mmax);
        }
        int nmax_inv = 0;
        for (const NodeDesc &N : ld) nmax_inv = std::max(nmax_inv, is_root ? N.m : N.m - N.k);
        if (nmax_inv < 96 || (nmax_inv < kBigNode && nn >= c->num_sms)) {
            { invert_kernel<T><<<nn, cta::kNT, 0, c->stream>>>(dl.get(), F, H->IA.get(), is_root, c->status); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        } else {
            std::vector<big::InvItem> items;
            for (const NodeDesc &N : ld) items.push_back(big::InvItem{N.drr, N.ipiv, is_root ? N.m : N.m - N.k});
            // blocked panels: about 3 launches per 32 pivots (one launch pair
            // per pivot for the unblocked batched form)
            KRR_TRY(big::gj_inverse_blocked<T>(c, items, F, H->IA.get()));
        }
        tr.mark("f_invert", h, nn, mmax);
        if (!is_root) {
            // Y = D'_rr^{-1} D'_rs ; Dt = D_ss - D'_rs^T Y
            GemmBatch<T> g4, g5;
            for (const NodeDesc &N : ld) {
                const int k = N.k, nr = N.m - N.k;
                g4.add(nr, k, nr, T(1), F + N.drr, nr, false, F + N.drs, k, false, T(0), F + N.ymat, k);
                g5.add(k, k, nr, T(-1), F + N.drs, k, true, F + N.ymat, k, false, T(1), F + N.dtil, k);
            }
            KRR_TRY(g4.launch(c));
            KRR_TRY(g5.launch(c));
            tr.mark("f_gemm45", h, nn, mmax);
        }
    }
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    H->factored = true;
    H->t_factor = now_ms() - t0;
    return KRR_OK;
}

template <class T>
GemmPlan<T, 16> &pick_s(HssImpl::LevelPlan &P, int which);
template <>
GemmPlan<float, 16> &pick_s<float>(HssImpl::LevelPlan &P, int which) { return P.sf[which]; }
template <>
GemmPlan<double, 16> &pick_s<double>(HssImpl::LevelPlan &P, int which) { return P.se[which]; }

template <class T>
GemmPlan<T, 16> &pick(HssImpl::LevelPlan &P, int which);
template <>
GemmPlan<float, 16> &pick<float>(HssImpl::LevelPlan &P, int which) {
    GemmPlan<float, 16> *a[6] = {&P.f1, &P.f2, &P.f3, &P.f4, &P.fd1, &P.fd2};
    return *a[which];
}
template <>
GemmPlan<double, 16> &pick<double>(HssImpl::LevelPlan &P, int which) {
    GemmPlan<double, 16> *a[6] = {&P.e1, &P.e2, &P.e3, &P.e4, &P.ed1, &P.ed2};
    return *a[which];
}

// Per-level descriptors and GEMM problem lists of the ULV sweeps for nrhs
// right-hand sides, uploaded once per factorization.
// The phase list of the one-launch ULV sweep (the same steps, in the same
// order, as ulv_solve below), for a grid of H->ulv_grid CTAs.
template <class T>
int build_sweep(HssImpl *H) {
    static_assert(fused_smem<T>() <= SkinnyCfg<T>::smem(), "the sweep's shared memory holds a small-node step");
    Ctx *c = H->c;
    if (H->ulv_grid < 0) {
        H->ulv_grid = 0;
        int coop = 0, nb = 0;
        KRR_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        const int smem = int(SkinnyCfg<T>::smem());
        static SmemLimitOnce smem_limit;
        KRR_CUDA(raise_smem_limit(smem_limit, c->device, ulv_sweep_kernel<T>, smem));
        KRR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ulv_sweep_kernel<T>, 256, smem));
        if (coop && nb > 0) H->ulv_grid = nb * c->num_sms;
        if (H->ulv_grid > 0 && !H->ulv_bar.reset(c, 2)) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
    }
    if (H->ulv_grid == 0) return KRR_OK;
    const int G = H->ulv_grid;
    std::vector<UlvPhase<T>> ph;
    // a phase over the level's large nodes (nn x per_node items), with the
    // level's small nodes' whole steps first when fdir != 0
    auto node_phase = [&](int kind, int h, int fdir) {
        HssImpl::LevelPlan &P = H->plan[h];
        UlvPhase<T> q{};
        q.kind = kind;
        q.is_root = h == H->H ? 1 : 0;
        q.nn = P.n_big;
        q.per_node = P.n_big ? std::max(1, std::min(32, G / P.n_big)) : 1;
        q.dl = P.dl_big.get();
        if (fdir) {
            q.fl = P.dl_small.get();
            q.nf = P.n_small;
            q.fdir = fdir;
        }
        q.items = q.nf + q.nn * q.per_node;
        return q;
    };
    auto gemm_phase = [&](const GemmPlan<T, 16> &gp, UlvPhase<T> q) {
        q.kind = kUlvGemm;
        q.probs = gp.d.get();
        q.tp = gp.tp.get();
        q.np = gp.np;
        q.tiles = gp.np ? gp.tiles : 0;
        q.items = q.nf + q.tiles;
        if (q.items > 0) ph.push_back(q);
    };
    const UlvPhase<T> none{};
    for (int h = 0; h <= H->H; ++h) {
        if (H->by_height[h].empty()) continue;
        HssImpl::LevelPlan &P = H->plan[h];
        UlvPhase<T> g = node_phase(kUlvGather, h, 1);
        if (P.nzall > 0) {
            g.z = reinterpret_cast<const ZeroJob<T> *>(P.zall.get());
            g.nz = P.nzall;
            g.zparts = int(std::min<int64_t>(64, std::max<int64_t>(1, cdiv(P.zmax_all, 256))));
            g.items += g.nz * g.zparts;
        }
        if (g.items > 0) ph.push_back(g);
        if (h == H->H) {
            gemm_phase(pick_s<T>(P, 0), none);
            break;
        }
        for (int q = 1; q <= 3; ++q) gemm_phase(pick_s<T>(P, q), none);
    }
    for (int h = H->H; h >= 0; --h) {
        if (H->by_height[h].empty()) continue;
        HssImpl::LevelPlan &P = H->plan[h];
        if (h < H->H) {
            UlvPhase<T> f = node_phase(kUlvGemm, h, 2);  // small nodes' down steps with the first product
            f.nn = 0;
            gemm_phase(pick_s<T>(P, 4), f);
            gemm_phase(pick_s<T>(P, 5), none);
            if (P.n_big) {
                ph.push_back(node_phase(kUlvPlace, h, 0));
                if (h > 0) ph.push_back(node_phase(kUlvScatter, h, 0));  // height 0 holds leaves only
            }
        } else {
            if (H->desc[H->root].is_leaf) ph.push_back(node_phase(kUlvRootLeaf, h, 0));
            else ph.push_back(node_phase(kUlvScatter, h, 0));
        }
    }
    H->ulv_nph = int(ph.size());
    if (!H->ulv_ph.reset(c, ph.size() * sizeof(UlvPhase<T>))) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
    KRR_CUDA(cudaMemcpyAsync(H->ulv_ph.get(), ph.data(), ph.size() * sizeof(UlvPhase<T>), cudaMemcpyHostToDevice,
                             c->stream));
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

template <class T>
int build_solve_plan(HssImpl *H, int nrhs) {
    Ctx *c = H->c;
    T *F = farena<T>(H);
    H->drop_graph();  // the captured solve refers to the old plan
    H->plan.clear();
    H->plan.resize(H->H + 1);
    for (int h = 0; h <= H->H; ++h) {
        std::vector<int> &lv = H->by_height[h];
        const int nn = int(lv.size());
        if (!nn) continue;
        HssImpl::LevelPlan &P = H->plan[h];
        std::vector<NodeDesc> ld(nn);
        for (int a = 0; a < nn; ++a) ld[a] = H->desc[lv[a]];
        if (!P.dl.reset(c, nn)) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
        KRR_CUDA(cudaMemcpyAsync(P.dl.get(), ld.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, c->stream));
        GemmBatch<T, 16> g[6], sw[6];  // every node (graph path); the sweep's large nodes
        for (int q = 0; q < 6; ++q) g[q].split_ok = sw[q].split_ok = true;
        std::vector<NodeDesc> small, big;
        for (const NodeDesc &N : ld) {
            const bool fuse = h < H->H && nrhs <= kFuseRhs && N.m <= kFuseMax;
            (fuse ? small : big).push_back(N);
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1 && fuse) break;
                GemmBatch<T, 16> *b = pass == 0 ? g : sw;
                if (h == H->H) {
                    b[0].add(N.m, nrhs, N.m, T(1), F + N.drr, N.m, false, F + N.zvec, nrhs, false, T(0), F + N.xloc,
                             nrhs);
                    continue;
                }
                const int k = N.k, nr = N.m - N.k;
                b[1].add(nr, nrhs, k, T(-1), F + N.tmat, nr, true, F + N.btil, nrhs, false, T(1), F + N.xloc, nrhs);
                b[2].add(nr, nrhs, nr, T(1), F + N.drr, nr, false, F + N.xloc, nrhs, false, T(0), F + N.zvec, nrhs);
                b[3].add(k, nrhs, nr, T(-1), F + N.drs, k, true, F + N.zvec, nrhs, false, T(1), F + N.btil, nrhs);
                b[4].add(nr, nrhs, k, T(-1), F + N.ymat, k, false, F + N.btil, nrhs, false, T(1), F + N.zvec, nrhs);
                b[5].add(k, nrhs, nr, T(-1), F + N.tmat, nr, false, F + N.zvec, nrhs, false, T(1), F + N.btil, nrhs);
            }
        }
        P.n_small = int(small.size());
        P.n_big = int(big.size());
        if ((P.n_small && !P.dl_small.reset(c, small.size())) || (P.n_big && !P.dl_big.reset(c, big.size())))
            return fail(KRR_ERR_OOM, "hss_solve: out of memory");
        if (P.n_small)
            KRR_CUDA(cudaMemcpyAsync(P.dl_small.get(), small.data(), small.size() * sizeof(NodeDesc),
                                     cudaMemcpyHostToDevice, c->stream));
        if (P.n_big)
            KRR_CUDA(cudaMemcpyAsync(P.dl_big.get(), big.data(), big.size() * sizeof(NodeDesc), cudaMemcpyHostToDevice,
                                     c->stream));
        {
            std::vector<ZeroJob<T>> zs;
            for (int q = 0; q < 4; ++q) zs.insert(zs.end(), sw[q].zj.begin(), sw[q].zj.end());
            P.nzall = int(zs.size());
            P.zmax_all = 0;
            for (const ZeroJob<T> &z : zs) P.zmax_all = std::max(P.zmax_all, z.M * z.N);
            if (!zs.empty()) {
                if (!P.zall.reset(c, zs.size() * sizeof(ZeroJob<T>))) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
                KRR_CUDA(cudaMemcpyAsync(P.zall.get(), zs.data(), zs.size() * sizeof(ZeroJob<T>),
                                         cudaMemcpyHostToDevice, c->stream));
            }
        }
        for (int q = 0; q < 6; ++q) {
            KRR_TRY(g[q].freeze(c, pick<T>(P, q)));
            KRR_TRY(sw[q].freeze(c, pick_s<T>(P, q)));
        }
    }
    H->plan_nrhs = nrhs;
    KRR_TRY(build_sweep<T>(H));
    return KRR_OK;
}

// x_perm = H^{-1} y_perm (both n x nrhs in cluster order, precision T)
template <class T>
int ulv_solve(HssImpl *H, const T *yperm, int64_t ldy, int nrhs, T *xperm, int64_t ldx) {
    Ctx *c = H->c;
    T *F = farena<T>(H);
    if (H->plan_nrhs != nrhs) KRR_TRY(build_solve_plan<T>(H, nrhs));
    for (int h = 0; h <= H->H; ++h) {
        const int nn = int(H->by_height[h].size());
        if (!nn) continue;
        HssImpl::LevelPlan &P = H->plan[h];
        const int is_root = h == H->H ? 1 : 0;
        const unsigned per_node = unsigned(std::max(1, std::min(32, 2 * c->num_sms / nn)));
        { solve_gather_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(P.dl.get(), H->ddesc.get(), yperm,
                                                                                 ldy, nrhs, F, H->IA.get(), is_root); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        if (is_root) {
            KRR_TRY(pick<T>(P, 0).run(c));
            break;
        }
        KRR_TRY(pick<T>(P, 1).run(c));
        KRR_TRY(pick<T>(P, 2).run(c));
        KRR_TRY(pick<T>(P, 3).run(c));
    }
    for (int h = H->H; h >= 0; --h) {
        const int nn = int(H->by_height[h].size());
        if (!nn) continue;
        HssImpl::LevelPlan &P = H->plan[h];
        const unsigned per_node = unsigned(std::max(1, std::min(32, 2 * c->num_sms / nn)));
        if (h < H->H) {
            KRR_TRY(pick<T>(P, 4).run(c));
            KRR_TRY(pick<T>(P, 5).run(c));
            { solve_place_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(P.dl.get(), nrhs, F, H->IA.get(),
                                                                                    xperm, ldx); ::krr::count_launch(); }
        } else if (H->desc[H->root].is_leaf) {  // single-leaf tree: the root's solve is the answer
            { root_leaf_out_kernel<T><<<1, cta::kNT, 0, c->stream>>>(P.dl.get(), nrhs, F, xperm, ldx); ::krr::count_launch(); }
        }
        { scatter_down_kernel<T><<<dim3(nn, per_node), cta::kNT, 0, c->stream>>>(P.dl.get(), H->ddesc.get(), nrhs,
                                                                                 F); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
    }
    return KRR_OK;
}

// ulv_solve through a captured CUDA graph: captured on a private stream the
// first time (and whenever the plan, the buffers or nrhs change), then
// replayed on the context's stream.  y and x must be the same fixed
// buffers on every call for the replay to be reused.
template <class T>
int ulv_solve_graph(HssImpl *H, const T *y, T *x, int nrhs) {
    Ctx *c = H->c;
    if (H->plan_nrhs != nrhs) KRR_TRY(build_solve_plan<T>(H, nrhs));
    if (H->ulv_grid > 0) {  // the whole sweep in one cooperative launch
        KRR_CUDA(cudaMemsetAsync(H->ulv_bar.get(), 0, sizeof(GridBar), c->stream));
        const UlvPhase<T> *phases = reinterpret_cast<const UlvPhase<T> *>(H->ulv_ph.get());
        int nph = H->ulv_nph;
        const NodeDesc *all = H->ddesc.get();
        T *F = farena<T>(H);
        const int32_t *I = H->IA.get();
        GridBar *bar = reinterpret_cast<GridBar *>(H->ulv_bar.get());
        long long budget = c->wait_cycles;
        DevStatus *st = c->status;
        void *args[] = {(void *)&phases, (void *)&nph, (void *)&all, (void *)&y, (void *)&x, (void *)&nrhs,
                        (void *)&F, (void *)&I, (void *)&bar, (void *)&budget, (void *)&st};
        KRR_CUDA(cudaLaunchCooperativeKernel((const void *)ulv_sweep_kernel<T>, dim3(unsigned(H->ulv_grid)), dim3(256),
                                             args, SkinnyCfg<T>::smem(), c->stream));
        count_launch();
        return KRR_OK;
    }
    if (!H->ulv_exec || H->g_y != y || H->g_x != x || H->g_nrhs != nrhs) {
        H->drop_graph();
        if (!H->cap_stream) KRR_CUDA(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
        cudaStream_t keep = c->stream;
        c->stream = H->cap_stream;
        const long long k0 = launches_so_far();
        cudaError_t e = cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal);
        int s = e == cudaSuccess ? ulv_solve<T>(H, y, nrhs, nrhs, x, nrhs) : KRR_OK;
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(H->cap_stream, &g) : e;
        c->stream = keep;
        H->g_kernels = launches_so_far() - k0;
        count_launches(-H->g_kernels);  // recorded, not run: counted at each replay
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        if (s != KRR_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
        const cudaError_t e3 = cudaGraphInstantiate(&H->ulv_exec, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            H->ulv_exec = nullptr;
            return cuda_fail(e3, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        H->g_y = y;
        H->g_x = x;
        H->g_nrhs = nrhs;
    }
    KRR_CUDA(cudaGraphLaunch(H->ulv_exec, c->stream));
    count_launches(H->g_kernels);
    return KRR_OK;
}

}  // namespace

// Fused product K(Xa, Xp) V for nrhs columns of V (double, n x nrhs, in
// cluster order) in the path's precision; out = double m x nrhs.  With
// lambda != 0 (Xa == Xp) adds lambda V.  Mixed: V is split into two FP16
// parts so the product keeps FP32 precision in V, and K too when precise
// (K = K_hi + K_lo); otherwise K is rounded to FP16 (relaxed GMRES inner
// products).
int hss_apply(HssImpl *H, const float *Xa32, const __half *XAa, int64_t ma, const double *V, int64_t ldv, int nrhs,
              double *out, int64_t ldo, double lambda, const double *y, int64_t ldy, double *res_norms,
              const BlockDiag *bd, const double *Xa64_rows = nullptr, bool precise = true) {
    Ctx *c = H->c;
    const int64_t n = H->n;
    if (H->tc()) {
        const int cols = 2 * nrhs;
        const int rpad = int(round_up(cols, 64));
        DBuf<float> Rs_own, Sm_own;
        DBuf<__half> RT_own;
        float *Rs, *Sm;
        __half *RTs;
        if (ma == n) {  // the residual / GMRES path: workspaces kept across calls
            if (H->ws_nrhs != nrhs) {
                if (!H->ws_rs.reset(c, size_t(n) * cols) || !H->ws_sm.reset(c, size_t(n) * cols) ||
                    !H->ws_rt.reset(c, size_t(rpad) * H->ldrt))
                    return fail(KRR_ERR_OOM, "hss: out of memory");
                H->ws_nrhs = nrhs;
            }
            Rs = H->ws_rs.get();
            Sm = H->ws_sm.get();
            RTs = H->ws_rt.get();
        } else {
            if (!Rs_own.reset(c, size_t(n) * cols) || !Sm_own.reset(c, size_t(ma) * cols) ||
                !RT_own.reset(c, size_t(rpad) * H->ldrt))
                return fail(KRR_ERR_OOM, "hss: out of memory");
            Rs = Rs_own.get();
            Sm = Sm_own.get();
            RTs = RT_own.get();
        }
        { split16_kernel<<<unsigned(cdiv(n * nrhs, 256)), 256, 0, c->stream>>>(V, n, nrhs, ldv, Rs, cols); ::krr::count_launch(); }
        KRR_TRY(transpose_half(c, Rs, n, cols, cols, RTs, rpad, H->ldrt));
        KRR_TRY(sample_mixed_prepared(c, XAa, ma, H->XB.get(), n, H->d, RTs, cols, H->ldrt, nullptr, nullptr,
                                      Sm, cols, precise, bd));
        if (y)
            { residual_kernel<float><<<unsigned(cdiv(ma * nrhs, 256)), 256, 0, c->stream>>>(
                y, ldy, Sm, cols, 1, V, ldv, ma, nrhs, lambda, out, ldo, res_norms); ::krr::count_launch(); }
        else
            { combine_kernel<float><<<unsigned(cdiv(ma * nrhs, 256)), 256, 0, c->stream>>>(Sm, cols, 1, V, ldv,
                                                                                        lambda, ma, nrhs, out, ldo); ::krr::count_launch(); }
    } else {
        DBuf<double> Sm(c, size_t(ma) * nrhs), Xa64;
        if (!Sm.get()) return fail(KRR_ERR_OOM, "hss: out of memory");
        const double *Xa = Xa64_rows ? Xa64_rows : H->Xp64.get();
        if (!Xa64_rows && Xa32 != H->Xp32.get()) {
            if (!Xa64.reset(c, size_t(ma) * H->d)) return fail(KRR_ERR_OOM, "hss: out of memory");
            KRR_TRY(widen(c, Xa32, ma * H->d, Xa64.get()));
            Xa = Xa64.get();
        }
        KRR_TRY(launch_sample_f64(c, Xa, ma, H->Xp64.get(), n, H->d, H->opt.h, V, nrhs, ldv, nullptr, nullptr,
                                  Sm.get(), nrhs, bd));
        if (y)
            { residual_kernel<double><<<unsigned(cdiv(ma * nrhs, 256)), 256, 0, c->stream>>>(
                y, ldy, Sm.get(), nrhs, 0, V, ldv, ma, nrhs, lambda, out, ldo, res_norms); ::krr::count_launch(); }
        else
            { combine_kernel<double><<<unsigned(cdiv(ma * nrhs, 256)), 256, 0, c->stream>>>(Sm.get(), nrhs, 0, V, ldv,
                                                                                         lambda, ma, nrhs, out, ldo); ::krr::count_launch(); }
    }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

int hss_build(Ctx *c, const float *X, int64_t n, int d, const krr_options *o, HssImpl *H,
              const std::vector<int64_t> *boff = nullptr, const std::vector<double> *bh = nullptr) {
    H->c = c;
    H->opt = *o;
    H->n = n;
    H->d = d;
    H->lambda = o->lambda;
    if (boff) {
        H->nprob = int(boff->size()) - 1;
        H->boff = *boff;
        H->bh = *bh;
        H->opt.h = 1.0;  // coordinates are divided by each problem's width below
        KRR_TRY(make_groups(c, H->boff, H->bgrp));
        if (!H->dboff.reset(c, H->boff.size())) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
        KRR_CUDA(cudaMemcpyAsync(H->dboff.get(), H->boff.data(), H->boff.size() * 8, cudaMemcpyHostToDevice,
                                 c->stream));
        KRR_TRY(make_tile_list(c, H->boff, H->boff, H->tl_lo, H->tl_hi, H->tl_off, H->tl_tiles));
    }
    const double t0 = now_ms();
    if (!H->perm.reset(c, n) || !H->leaf_of.reset(c, n) || !H->Xp32.reset(c, size_t(n) * d))
        return fail(KRR_ERR_OOM, "hss_compress: out of memory");
    KRR_TRY(cluster(c, X, n, d, o->leaf, o->seed, H->perm.get(), H->tb, H->te, H->tl, H->tr, H->tp, H->tv, boff,
                    o->ordering));
    H->t_cluster = now_ms() - t0;
    const int nn = int(H->tb.size());
    H->root = nn - 1;
    // heights
    H->height.assign(nn, 0);
    for (int v = 0; v < nn; ++v)
        if (H->tl[v] >= 0) H->height[v] = 1 + std::max(H->height[H->tl[v]], H->height[H->tr[v]]);
    H->H = H->height[H->root];
    H->by_height.assign(H->H + 1, {});
    for (int v = 0; v < nn; ++v) H->by_height[H->height[v]].push_back(v);
    if (H->nprob > 0) {
        // whole-problem nodes: [begin, end) a union of whole problems
        std::vector<char> bound(n + 1, 0);
        for (int64_t b : H->boff) bound[b] = 1;
        H->top.assign(nn, 0);
        for (int v = 0; v < nn; ++v) H->top[v] = bound[H->tb[v]] && bound[H->te[v]];
    }
    H->desc.assign(nn, NodeDesc{});
    for (int v = 0; v < nn; ++v) {
        NodeDesc &N = H->desc[v];
        N.is_leaf = H->tl[v] < 0;
        N.leaf_begin = H->tb[v];
        N.m = N.is_leaf ? H->te[v] - H->tb[v] : 0;
        N.k = 0;
        N.child_a = H->tl[v];
        N.child_b = H->tr[v];
    }
    // leaf id per row, permuted coordinates, augmented operands
    {
        std::vector<int32_t> isl(nn);
        for (int v = 0; v < nn; ++v) isl[v] = H->tl[v] < 0;
        DBuf<int32_t> db(c, nn), de(c, nn), dl(c, nn);
        if (!db.get() || !de.get() || !dl.get()) return fail(KRR_ERR_OOM, "hss_compress: out of memory");
        KRR_CUDA(cudaMemcpyAsync(db.get(), H->tb.data(), nn * 4, cudaMemcpyHostToDevice, c->stream));
        KRR_CUDA(cudaMemcpyAsync(de.get(), H->te.data(), nn * 4, cudaMemcpyHostToDevice, c->stream));
        KRR_CUDA(cudaMemcpyAsync(dl.get(), isl.data(), nn * 4, cudaMemcpyHostToDevice, c->stream));
        { leaf_id_kernel<<<nn, 128, 0, c->stream>>>(n, db.get(), de.get(), dl.get(), nn, H->leaf_of.get()); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        KRR_CUDA(cudaStreamSynchronize(c->stream));
    }
    KRR_TRY((gather_rows<float, float>(c, X, d, H->perm.get(), n, d, H->Xp32.get(), d)));
    // batched: each problem's coordinates divided by its width (FP64 path: in FP64, below)
    if (H->nprob > 0 && H->tc()) KRR_TRY(scale_by_width(c, H->Xp32.get(), n, d, H->bgrp.get(), H->bh));
    H->r_cap = int(round_up(std::max(o->r0, o->r_max), 64));
    H->r = int(round_up(o->r0, 64));
    H->nrhs_cap = 64;
    if (H->tc()) {
        H->kpad = aug_kpad(d);
        H->ldrt = round_up(n, 8);
        if (!H->XA.reset(c, size_t(n) * H->kpad) || !H->XB.reset(c, size_t(n) * H->kpad) ||
            !H->R32.reset(c, size_t(n) * H->r_cap) || !H->S32.reset(c, size_t(n) * H->r_cap) ||
            !H->RT.reset(c, size_t(round_up(H->r_cap, 64)) * H->ldrt))
            return fail(KRR_ERR_OOM, "hss_compress: out of memory");
        KRR_TRY(augment(c, H->Xp32.get(), n, d, H->opt.h, 0, H->XA.get(), H->kpad));
        KRR_TRY(augment(c, H->Xp32.get(), n, d, H->opt.h, 1, H->XB.get(), H->kpad));
    }
    if (!H->f32()) {
        if (!H->Xp64.reset(c, size_t(n) * d) || !H->R64.reset(c, size_t(n) * H->r_cap) ||
            !H->S64.reset(c, size_t(n) * H->r_cap))
            return fail(KRR_ERR_OOM, "hss_compress: out of memory");
        // KRR_MIXED_F64: Xp32 is already divided by the problems' widths
        KRR_TRY(widen(c, H->Xp32.get(), n * d, H->Xp64.get()));
        if (H->nprob > 0 && !H->tc()) KRR_TRY(scale_by_width(c, H->Xp64.get(), n, d, H->bgrp.get(), H->bh));
    }
    if (H->f32()) KRR_TRY(compress<float>(H));
    else KRR_TRY(compress<double>(H));
    // the samples are no longer needed
    H->R32.release();
    H->S32.release();
    H->RT.release();
    H->R64.release();
    H->S64.release();
    return KRR_OK;
}

int hss_factor_impl(HssImpl *H) {
    H->plan_nrhs = -1;  // the cached solve plan refers to the old factors
    H->drop_graph();
    return H->f32() ? factor<float>(H) : factor<double>(H);
}

// Solve (K + lambda I) a = y in cluster order: yp, ap device double
// n x nrhs (row stride nrhs).  tol <= 0: one ULV solve; else restarted
// GMRES preconditioned by the ULV solve.  rmax: final relative residual
// (max over columns) or -1.
int solve_perm(HssImpl *H, const double *yp, int nrhs, double *ap, double tol, int max_refine, double &rmax) {
    Ctx *c = H->c;
    const int64_t n = H->n;
    const BlockDiag btrain = H->bd_train();
    DBuf<double> res(c, size_t(n) * nrhs), norms(c, 2 * nrhs);
    if (!res.get() || !norms.get()) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
    auto ulv = [&](const double *b, double *x) -> int {
        if (H->f32()) {
            if (H->ws_bf.n < size_t(n) * nrhs &&
                (!H->ws_bf.reset(c, size_t(n) * nrhs) || !H->ws_xf.reset(c, size_t(n) * nrhs)))
                return fail(KRR_ERR_OOM, "hss_solve: out of memory");
            float *bf = H->ws_bf.get(), *xf = H->ws_xf.get();
            { convert_kernel<double, float><<<unsigned(cdiv(n * nrhs, 256)), 256, 0, c->stream>>>(b, n * nrhs, bf); ::krr::count_launch(); }
            KRR_TRY(ulv_solve_graph<float>(H, bf, xf, nrhs));
            { convert_kernel<float, double><<<unsigned(cdiv(n * nrhs, 256)), 256, 0, c->stream>>>(xf, n * nrhs, x); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            return KRR_OK;
        }
        if (H->ws_b64.n < size_t(n) * nrhs &&
            (!H->ws_b64.reset(c, size_t(n) * nrhs) || !H->ws_x64.reset(c, size_t(n) * nrhs)))
            return fail(KRR_ERR_OOM, "hss_solve: out of memory");
        KRR_CUDA(cudaMemcpyAsync(H->ws_b64.get(), b, size_t(n) * nrhs * 8, cudaMemcpyDeviceToDevice, c->stream));
        KRR_TRY(ulv_solve_graph<double>(H, H->ws_b64.get(), H->ws_x64.get(), nrhs));
        KRR_CUDA(cudaMemcpyAsync(x, H->ws_x64.get(), size_t(n) * nrhs * 8, cudaMemcpyDeviceToDevice, c->stream));
        return KRR_OK;
    };
    rmax = -1.0;
    H->refine_steps = 0;
    if (tol <= 0) {
        KRR_TRY(ulv(yp, ap));
    } else {
        // Right-preconditioned restarted GMRES, one Krylov space per column:
        // A M^{-1} u = y, alpha = M^{-1} u, M^{-1} = the ULV solve.  Every
        // column advances together (one fused product and one ULV solve per
        // iteration); Gram-Schmidt runs twice (CGS2).  Restarts recompute
        // the true residual with the precise (split-K) fused product.
        const int mres = 30;
        constexpr double kRelaxSwitch = 0.03 * 2048.0;  // 0.03 / 2^-11
        const int64_t nn = n * nrhs;
        // dots: the two Gram-Schmidt passes' coefficients (mres + 1 rows of
        // nrhs each) and the new vector's squared norms, read back together
        DBuf<double> V(c, size_t(mres + 1) * nn), Wv(c, nn), Zv(c, nn), dots(c, size_t(2 * (mres + 1) + 1) * nrhs),
            coef(c, size_t(mres + 1) * nrhs), sc(c, nrhs), ynorm(c, 2 * nrhs);
        if (!V.get() || !Wv.get() || !Zv.get() || !dots.get() || !coef.get() || !sc.get() || !ynorm.get())
            return fail(KRR_ERR_OOM, "hss_solve: out of memory");
        KRR_CUDA(cudaMemsetAsync(ap, 0, nn * sizeof(double), c->stream));
        const unsigned g1 = unsigned(cdiv(nn, 256));
        const unsigned gd = unsigned(std::min<int64_t>(2 * c->num_sms, cdiv(n, 256)));
        const unsigned gz = unsigned(cdiv(nrhs, 16));
        // out[i][c] = <A_i(:, c), B(:, c)> (out zeroed here)
        auto mdot = [&](const double *A, int nb, const double *B, double *out) -> int {
            KRR_CUDA(cudaMemsetAsync(out, 0, size_t(nb) * nrhs * sizeof(double), c->stream));
            { multidot_kernel<<<dim3(gd, nb, gz), 256, 0, c->stream>>>(A, nn, nb, B, n, nrhs, out); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            return KRR_OK;
        };
        double *d1 = dots.get(), *d2 = dots.get() + size_t(mres + 1) * nrhs, *dw = dots.get() + size_t(2 * (mres + 1)) * nrhs;
        std::vector<double> ynrm(nrhs), hd((mres + 1) * nrhs), hdots(size_t(2 * (mres + 1) + 1) * nrhs);
        Tracer tr(c);
        KRR_TRY(mdot(yp, 1, yp, d1));
        KRR_CUDA(cudaMemcpyAsync(ynrm.data(), d1, nrhs * 8, cudaMemcpyDeviceToHost, c->stream));
        KRR_CUDA(cudaStreamSynchronize(c->stream));
        for (auto &v : ynrm) v = std::sqrt(v) > 0 ? std::sqrt(v) : 1.0;
        // per-column Hessenberg (column-major (mres+1) x mres), Givens, rhs
        std::vector<double> Hm(size_t(nrhs) * (mres + 1) * mres), cs(size_t(nrhs) * mres), sn(size_t(nrhs) * mres),
            g(size_t(nrhs) * (mres + 1)), beta(nrhs), yv(size_t(mres) * nrhs);
        int total_it = 0;
        for (int cycle = 0;; ++cycle) {
            // r = y - A alpha (precise product); V0 = r / |r|
            KRR_CUDA(cudaMemsetAsync(norms.get(), 0, 2 * nrhs * sizeof(double), c->stream));
            KRR_TRY(hss_apply(H, H->Xp32.get(), H->XA.get(), n, ap, nrhs, nrhs, res.get(), nrhs, H->lambda,
                              yp, nrhs, norms.get(), H->bd_or_null(btrain)));
            std::vector<double> hn(2 * nrhs);
            KRR_CUDA(cudaMemcpyAsync(hn.data(), norms.get(), 2 * nrhs * 8, cudaMemcpyDeviceToHost, c->stream));
            KRR_CUDA(cudaStreamSynchronize(c->stream));
            rmax = 0;
            for (int q = 0; q < nrhs; ++q) {
                beta[q] = std::sqrt(hn[2 * q]);
                // a NaN would compare false against tol and pass for convergence
                if (!std::isfinite(beta[q])) return fail(KRR_ERR_NO_CONVERGENCE, "hss_solve: non-finite residual");
                rmax = std::max(rmax, beta[q] / ynrm[q]);
            }
            if (rmax <= tol || total_it >= max_refine) break;
            std::vector<double> inv(nrhs);
            for (int q = 0; q < nrhs; ++q) inv[q] = beta[q] > 0 ? 1.0 / beta[q] : 0.0;
            KRR_CUDA(cudaMemcpyAsync(sc.get(), inv.data(), nrhs * 8, cudaMemcpyHostToDevice, c->stream));
            { colscale_kernel<<<g1, 256, 0, c->stream>>>(V.get(), res.get(), sc.get(), n, nrhs); ::krr::count_launch(); }
            std::fill(Hm.begin(), Hm.end(), 0.0);
            std::fill(g.begin(), g.end(), 0.0);
            for (int q = 0; q < nrhs; ++q) g[size_t(q) * (mres + 1)] = beta[q];
            int jdone = 0;
            double est = rmax;
            for (int j = 0; j < mres && total_it < max_refine; ++j) {
                ++total_it;
                double *Vj = V.get() + int64_t(j) * nn;
                KRR_TRY(ulv(Vj, Zv.get()));
                tr.mark("g_ulv", j, 0, 0);
                // Relaxed inner products (inexact Krylov): once the estimated
                // residual est is small, an operator error of eta est is
                // allowed with eta ~ tol / est; K rounded to FP16 (2^-11 per
                // entry) is used where 2^-11 <= 0.03 tol / est.  Restarts and
                // the final check use the precise product.
                const bool precise = est > kRelaxSwitch * tol;
                KRR_TRY(hss_apply(H, H->Xp32.get(), H->XA.get(), n, Zv.get(), nrhs, nrhs, Wv.get(), nrhs, H->lambda,
                                  nullptr, 0, nullptr, H->bd_or_null(btrain), nullptr, precise));
                tr.mark("g_apply", j, 0, 0);
                // two passes of classical Gram-Schmidt on the device (the
                // coefficients stay there), the next vector normalized there
                // too; one read-back per iteration for the Hessenberg column
                for (int pass = 0; pass < 2; ++pass) {
                    double *dp = pass == 0 ? d1 : d2;
                    KRR_TRY(mdot(V.get(), j + 1, Wv.get(), dp));
                    { combo_kernel<<<g1, 256, 0, c->stream>>>(Wv.get(), V.get(), nn, j + 1, dp, -1.0, n, nrhs); ::krr::count_launch(); }
                }
                KRR_TRY(mdot(Wv.get(), 1, Wv.get(), dw));
                { colnorm_kernel<<<g1, 256, 0, c->stream>>>(V.get() + int64_t(j + 1) * nn, Wv.get(), dw, n, nrhs); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
                KRR_CUDA(cudaMemcpyAsync(hdots.data(), dots.get(), hdots.size() * 8, cudaMemcpyDeviceToHost, c->stream));
                KRR_CUDA(cudaStreamSynchronize(c->stream));
                tr.mark("g_ortho", j, 0, 0);
                for (size_t e = 0; e < size_t(j + 1) * nrhs; ++e) hd[e] = hdots[e] + hdots[size_t(mres + 1) * nrhs + e];
                const double *wn = hdots.data() + size_t(2 * (mres + 1)) * nrhs;
                est = 0;
                for (int q = 0; q < nrhs; ++q) {
                    double *Hq = Hm.data() + size_t(q) * (mres + 1) * mres;
                    double *col = Hq + size_t(j) * (mres + 1);
                    for (int i = 0; i <= j; ++i) col[i] = hd[size_t(i) * nrhs + q];
                    if (!std::isfinite(wn[q])) return fail(KRR_ERR_NO_CONVERGENCE, "hss_solve: non-finite Krylov vector");
                    const double hn1 = std::sqrt(std::max(wn[q], 0.0));
                    col[j + 1] = hn1;
                    double *csq = cs.data() + size_t(q) * mres, *snq = sn.data() + size_t(q) * mres;
                    double *gq = g.data() + size_t(q) * (mres + 1);
                    for (int i = 0; i < j; ++i) {
                        const double a = col[i], b = col[i + 1];
                        col[i] = csq[i] * a + snq[i] * b;
                        col[i + 1] = -snq[i] * a + csq[i] * b;
                    }
                    const double a = col[j], b = col[j + 1];
                    const double rr = std::hypot(a, b);
                    csq[j] = rr > 0 ? a / rr : 1.0;
                    snq[j] = rr > 0 ? b / rr : 0.0;
                    col[j] = rr;
                    col[j + 1] = 0.0;
                    gq[j + 1] = -snq[j] * gq[j];
                    gq[j] = csq[j] * gq[j];
                    est = std::max(est, std::fabs(gq[j + 1]) / ynrm[q]);
                }
                jdone = j + 1;
                // stop a little below tol so the true residual also meets it
                if (est <= 0.5 * tol) break;
            }
            // y = H^{-1} g per column; alpha += M^{-1} (V y)
            for (int q = 0; q < nrhs; ++q) {
                const double *Hq = Hm.data() + size_t(q) * (mres + 1) * mres;
                const double *gq = g.data() + size_t(q) * (mres + 1);
                for (int i = jdone - 1; i >= 0; --i) {
                    double sacc = gq[i];
                    for (int k2 = i + 1; k2 < jdone; ++k2) sacc -= Hq[size_t(k2) * (mres + 1) + i] * yv[size_t(k2) * nrhs + q];
                    const double dgn = Hq[size_t(i) * (mres + 1) + i];
                    yv[size_t(i) * nrhs + q] = dgn != 0 ? sacc / dgn : 0.0;
                }
            }
            KRR_CUDA(cudaMemcpyAsync(coef.get(), yv.data(), size_t(jdone) * nrhs * 8, cudaMemcpyHostToDevice, c->stream));
            KRR_CUDA(cudaMemsetAsync(Wv.get(), 0, nn * sizeof(double), c->stream));
            { combo_kernel<<<g1, 256, 0, c->stream>>>(Wv.get(), V.get(), nn, jdone, coef.get(), 1.0, n, nrhs); ::krr::count_launch(); }
            KRR_TRY(ulv(Wv.get(), Zv.get()));
            { axpy_kernel<<<g1, 256, 0, c->stream>>>(ap, Zv.get(), nn); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
        }
        H->refine_steps = total_it;
    }
    return KRR_OK;
}

int hss_solve_impl(HssImpl *H, const double *y, int nrhs, int64_t ldy, double *alpha, int64_t lda, double tol,
                   int max_refine, double *resid) {
    Ctx *c = H->c;
    if (!H->factored) KRR_TRY(hss_factor_impl(H));
    const double t0 = now_ms();
    const int64_t n = H->n;
    if (nrhs > H->nrhs_cap) return fail(KRR_ERR_INVALID_ARG, "hss_solve: nrhs > 64");
    DBuf<double> yp(c, size_t(n) * nrhs), ap(c, size_t(n) * nrhs);
    if (!yp.get() || !ap.get()) return fail(KRR_ERR_OOM, "hss_solve: out of memory");
    KRR_TRY((gather_rows<double, double>(c, y, ldy, H->perm.get(), n, nrhs, yp.get(), nrhs)));
    double rmax = -1.0;
    KRR_TRY(solve_perm(H, yp.get(), nrhs, ap.get(), tol, max_refine, rmax));
    KRR_TRY((scatter_rows<double, double>(c, ap.get(), nrhs, H->perm.get(), n, nrhs, alpha, lda)));
    KRR_TRY(take_status(c, "hss_solve"));
    if (resid) *resid = rmax;
    H->t_solve = now_ms() - t0;
    if (tol > 0 && rmax > tol) return fail(KRR_ERR_NO_CONVERGENCE, "hss_solve: refinement did not reach tol");
    return KRR_OK;
}

int hss_predict_impl(HssImpl *H, const float *Xt, int64_t m, const double *alpha, int nrhs, int64_t lda, double *out,
                     int64_t ldo, const BlockDiag *bd = nullptr, const double *Xt64 = nullptr) {
    Ctx *c = H->c;
    const int64_t n = H->n;
    DBuf<double> ap(c, size_t(n) * nrhs);
    if (!ap.get()) return fail(KRR_ERR_OOM, "krr_predict: out of memory");
    KRR_TRY((gather_rows<double, double>(c, alpha, lda, H->perm.get(), n, nrhs, ap.get(), nrhs)));
    DBuf<__half> xa;
    if (H->tc()) {
        if (!xa.reset(c, size_t(m) * H->kpad)) return fail(KRR_ERR_OOM, "krr_predict: out of memory");
        KRR_TRY(augment(c, Xt, m, H->d, H->opt.h, 0, xa.get(), H->kpad));
    }
    return hss_apply(H, Xt, xa.get(), m, ap.get(), nrhs, nrhs, out, ldo, 0.0, nullptr, 0, nullptr, bd, Xt64);
}

// Decision values of a block-diagonal system: test rows [toff[p], toff[p+1])
// against problem p's training points only.
int hss_predict_batched_impl(HssImpl *H, const float *Xt, int64_t m, const std::vector<int64_t> &toff,
                             const double *alpha, int nrhs, int64_t lda, double *out, int64_t ldo) {
    Ctx *c = H->c;
    const int d = H->d;
    DBuf<float> xs(c, size_t(m) * d);
    DBuf<int32_t> tgrp, lo, hi;
    DBuf<int64_t> off;
    if (!xs.get()) return fail(KRR_ERR_OOM, "krr_predict_batched: out of memory");
    DBuf<double> xs64;
    KRR_CUDA(cudaMemcpyAsync(xs.get(), Xt, size_t(m) * d * 4, cudaMemcpyDeviceToDevice, c->stream));
    KRR_TRY(make_groups(c, toff, tgrp));
    if (H->tc()) {
        KRR_TRY(scale_by_width(c, xs.get(), m, d, tgrp.get(), H->bh));
    } else {
        if (!xs64.reset(c, size_t(m) * d)) return fail(KRR_ERR_OOM, "krr_predict_batched: out of memory");
        KRR_TRY(widen(c, Xt, m * d, xs64.get()));
        KRR_TRY(scale_by_width(c, xs64.get(), m, d, tgrp.get(), H->bh));
    }
    BlockDiag b;
    KRR_TRY(make_tile_list(c, toff, H->boff, lo, hi, off, b.tiles));
    b.grp_a = tgrp.get();
    b.grp_b = H->bgrp.get();
    b.off_b = H->dboff.get();
    b.tl_lo = lo.get();
    b.tl_hi = hi.get();
    b.tl_off = off.get();
    KRR_TRY(hss_predict_impl(H, xs.get(), m, alpha, nrhs, lda, out, ldo, &b, xs64.get()));
    KRR_CUDA(cudaStreamSynchronize(c->stream));  // the temporaries above die here
    return KRR_OK;
}

// ------------------------------------------------------------ multi-class
// One-vs-all classification (Section 2, after Algorithm 1): c binary
// right-hand sides solved at once, the class of a test point the argmax of
// its c decision values.
namespace {

__global__ void one_vs_all_kernel(const int32_t *cls, int64_t n, int c, double *Y, int64_t ldy) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * c) return;
    const int64_t i = e / c;
    const int k = int(e % c);
    Y[i * ldy + k] = cls[i] == k ? 1.0 : -1.0;
}

// Lowest class index on ties; score = decision value, or its magnitude.
__global__ void class_argmax_kernel(const double *dec, int64_t m, int c, int64_t ldd, int absolute,
                                    int32_t *labels) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double *row = dec + i * ldd;
    double best = absolute ? fabs(row[0]) : row[0];
    int arg = 0;
    for (int k = 1; k < c; ++k) {
        const double v = absolute ? fabs(row[k]) : row[k];
        if (v > best) {
            best = v;
            arg = k;
        }
    }
    labels[i] = arg;
}

}  // namespace

int one_vs_all_impl(Ctx *c, const int32_t *cls, int64_t n, int nc, double *Y, int64_t ldy) {
    { one_vs_all_kernel<<<unsigned(cdiv(n * nc, 256)), 256, 0, c->stream>>>(cls, n, nc, Y, ldy); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

int predict_classes_impl(HssImpl *H, const float *Xt, int64_t m, const double *alpha, int nc, int64_t lda,
                         int absolute, double *dec, int64_t ldd, int32_t *labels) {
    Ctx *c = H->c;
    DBuf<double> own;
    if (!dec) {
        if (!own.reset(c, size_t(m) * nc)) return fail(KRR_ERR_OOM, "krr_predict_classes: out of memory");
        dec = own.get();
        ldd = nc;
    }
    KRR_TRY(hss_predict_impl(H, Xt, m, alpha, nc, lda, dec, ldd));
    { class_argmax_kernel<<<unsigned(cdiv(m, 256)), 256, 0, c->stream>>>(dec, m, nc, ldd, absolute, labels); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// ------------------------------------------------------------ matvec
// y = H x for the HSS matrix H the compression built (Section 3.1: leaf
// blocks D = K(I, I) + lambda I, nested bases U = Pi [I; T^T] from the
// interpolative decompositions, sibling blocks B_ab = K(J_a, J_b)):
//   up:    xhat_tau = U_tau^T [x_tau (leaf) | xhat_a; xhat_b (parent)]
//   down:  u = U_tau yhat_tau (0 at the root);
//          yhat_a = u_a + B_ab xhat_b,  yhat_b = u_b + B_ab^T xhat_a
//   leaf:  y_tau = D_tau x_tau + U_tau yhat_tau
// The ULV factorization eliminates exactly this matrix, so solving H x
// returns x to rounding; products of H with random x against (K + lambda I)x
// measure the compression error.  Sums in FP64 over the stored generators.
namespace {

// W: per node v, xhat at W + off[v] (k x nrhs), yhat at W + off[v] + m * nrhs
template <class T>
__global__ void __launch_bounds__(cta::kNT) mv_up_kernel(const int *ids, const NodeDesc *all, const double *xp,
                                                         int nrhs, const int64_t *off, double *W, const T *F,
                                                         const int32_t *I) {
    const int v = ids[blockIdx.x];
    const NodeDesc &N = all[v];
    const int m = N.m, k = N.k, nr = m - k;
    const int32_t *piv = I + N.piv;
    const T *Tm = F + N.tmat;
    const NodeDesc *A = N.is_leaf ? nullptr : &all[N.child_a];
    auto local = [&](int a, int c) -> double {
        if (N.is_leaf) return xp[(N.leaf_begin + int64_t(a)) * nrhs + c];
        if (a < A->k) return W[off[N.child_a] + int64_t(a) * nrhs + c];
        return W[off[N.child_b] + int64_t(a - A->k) * nrhs + c];
    };
    double *xh = W + off[v];
    for (int e = threadIdx.x; e < k * nrhs; e += blockDim.x) {
        const int j = e / nrhs, c = e % nrhs;
        double s = local(piv[j], c);
        for (int i = 0; i < nr; ++i) s += double(Tm[int64_t(j) * nr + i]) * local(piv[k + i], c);
        xh[e] = s;
    }
}

template <class T>
__global__ void __launch_bounds__(cta::kNT) mv_down_kernel(const int *ids, const NodeDesc *all, const double *xp,
                                                           const T *X, int d, T inv2h2, double lambda, int nrhs,
                                                           const int64_t *off, double *W, const T *F,
                                                           const int32_t *I, double *yp, int is_root) {
    const int v = ids[blockIdx.x];
    const NodeDesc &N = all[v];
    const int m = N.m, k = is_root ? 0 : N.k, nr = m - k;
    const int32_t *piv = I + N.piv;
    const T *Tm = F + N.tmat;
    const double *yh = W + off[v] + int64_t(m) * nrhs;
    for (int e = threadIdx.x; e < m * nrhs; e += blockDim.x) {
        const int p = e / nrhs, c = e % nrhs;
        // (U yhat) at local row a: the skeleton rows take yhat, the redundant
        // ones T^T yhat (local rows in pivot order; a root has no basis)
        const int a = is_root ? p : piv[p];
        double u = 0.0;
        if (p < k) u = yh[int64_t(p) * nrhs + c];
        else if (k > 0)
            for (int j = 0; j < k; ++j) u += double(Tm[int64_t(j) * nr + (p - k)]) * yh[int64_t(j) * nrhs + c];
        if (N.is_leaf) {
            const T *xa = X + (N.leaf_begin + int64_t(a)) * d;
            double s = 0.0;
            for (int b = 0; b < m; ++b) {
                const double dab = a == b ? 1.0 + lambda : double(kern(xa, X + (N.leaf_begin + int64_t(b)) * d, d, inv2h2));
                s += dab * xp[(N.leaf_begin + int64_t(b)) * nrhs + c];
            }
            yp[(N.leaf_begin + int64_t(a)) * nrhs + c] = s + u;
            continue;
        }
        const NodeDesc &A = all[N.child_a], &B = all[N.child_b];
        const int ka = A.k, kb = B.k;
        const T *Bm = F + N.bmat;  // ka x kb
        if (a < ka) {
            const double *xb = W + off[N.child_b];
            for (int j = 0; j < kb; ++j) u += double(Bm[int64_t(a) * kb + j]) * xb[int64_t(j) * nrhs + c];
            W[off[N.child_a] + int64_t(A.m) * nrhs + int64_t(a) * nrhs + c] = u;
        } else {
            const double *xa = W + off[N.child_a];
            for (int i = 0; i < ka; ++i) u += double(Bm[int64_t(i) * kb + (a - ka)]) * xa[int64_t(i) * nrhs + c];
            W[off[N.child_b] + int64_t(B.m) * nrhs + int64_t(a - ka) * nrhs + c] = u;
        }
    }
}

template <class T>
int matvec_t(HssImpl *H, const double *xp, int nrhs, double *yp) {
    Ctx *c = H->c;
    const int nn = int(H->desc.size());
    std::vector<int64_t> off(nn);
    int64_t tot = 0;
    for (int v = 0; v < nn; ++v) {
        off[v] = tot;
        tot += 2 * int64_t(H->desc[v].m) * nrhs;
    }
    DBuf<double> W(c, size_t(tot));
    DBuf<int64_t> doff(c, nn);
    DBuf<int> ids(c, nn);
    if (!W.get() || !doff.get() || !ids.get()) return fail(KRR_ERR_OOM, "hss_matvec: out of memory");
    std::vector<int> order;
    std::vector<int> lvl_start(H->H + 2, 0);
    for (int h = 0; h <= H->H; ++h) {
        lvl_start[h] = int(order.size());
        for (int v : H->by_height[h]) order.push_back(v);
    }
    lvl_start[H->H + 1] = int(order.size());
    KRR_CUDA(cudaMemcpyAsync(H->ddesc.get(), H->desc.data(), nn * sizeof(NodeDesc), cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaMemcpyAsync(doff.get(), off.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    KRR_CUDA(cudaMemcpyAsync(ids.get(), order.data(), nn * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    const T *F = farena<T>(H);
    const T *X = H->f32() ? reinterpret_cast<const T *>(H->Xp32.get()) : reinterpret_cast<const T *>(H->Xp64.get());
    const T inv2h2 = T(1.0 / (2.0 * H->opt.h * H->opt.h));
    for (int h = 0; h < H->H; ++h) {
        const int cnt = lvl_start[h + 1] - lvl_start[h];
        if (!cnt) continue;
        { mv_up_kernel<T><<<cnt, cta::kNT, 0, c->stream>>>(ids.get() + lvl_start[h], H->ddesc.get(), xp, nrhs,
                                                            doff.get(), W.get(), F, H->IA.get()); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
    }
    for (int h = H->H; h >= 0; --h) {
        const int cnt = lvl_start[h + 1] - lvl_start[h];
        if (!cnt) continue;
        { mv_down_kernel<T><<<cnt, cta::kNT, 0, c->stream>>>(ids.get() + lvl_start[h], H->ddesc.get(), xp, X, H->d,
                                                              inv2h2, H->lambda, nrhs, doff.get(), W.get(), F,
                                                              H->IA.get(), yp, h == H->H ? 1 : 0); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
    }
    KRR_CUDA(cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

}  // namespace

int hss_matvec_impl(HssImpl *H, const double *x, int nrhs, int64_t ldx, double *y, int64_t ldy) {
    Ctx *c = H->c;
    const int64_t n = H->n;
    DBuf<double> xp(c, size_t(n) * nrhs), yp(c, size_t(n) * nrhs);
    if (!xp.get() || !yp.get()) return fail(KRR_ERR_OOM, "hss_matvec: out of memory");
    KRR_TRY((gather_rows<double, double>(c, x, ldx, H->perm.get(), n, nrhs, xp.get(), nrhs)));
    if (H->f32()) KRR_TRY(matvec_t<float>(H, xp.get(), nrhs, yp.get()));
    else KRR_TRY(matvec_t<double>(H, xp.get(), nrhs, yp.get()));
    KRR_TRY((scatter_rows<double, double>(c, yp.get(), nrhs, H->perm.get(), n, nrhs, y, ldy)));
    return take_status(c, "hss_matvec");
}

// ------------------------------------------------------------ gradient
// Held-out loss L = 1/2 ||K(Xt, X) alpha - yt||^2 with alpha =
// (K + lambda I)^{-1} y and its adjoint gradient in h, lambda and X (the
// parameters of Eq. (1) and Algorithm 1 that Section 5.3 tunes on held-out
// data).  Every kernel sum is a fused product against augmented columns,
// using  |u - v|^2 = |u|^2 - 2 u.v + |v|^2  on coordinates centred on the
// training mean (the kernel depends only on differences).
namespace {

// sum[q] += sum_i X(i, q)  (FP64; blockDim.x threads over a grid-stride)
__global__ void colsum_kernel(const float *X, int64_t n, int d, double *sum) {
    extern __shared__ double sh[];
    for (int q = threadIdx.x; q < d; q += blockDim.x) sh[q] = 0.0;
    __syncthreads();
    const int64_t tot = n * d;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < tot; e += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&sh[e % d], double(X[e]));
    __syncthreads();
    for (int q = threadIdx.x; q < d; q += blockDim.x) atomicAdd(&sum[q], sh[q]);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per training row i (cluster order), xc = x_i - mean:
//   which 0: V(i, 0 .. d+1) = [v_i, v_i |xc|^2, v_i xc]
//   which 1: V(i, d+2 .. 2d+2) = [v_i, v_i xc]
__global__ void grad_cols_kernel(const float *X, int64_t n, int d, const double *sum, double inv_n, const double *v,
                                 int which, double *V, int64_t ldv) {
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (i >= n) return;
    const double vi = v[i];
    double nrm = 0.0;
    double *row = V + i * ldv;
    for (int q = l; q < d; q += 32) {
        const double xc = double(X[i * d + q]) - sum[q] * inv_n;
        nrm += xc * xc;
        if (which == 0) row[2 + q] = vi * xc;
        else row[d + 3 + q] = vi * xc;
    }
    nrm = warp_sum(nrm);
    if (l == 0) {
        if (which == 0) {
            row[0] = vi;
            row[1] = vi * nrm;
        } else {
            row[d + 2] = vi;
        }
    }
}

// One warp per held-out row k.  P(k, :) = K(xt_k, X) [alpha, alpha |xc|^2,
// alpha xc] (only column 0 when full == 0).  g_k = P(k, 0) - yt_k;
// W(k, :) = [g_k, g_k xtc_k];  acc[0] += g_k^2 / 2;
// acc[1] += g_k (|xtc_k|^2 P(k,0) - 2 xtc_k . P(k, 2..) + P(k, 1))
//        = g_k sum_i K(xt_k, x_i) |xt_k - x_i|^2 alpha_i.
__global__ void grad_test_kernel(const float *Xt, int64_t m, int d, const double *sum, double inv_n,
                                 const double *P, int64_t ldp, const double *yt, int full, double *W, int64_t ldw,
                                 double *acc) {
    const int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (k >= m) return;
    const double *pk = P + k * ldp;
    const double g = pk[0] - yt[k];
    double nrm = 0.0, dot = 0.0;
    if (full) {
        for (int q = l; q < d; q += 32) {
            const double xc = double(Xt[k * d + q]) - sum[q] * inv_n;
            nrm += xc * xc;
            dot += xc * pk[2 + q];
            W[k * ldw + 1 + q] = g * xc;
        }
        nrm = warp_sum(nrm);
        dot = warp_sum(dot);
    }
    if (l == 0) {
        atomicAdd(&acc[0], 0.5 * g * g);
        if (full) {
            W[k * ldw] = g;
            atomicAdd(&acc[1], g * (nrm * pk[0] - 2.0 * dot + pk[1]));
        }
    }
}

// One warp per training row p (cluster order).  Q(p, :) = K(x_p, Xt) [g, g xtc]
// (so Q(p, 0) = a_p), Pn(p, :) = K(x_p, X) [alpha, alpha |xc|^2, alpha xc,
// z, z xc].  acc[2] += z_p sum_j K_pj |x_p - x_j|^2 alpha_j;
// acc[3] += z_p alpha_p;  dX(perm[p], :) = h^-2 [alpha_p (Q(p,1..) - xc_p Q(p,0))
//   - z_p (Pn(p,2..) - xc_p Pn(p,0)) - alpha_p (Pn(p,d+3..) - xc_p Pn(p,d+2))].
__global__ void grad_train_kernel(const float *X, int64_t n, int d, const double *sum, double inv_n,
                                  const double *alpha, const double *z, const double *Q, int64_t ldq,
                                  const double *Pn, int64_t ldpn, double inv_h2, const int32_t *perm, double *dX,
                                  int64_t lddx, double *acc) {
    const int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int l = threadIdx.x & 31;
    if (p >= n) return;
    const double ap = alpha[p], zp = z[p];
    const double *qp = Q + p * ldq;
    const double *pp = Pn + p * ldpn;
    double *out = dX ? dX + int64_t(perm[p]) * lddx : nullptr;
    double nrm = 0.0, dot = 0.0;
    for (int q = l; q < d; q += 32) {
        const double xc = double(X[p * d + q]) - sum[q] * inv_n;
        nrm += xc * xc;
        dot += xc * pp[2 + q];
        if (out) {
            const double t = ap * (qp[1 + q] - xc * qp[0]) - zp * (pp[2 + q] - xc * pp[0]) -
                             ap * (pp[d + 3 + q] - xc * pp[d + 2]);
            out[q] = inv_h2 * t;
        }
    }
    nrm = warp_sum(nrm);
    dot = warp_sum(dot);
    if (l == 0) {
        atomicAdd(&acc[2], zp * (nrm * pp[0] - 2.0 * dot + pp[1]));
        atomicAdd(&acc[3], zp * ap);
    }
}

}  // namespace

// out (ma x nv, row stride ldo) = K(Xa, Xb) V for V (nb x nv, row stride
// ldv): no lambda, no leaf mask.  Mixed: XAa / XBb are the augmented
// operands (rows in role 0, columns in role 1); V is split into FP16 hi/lo
// parts and K into a hi/lo pair, so the product keeps about FP32 accuracy.
// FP64: Xa64 / Xb64 on the CUDA cores.
int kprod(HssImpl *H, const __half *XAa, const double *Xa64, int64_t ma, const __half *XBb, const double *Xb64,
          int64_t nb, const double *V, int64_t ldv, int nv, double *out, int64_t ldo) {
    Ctx *c = H->c;
    if (ma == 0 || nv == 0) return KRR_OK;
    if (H->tc()) {
        const int cols = 2 * nv;
        const int rpad = int(round_up(cols, 64));
        const int64_t ldrt = round_up(nb, 8);
        DBuf<float> Rs(c, size_t(nb) * cols), Sm(c, size_t(ma) * cols);
        DBuf<__half> RT(c, size_t(rpad) * ldrt);
        if (!Rs.get() || !Sm.get() || !RT.get()) return fail(KRR_ERR_OOM, "kernel product: out of memory");
        { split16_kernel<<<unsigned(cdiv(nb * nv, 256)), 256, 0, c->stream>>>(V, nb, nv, ldv, Rs.get(), cols); ::krr::count_launch(); }
        KRR_TRY(transpose_half(c, Rs.get(), nb, cols, cols, RT.get(), rpad, ldrt));
        KRR_TRY(sample_mixed_prepared(c, XAa, ma, XBb, nb, H->d, RT.get(), cols, ldrt, nullptr, nullptr, Sm.get(),
                                      cols, true));
        { combine_kernel<float><<<unsigned(cdiv(ma * nv, 256)), 256, 0, c->stream>>>(Sm.get(), cols, 1, nullptr, 0,
                                                                                   0.0, ma, nv, out, ldo); ::krr::count_launch(); }
    } else {
        DBuf<double> Sm(c, size_t(ma) * nv);
        if (!Sm.get()) return fail(KRR_ERR_OOM, "kernel product: out of memory");
        KRR_TRY(launch_sample_f64(c, Xa64, ma, Xb64, nb, H->d, H->opt.h, V, nv, ldv, nullptr, nullptr, Sm.get(), nv));
        { combine_kernel<double><<<unsigned(cdiv(ma * nv, 256)), 256, 0, c->stream>>>(Sm.get(), nv, 0, nullptr, 0,
                                                                                    0.0, ma, nv, out, ldo); ::krr::count_launch(); }
    }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

int heldout_grad_impl(HssImpl *H, const float *Xt, int64_t m, const double *y, const double *yt, double tol,
                      int max_refine, double *loss, double *dh, double *dlambda, double *dX, int64_t lddx,
                      double *alpha, double *resid) {
    Ctx *c = H->c;
    if (!H->factored) KRR_TRY(hss_factor_impl(H));
    const int64_t n = H->n;
    const int d = H->d;
    const bool full = dh || dlambda || dX;
    const double h = H->opt.h;
    const int ldv = 2 * d + 3;  // [alpha, alpha |xc|^2, alpha xc, z, z xc]
    DBuf<double> yp(c, n), ap(c, n), zp(c, n), av(c, n), V(c, size_t(n) * ldv), P(c, size_t(m) * (d + 2)),
        W(c, size_t(m) * (d + 1)), Q(c, size_t(n) * (d + 1)), Pn(c, size_t(n) * ldv), sum(c, d), acc(c, 4);
    if (!yp.get() || !ap.get() || !zp.get() || !av.get() || !V.get() || !P.get() || !W.get() || !Q.get() ||
        !Pn.get() || !sum.get() || !acc.get())
        return fail(KRR_ERR_OOM, "krr_heldout_grad: out of memory");
    // held-out operands: augmented (mixed) or widened (FP64)
    DBuf<__half> tA, tB;
    DBuf<double> t64;
    if (H->tc()) {
        if (!tA.reset(c, size_t(m) * H->kpad) || (full && !tB.reset(c, size_t(m) * H->kpad)))
            return fail(KRR_ERR_OOM, "krr_heldout_grad: out of memory");
        KRR_TRY(augment(c, Xt, m, d, h, 0, tA.get(), H->kpad));
        if (full) KRR_TRY(augment(c, Xt, m, d, h, 1, tB.get(), H->kpad));
    } else {
        if (!t64.reset(c, size_t(m) * d)) return fail(KRR_ERR_OOM, "krr_heldout_grad: out of memory");
        KRR_TRY(widen(c, Xt, m * d, t64.get()));
    }
    const float *X = H->Xp32.get();
    const double inv_n = 1.0 / double(n);
    KRR_CUDA(cudaMemsetAsync(sum.get(), 0, d * sizeof(double), c->stream));
    KRR_CUDA(cudaMemsetAsync(acc.get(), 0, 4 * sizeof(double), c->stream));
    { colsum_kernel<<<unsigned(std::min<int64_t>(cdiv(n * d, 256), 2 * c->num_sms)), 256, d * sizeof(double),
                      c->stream>>>(X, n, d, sum.get()); ::krr::count_launch(); }
    // alpha = (K + lambda I)^{-1} y
    KRR_TRY((gather_rows<double, double>(c, y, 1, H->perm.get(), n, 1, yp.get(), 1)));
    double r1 = -1.0, r2 = -1.0;
    KRR_TRY(solve_perm(H, yp.get(), 1, ap.get(), tol, max_refine, r1));
    const unsigned gw_n = unsigned(cdiv(n * 32, 256)), gw_m = unsigned(cdiv(m * 32, 256));
    { grad_cols_kernel<<<gw_n, 256, 0, c->stream>>>(X, n, d, sum.get(), inv_n, ap.get(), 0, V.get(), ldv); ::krr::count_launch(); }
    // P = K(Xt, X) [alpha, alpha |xc|^2, alpha xc]; g, W, loss, first h term
    const int nvp = full ? d + 2 : 1;
    KRR_TRY(kprod(H, tA.get(), t64.get(), m, H->XB.get(), H->Xp64.get(), n, V.get(), ldv, nvp, P.get(), d + 2));
    { grad_test_kernel<<<gw_m, 256, 0, c->stream>>>(Xt, m, d, sum.get(), inv_n, P.get(), d + 2, yt, full ? 1 : 0,
                                                    W.get(), d + 1, acc.get()); ::krr::count_launch(); }
    if (full) {
        // Q = K(X, Xt) [g, g xtc]; a = Q(:, 0); z = (K + lambda I)^{-1} a
        KRR_TRY(kprod(H, H->XA.get(), H->Xp64.get(), n, tB.get(), t64.get(), m, W.get(), d + 1, d + 1, Q.get(),
                      d + 1));
        KRR_CUDA(cudaMemcpy2DAsync(av.get(), sizeof(double), Q.get(), size_t(d + 1) * sizeof(double), sizeof(double),
                                   size_t(n), cudaMemcpyDeviceToDevice, c->stream));
        const int steps1 = H->refine_steps;
        KRR_TRY(solve_perm(H, av.get(), 1, zp.get(), tol, max_refine, r2));
        H->refine_steps += steps1;
        { grad_cols_kernel<<<gw_n, 256, 0, c->stream>>>(X, n, d, sum.get(), inv_n, zp.get(), 1, V.get(), ldv); ::krr::count_launch(); }
        // Pn = K(X, X) V (no lambda: d/dh and d/dX of lambda I vanish)
        KRR_TRY(kprod(H, H->XA.get(), H->Xp64.get(), n, H->XB.get(), H->Xp64.get(), n, V.get(), ldv, ldv, Pn.get(),
                      ldv));
        { grad_train_kernel<<<gw_n, 256, 0, c->stream>>>(X, n, d, sum.get(), inv_n, ap.get(), zp.get(), Q.get(), d + 1,
                                                         Pn.get(), ldv, 1.0 / (h * h), H->perm.get(), dX, lddx,
                                                         acc.get()); ::krr::count_launch(); }
    }
    KRR_CUDA(cudaGetLastError());
    if (alpha) KRR_TRY((scatter_rows<double, double>(c, ap.get(), 1, H->perm.get(), n, 1, alpha, 1)));
    double hacc[4];
    KRR_CUDA(cudaMemcpyAsync(hacc, acc.get(), sizeof hacc, cudaMemcpyDeviceToHost, c->stream));
    KRR_TRY(take_status(c, "krr_heldout_grad"));
    *loss = hacc[0];
    if (dh) *dh = (hacc[1] - hacc[2]) / (h * h * h);
    if (dlambda) *dlambda = -hacc[3];
    if (resid) *resid = std::max(r1, r2);
    if (tol > 0 && (r1 > tol || r2 > tol))
        return fail(KRR_ERR_NO_CONVERGENCE, "krr_heldout_grad: a solve did not reach tol");
    return KRR_OK;
}

int64_t hss_memory_bytes(const HssImpl *H) {
    // D at leaves, U (T) at non-root nodes, B at parents: the generators
    int64_t e = 0;
    for (size_t v = 0; v < H->desc.size(); ++v) {
        const NodeDesc &N = H->desc[v];
        if (N.is_leaf) e += int64_t(N.m) * N.m;
        if (int(v) != H->root) e += int64_t(N.k) * (N.m - N.k) + N.k;
        if (!N.is_leaf) e += int64_t(H->desc[N.child_a].k) * H->desc[N.child_b].k;
    }
    return e * (H->f32() ? 4 : 8);
}

}  // namespace krr

struct krr_hss {
    krr::HssImpl h;
};

using namespace krr;

extern "C" {

int hss_compress(krr_ctx *k, const float *X, int64_t n, int32_t d, const krr_options *o, krr_hss **out) {
    if (out) *out = nullptr;
    if (!k || !X || !o || !out || n <= 0 || d <= 0) return fail(KRR_ERR_INVALID_ARG, "hss_compress: bad arguments");
    if (!(o->h > 0) || !(o->lambda > 0) || !(o->eps_c > 0) || o->eps_abs < 0 || o->leaf < 1 || o->r0 < 1 ||
        o->p < 0 || o->r_max < o->r0 ||
        (o->precision != KRR_MIXED && o->precision != KRR_FP64 && o->precision != KRR_MIXED_F64) ||
        o->ordering < KRR_ORDER_TWO_MEANS || o->ordering > KRR_ORDER_PCA)
        return fail(KRR_ERR_INVALID_ARG, "hss_compress: bad options");
    if (o->precision != KRR_FP64 && d > kMaxMixedDim)
        return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_compress: mixed path supports d <= 1024");
    if (n > (int64_t(1) << 30)) return fail(KRR_ERR_INVALID_ARG, "hss_compress: n too large");
    krr_hss *H = new (std::nothrow) krr_hss();
    if (!H) return fail(KRR_ERR_OOM, "hss_compress: host allocation failed");
    const int s = hss_build(&k->c, X, n, d, o, &H->h);
    if (s != KRR_OK) {
        delete H;
        return s;
    }
    *out = H;
    return KRR_OK;
}

int hss_compress_batched(krr_ctx *k, const float *X, int64_t n, int32_t d, int32_t nprob, const int64_t *offsets,
                         const double *h, const krr_options *o, krr_hss **out) {
    if (out) *out = nullptr;
    if (!k || !X || !o || !out || !offsets || !h || n <= 0 || d <= 0 || nprob < 1)
        return fail(KRR_ERR_INVALID_ARG, "hss_compress_batched: bad arguments");
    if (!(o->lambda > 0) || !(o->eps_c > 0) || o->eps_abs < 0 || o->leaf < 1 || o->r0 < 1 || o->p < 0 ||
        o->r_max < o->r0 ||
        (o->precision != KRR_MIXED && o->precision != KRR_FP64 && o->precision != KRR_MIXED_F64))
        return fail(KRR_ERR_INVALID_ARG, "hss_compress_batched: bad options");
    if (o->precision != KRR_FP64 && d > kMaxMixedDim)
        return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_compress_batched: mixed path supports d <= 1024");
    if (n > (int64_t(1) << 30)) return fail(KRR_ERR_INVALID_ARG, "hss_compress_batched: n too large");
    std::vector<int64_t> off(offsets, offsets + nprob + 1);
    std::vector<double> hw(h, h + nprob);
    if (off[0] != 0 || off[nprob] != n) return fail(KRR_ERR_INVALID_ARG, "hss_compress_batched: bad offsets");
    for (int p = 0; p < nprob; ++p)
        if (off[p + 1] <= off[p] || !(hw[p] > 0))
            return fail(KRR_ERR_INVALID_ARG, "hss_compress_batched: empty problem or width <= 0");
    krr_hss *H = new (std::nothrow) krr_hss();
    if (!H) return fail(KRR_ERR_OOM, "hss_compress_batched: host allocation failed");
    const int s = hss_build(&k->c, X, n, d, o, &H->h, &off, &hw);
    if (s != KRR_OK) {
        delete H;
        return s;
    }
    *out = H;
    return KRR_OK;
}

int krr_predict_batched(krr_hss *H, const float *Xt, int64_t m, const int64_t *test_offsets, const double *alpha,
                        int32_t nrhs, int64_t lda, double *out, int64_t ldo) {
    if (!H || !test_offsets || !alpha || m < 0 || nrhs < 1 || nrhs > 64 || lda < nrhs || ldo < nrhs ||
        (m > 0 && (!Xt || !out)))
        return fail(KRR_ERR_INVALID_ARG, "krr_predict_batched: bad arguments");
    if (H->h.nprob == 0) return fail(KRR_ERR_INVALID_ARG, "krr_predict_batched: not a batched handle");
    const int P = H->h.nprob;
    std::vector<int64_t> toff(test_offsets, test_offsets + P + 1);
    if (toff[0] != 0 || toff[P] != m) return fail(KRR_ERR_INVALID_ARG, "krr_predict_batched: bad offsets");
    for (int p = 0; p < P; ++p)
        if (toff[p + 1] < toff[p]) return fail(KRR_ERR_INVALID_ARG, "krr_predict_batched: bad offsets");
    if (m == 0) return KRR_OK;
    return hss_predict_batched_impl(&H->h, Xt, m, toff, alpha, nrhs, lda, out, ldo);
}

int hss_update_lambda(krr_hss *H, double lambda) {
    if (!H || !(lambda > 0)) return fail(KRR_ERR_INVALID_ARG, "hss_update_lambda: bad arguments");
    H->h.lambda = lambda;
    H->h.opt.lambda = lambda;
    H->h.factored = false;
    return KRR_OK;
}

int hss_factor(krr_hss *H) {
    if (!H) return fail(KRR_ERR_INVALID_ARG, "hss_factor: NULL");
    KRR_TRY(hss_factor_impl(&H->h));
    const int s = take_status(H->h.c, "hss_factor");
    if (s != KRR_OK) H->h.factored = false;
    return s;
}

int hss_solve(krr_hss *H, const double *y, int32_t nrhs, int64_t ldy, double *alpha, int64_t lda, double tol,
              int32_t max_refine, double *resid) {
    if (!H || !y || !alpha || nrhs < 1 || ldy < nrhs || lda < nrhs || max_refine < 0)
        return fail(KRR_ERR_INVALID_ARG, "hss_solve: bad arguments");
    return hss_solve_impl(&H->h, y, nrhs, ldy, alpha, lda, tol, max_refine, resid);
}

int krr_one_vs_all(krr_ctx *k, const int32_t *cls, int64_t n, int32_t c, double *Y, int64_t ldy) {
    if (!k || !cls || !Y || n < 0 || c < 2 || ldy < c) return fail(KRR_ERR_INVALID_ARG, "krr_one_vs_all: bad arguments");
    if (n == 0) return KRR_OK;
    return one_vs_all_impl(&k->c, cls, n, c, Y, ldy);
}

int krr_predict_classes(krr_hss *H, const float *Xt, int64_t m, const double *alpha, int32_t c, int64_t lda,
                        int32_t absolute, double *dec, int64_t ldd, int32_t *labels) {
    if (!H || !Xt || !alpha || !labels || m < 0 || c < 2 || c > 64 || lda < c || (dec && ldd < c) ||
        (absolute != 0 && absolute != 1))
        return fail(KRR_ERR_INVALID_ARG, "krr_predict_classes: bad arguments");
    if (H->h.nprob > 0) return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_predict_classes: batched handle");
    if (m == 0) return KRR_OK;
    return predict_classes_impl(&H->h, Xt, m, alpha, c, lda, absolute, dec, ldd, labels);
}

int hss_matvec(krr_hss *H, const double *x, int32_t nrhs, int64_t ldx, double *y, int64_t ldy) {
    if (!H || !x || !y || nrhs < 1 || nrhs > 64 || ldx < nrhs || ldy < nrhs)
        return fail(KRR_ERR_INVALID_ARG, "hss_matvec: bad arguments");
    if (H->h.nprob > 0) return fail(KRR_ERR_NOT_IMPLEMENTED, "hss_matvec: batched handle");
    return hss_matvec_impl(&H->h, x, nrhs, ldx, y, ldy);
}

int krr_predict(krr_hss *H, const float *Xt, int64_t m, const double *alpha, int32_t nrhs, int64_t lda, double *out,
                int64_t ldo) {
    if (!H || !Xt || !alpha || !out || m < 0 || nrhs < 1 || nrhs > 64 || lda < nrhs || ldo < nrhs)
        return fail(KRR_ERR_INVALID_ARG, "krr_predict: bad arguments");
    if (H->h.nprob > 0) return fail(KRR_ERR_INVALID_ARG, "krr_predict: batched handle (use krr_predict_batched)");
    if (m == 0) return KRR_OK;
    return hss_predict_impl(&H->h, Xt, m, alpha, nrhs, lda, out, ldo);
}

int krr_heldout_grad(krr_hss *H, const float *Xt, int64_t m, const double *y, const double *yt, double tol,
                     int32_t max_refine, double *loss, double *dh, double *dlambda, double *dX, int64_t lddx,
                     double *alpha, double *resid) {
    if (!H || !Xt || !y || !yt || !loss || m < 1 || max_refine < 0 || (dX && lddx < H->h.d))
        return fail(KRR_ERR_INVALID_ARG, "krr_heldout_grad: bad arguments");
    if (m > (int64_t(1) << 30)) return fail(KRR_ERR_INVALID_ARG, "krr_heldout_grad: m too large");
    if (H->h.nprob > 0) return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_heldout_grad: batched handle");
    return heldout_grad_impl(&H->h, Xt, m, y, yt, tol, max_refine, loss, dh, dlambda, dX, lddx, alpha, resid);
}

int hss_stats(const krr_hss *H, krr_hss_stats *st) {
    if (!H || !st) return fail(KRR_ERR_INVALID_ARG, "hss_stats: bad arguments");
    const HssImpl &h = H->h;
    st->n = h.n;
    st->n_nodes = int32_t(h.desc.size());
    st->n_levels = h.H + 1;
    st->max_rank = h.max_rank;
    st->samples = h.r;
    st->rounds = h.rounds;
    st->refine_steps = h.refine_steps;
    st->memory_bytes = hss_memory_bytes(&h);
    st->t_cluster_ms = h.t_cluster;
    st->t_sample_ms = h.t_sample;
    st->t_compress_ms = h.t_compress;
    st->t_factor_ms = h.t_factor;
    st->t_solve_ms = h.t_solve;
    st->truncated = h.truncated ? 1 : 0;
    st->pad = 0;
    return KRR_OK;
}

const int32_t *hss_permutation(const krr_hss *H) { return H ? H->h.perm.get() : nullptr; }

void hss_destroy(krr_hss *H) {
    if (!H) return;
    cudaStreamSynchronize(H->h.c->stream);
    delete H;
}

}  // extern "C"
