// Recursive two-means ordering (paper Sections 4.2-4.3, Algorithm 1 step 0)
// on the GPU, level by level: every node of a tree level is split at once.
//
// Arithmetic is exact so that any schedule reaches the same permutation
// (when every segment has n d >= 3 the bound below keeps |q| <= 2^29, so a
// coordinate minus a centre fits in 32 bits and each square is one
// 32 x 32 -> 64-bit product; otherwise the squares are taken in 64 bits):
// coordinates are quantized once to 64-bit integers q = rint(x 2^k) with k
// the largest exponent for which every squared distance inside the data
// hull, summed over all n points, stays below 2^63; distances, sums and
// centres are integers and sums are accumulated with integer atomics
// (associative, so order-free).
//
// Per node covering rows [b, b + m) (m > leaf):
//   * seeds: Philox4x64-10 words (w0, w1) at counter (b, m, 0, 0), key
//     (seed, 0x43).  First representative: row b + floor(w0 m / 2^64).
//     Second: drawn with probability proportional to the squared distance
//     to the first (first row whose inclusive prefix sum of squared
//     distances exceeds floor(w1 total / 2^64)); all-identical points are
//     split in halves.
//   * Lloyd: a point joins group 0 iff d0 <= d1; stop when no label
//     changed (the first assignment counts as a change), when a group is
//     empty, or after 100 centre updates; centre = floor((2 sum + cnt) /
//     (2 cnt)) per coordinate.  An empty group at the end means halves.
//   * stable partition, group 0 first; children recurse while size > leaf.
// Nodes are numbered in postorder (Figure 2) on the host at the end.
//
// Many problems at once: rows split into contiguous segments (one per
// problem); the top of the tree is a balanced binary tree over the
// segments, each segment is then ordered on its own.  Quantization and the
// seed counters are per segment (counter (b - segment start, m)), so each
// segment's subtree and order are exactly those of the segment alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace krr {
namespace {

constexpr int kMaxIter = 100;
constexpr int kMaxD = 1024;  // feature dimensions the node state holds
constexpr int kTB = 256;
constexpr int kWarpDim = 64;  // from this dimension on, a warp computes one point's distances
// Coordinates per lane of the wide-row kernels (JS): the smallest of 4, 8,
// 16, 32 with 32 JS >= d.
inline int wide_slots(int d) { return d <= 128 ? 4 : d <= 256 ? 8 : d <= 512 ? 16 : 32; }

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {  // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// max |x| (as float bits) and a non-finite flag
__global__ void absmax_kernel(const float *X, int64_t cnt, unsigned int *maxbits, int *nonfinite) {
    unsigned int m = 0;
    int bad = 0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < cnt; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = X[k];
        if (!isfinite(v)) bad = 1;
        m = max(m, __float_as_uint(fabsf(v)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxbits, m);
        if (bad) atomicOr(nonfinite, 1);
    }
}

__global__ void quantize_kernel(const float *X, int64_t cnt, double scale, int64_t *q) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < cnt) q[k] = __double2ll_rn(double(X[k]) * scale);
}

// Per segment (blockIdx.y): max |x| as float bits, and a non-finite flag.
__global__ void absmax_seg_kernel(const float *X, int d, const int64_t *seg, unsigned int *maxbits, int *nonfinite) {
    const int p = blockIdx.y;
    const int64_t b = seg[p] * d, e = seg[p + 1] * d;
    unsigned int m = 0;
    int bad = 0;
    for (int64_t k = b + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < e; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = X[k];
        if (!isfinite(v)) bad = 1;
        m = max(m, __float_as_uint(fabsf(v)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxbits + p, m);
        if (bad) atomicOr(nonfinite, 1);
    }
}

// Per segment (blockIdx.y): q = rint(x 2^kexp[p]).
__global__ void quantize_seg_kernel(const float *X, int d, const int64_t *seg, const int *kexp, int64_t *q) {
    const int p = blockIdx.y;
    const int64_t b = seg[p] * d, e = seg[p + 1] * d;
    const double scale = ldexp(1.0, kexp[p]);
    for (int64_t k = b + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < e; k += int64_t(gridDim.x) * blockDim.x)
        q[k] = __double2ll_rn(double(X[k]) * scale);
}

// (x - c)^2 exactly: in 32-bit differences when `narrow` (see above)
__device__ __forceinline__ long long sq_diff(int64_t x, int64_t c, bool narrow) {
    if (narrow) {
        const int32_t a = int32_t(x - c);
        return (long long)a * a;
    }
    const int64_t a = x - c;
    return a * a;
}

struct NodeState {
    int64_t c0[kMaxD], c1[kMaxD];
    int64_t sum0[kMaxD], sum1[kMaxD];
    unsigned long long cnt1;
    int it, done, changed, halved, first;
};

// One block per node: seeds and initial state.
__global__ void seed_kernel(const int64_t *q, int d, const int64_t *nbeg, const int64_t *nsize, const int64_t *nbase,
                            NodeState *ns, uint64_t seed, bool narrow) {
    const int v = blockIdx.x;
    const int64_t b = nbeg[v], m = nsize[v];
    NodeState &S = ns[v];
    __shared__ unsigned long long warp_tot[kTB / 32];
    __shared__ unsigned long long s_total;
    __shared__ int64_t s_second;
    const U64x4 w = philox4x64_10(uint64_t(b - nbase[v]), uint64_t(m), 0, 0, seed, kStreamCluster);
    const int64_t first = b + int64_t(__umul64hi(w.v[0], uint64_t(m)));
    const int64_t *c0 = q + first * d;
    auto dist0 = [&](int64_t i) -> unsigned long long {
        int64_t s = 0;
        for (int k = 0; k < d; ++k) {
            s += sq_diff(q[i * d + k], c0[k], narrow);
        }
        return (unsigned long long)s;
    };
    // pass 1: total of squared distances
    unsigned long long part = 0;
    for (int64_t i = b + threadIdx.x; i < b + m; i += blockDim.x) part += dist0(i);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < kTB / 32; ++k) t += warp_tot[k];
        s_total = t;
        s_second = -1;
    }
    __syncthreads();
    const unsigned long long total = s_total;
    if (total == 0) {
        if (threadIdx.x == 0) {
            S.done = 1;
            S.halved = 1;
            S.it = 0;
            S.first = 0;
        }
        return;
    }
    const unsigned long long target = __umul64hi(w.v[1], total);
    // pass 2: the first row whose inclusive prefix sum exceeds target
    unsigned long long carry = 0;
    for (int64_t base = b; base < b + m; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long di = i < b + m ? dist0(i) : 0ull;
        // inclusive block scan
        unsigned long long x = di;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
        __syncthreads();
        unsigned long long wpre = 0;
        for (int k = 0; k < (threadIdx.x >> 5); ++k) wpre += warp_tot[k];
        const unsigned long long incl = carry + wpre + x;
        if (i < b + m && incl > target && incl - di <= target) s_second = i;
        unsigned long long btot = 0;
        for (int k = 0; k < kTB / 32; ++k) btot += warp_tot[k];
        carry += btot;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t sec = s_second;
        for (int k = 0; k < d; ++k) {
            S.c0[k] = c0[k];
            S.c1[k] = q[sec * d + k];
            S.sum0[k] = S.sum1[k] = 0;
        }
        S.cnt1 = 0;
        S.it = 0;
        S.done = 0;
        S.changed = 0;
        S.halved = 0;
        S.first = 1;
    }
}

// seed_kernel for wide rows (d >= kWarpDim), in three launches so that all
// SMs share the distance pass (the one-block-per-node kernel leaves the
// top levels' work to a few SMs):
//   seed_first_wide_kernel   per node: the first representative (same draw)
//                            into c0, sums cleared, total cleared;
//   seed_dist_wide_kernel    per row: squared distance to c0 (a warp per
//                            row, lanes over the coordinates) into dist,
//                            summed into the node's total;
//   seed_second_wide_kernel  per node: the same second draw over the
//                            inclusive prefix sums of dist in row order.
// The distances, total and target are the same integers as in seed_kernel.
__global__ void seed_first_wide_kernel(const int64_t *q, int d, const int64_t *nbeg, const int64_t *nsize,
                                       const int64_t *nbase, NodeState *ns, uint64_t seed,
                                       unsigned long long *tot) {
    const int v = blockIdx.x;
    const int64_t b = nbeg[v], m = nsize[v];
    NodeState &S = ns[v];
    const U64x4 w = philox4x64_10(uint64_t(b - nbase[v]), uint64_t(m), 0, 0, seed, kStreamCluster);
    const int64_t first = b + int64_t(__umul64hi(w.v[0], uint64_t(m)));
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        S.c0[k] = q[first * d + k];
        S.sum0[k] = S.sum1[k] = 0;
    }
    if (threadIdx.x == 0) tot[v] = 0ull;
}

template <int JS>
__global__ void __launch_bounds__(kTB) seed_dist_wide_kernel(const int64_t *q, int d, int64_t n,
                                                             const int32_t *node_of, const NodeState *ns,
                                                             unsigned long long *dist, unsigned long long *tot,
                                                             bool narrow) {
    const int lane = threadIdx.x & 31;
    const int64_t wbase = int64_t(blockIdx.x) * kTB + (threadIdx.x & ~31);
    int32_t cur = -1;
    unsigned long long part = 0;  // the warp's running total for node cur
#pragma unroll 1
    for (int pl = 0; pl < 32; ++pl) {
        const int64_t ip = wbase + pl;
        const int32_t vp = ip < n ? node_of[ip] : -1;  // the same for every lane
        if (vp < 0) continue;
        if (vp != cur) {
            if (cur >= 0 && lane == 0 && part) atomicAdd(&tot[cur], part);
            cur = vp;
            part = 0;
        }
        const int64_t *row = q + ip * d;
        const int64_t *c0 = ns[vp].c0;
        int64_t x[JS];
#pragma unroll
        for (int j = 0; j < JS; ++j) {
            const int k = lane + 32 * j;
            int64_t xv = 0;
            if (k < d) xv = row[k];
            x[j] = xv;
        }
        long long s = 0;
#pragma unroll
        for (int j = 0; j < JS; ++j) {
            const int k = lane + 32 * j;
            if (k < d) s += sq_diff(x[j], c0[k], narrow);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dist[ip] = (unsigned long long)s;
        part += (unsigned long long)s;
    }
    if (cur >= 0 && lane == 0 && part) atomicAdd(&tot[cur], part);
}

constexpr int kScanPer = 4;  // rows per thread in one step of the second draw's scan

__global__ void seed_second_wide_kernel(const int64_t *q, int d, const int64_t *nbeg, const int64_t *nsize,
                                        const int64_t *nbase, NodeState *ns, uint64_t seed,
                                        const unsigned long long *dist, const unsigned long long *tot) {
    const int v = blockIdx.x;
    const int64_t b = nbeg[v], m = nsize[v];
    NodeState &S = ns[v];
    __shared__ unsigned long long warp_tot[kTB / 32];
    __shared__ int64_t s_second;
    const unsigned long long total = tot[v];
    if (total == 0) {  // all points identical: halves
        if (threadIdx.x == 0) {
            S.done = 1;
            S.halved = 1;
            S.it = 0;
            S.first = 0;
        }
        return;
    }
    const U64x4 w = philox4x64_10(uint64_t(b - nbase[v]), uint64_t(m), 0, 0, seed, kStreamCluster);
    const unsigned long long target = __umul64hi(w.v[1], total);
    if (threadIdx.x == 0) s_second = -1;
    // the first row whose inclusive prefix sum exceeds target: kTB x kScanPer
    // rows per step, each thread's rows consecutive
    unsigned long long carry = 0;
    for (int64_t base = b; base < b + m; base += int64_t(kTB) * kScanPer) {
        const int64_t r0 = base + int64_t(threadIdx.x) * kScanPer;
        unsigned long long dv[kScanPer], own = 0;
#pragma unroll
        for (int u = 0; u < kScanPer; ++u) {
            dv[u] = r0 + u < b + m ? dist[r0 + u] : 0ull;
            own += dv[u];
        }
        unsigned long long x = own;  // inclusive scan of the threads' sums
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
        __syncthreads();
        unsigned long long wpre = 0;
        for (int k = 0; k < (threadIdx.x >> 5); ++k) wpre += warp_tot[k];
        unsigned long long incl = carry + wpre + x - own;  // before this thread's rows
#pragma unroll
        for (int u = 0; u < kScanPer; ++u) {
            incl += dv[u];
            if (r0 + u < b + m && incl > target && incl - dv[u] <= target) s_second = r0 + u;
        }
        unsigned long long btot = 0;
        for (int k = 0; k < kTB / 32; ++k) btot += warp_tot[k];
        carry += btot;
        __syncthreads();
    }
    const int64_t sec = s_second;
    for (int k = threadIdx.x; k < d; k += blockDim.x) S.c1[k] = q[sec * d + k];
    if (threadIdx.x == 0) {
        S.cnt1 = 0;
        S.it = 0;
        S.done = 0;
        S.changed = 0;
        S.halved = 0;
        S.first = 1;
    }
}

template <int JS>
int launch_seed_dist_t(Ctx *c, unsigned grid, const int64_t *q, int d, int64_t n, const int32_t *node_of,
                       const NodeState *ns, unsigned long long *dist, unsigned long long *tot, bool narrow) {
    { seed_dist_wide_kernel<JS><<<grid, kTB, 0, c->stream>>>(q, d, n, node_of, ns, dist, tot, narrow); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

int launch_seed_wide(Ctx *c, int nn, unsigned grid, const int64_t *q, int d, int64_t n, const int64_t *nbeg,
                     const int64_t *nsize, const int64_t *nbase, const int32_t *node_of, NodeState *ns,
                     uint64_t seed, unsigned long long *dist, unsigned long long *tot, bool narrow) {
    { seed_first_wide_kernel<<<nn, kTB, 0, c->stream>>>(q, d, nbeg, nsize, nbase, ns, seed, tot); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    switch (wide_slots(d)) {
        case 4: KRR_TRY(launch_seed_dist_t<4>(c, grid, q, d, n, node_of, ns, dist, tot, narrow)); break;
        case 8: KRR_TRY(launch_seed_dist_t<8>(c, grid, q, d, n, node_of, ns, dist, tot, narrow)); break;
        case 16: KRR_TRY(launch_seed_dist_t<16>(c, grid, q, d, n, node_of, ns, dist, tot, narrow)); break;
        default: KRR_TRY(launch_seed_dist_t<32>(c, grid, q, d, n, node_of, ns, dist, tot, narrow)); break;
    }
    { seed_second_wide_kernel<<<nn, kTB, 0, c->stream>>>(q, d, nbeg, nsize, nbase, ns, seed, dist, tot); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// Assign each point of a still-running node to its nearer centre and
// accumulate the new groups' sums and counts (narrow rows, d < kWarpDim:
// one thread per point).  When a block's points all belong to one node,
// the sums are gathered per coordinate in shared memory (int64 atomics,
// exact and order-free) and added to the node once per coordinate; dynamic
// shared memory: 2 d int64.
__global__ void assign_kernel(const int64_t *q, int d, int64_t n, const int32_t *node_of, NodeState *ns,
                              int8_t *label, bool narrow) {
    extern __shared__ unsigned long long s_sum[];  // [2][d]
    __shared__ int s_uniform;
    __shared__ int32_t s_node;
    __shared__ int8_t s_lab[kTB];
    __shared__ int s_cnt1;
    const int64_t i0 = int64_t(blockIdx.x) * blockDim.x;
    const int64_t i = i0 + threadIdx.x;
    const int32_t v = i < n ? node_of[i] : -1;
    if (threadIdx.x == 0) {
        const int64_t last = min(i0 + blockDim.x - 1, n - 1);
        s_node = v;
        s_uniform = (v >= 0 && node_of[last] == v) ? 1 : 0;
        s_cnt1 = 0;
    }
    __syncthreads();
    const bool uniform = s_uniform != 0;
    bool active = v >= 0 && !ns[v].done;
    int lab = 0;
    if (active) {
        const NodeState &S = ns[v];
        int64_t d0 = 0, d1 = 0;
        for (int k = 0; k < d; ++k) {
            const int64_t x = q[i * d + k];
            d0 += sq_diff(x, S.c0[k], narrow);
            d1 += sq_diff(x, S.c1[k], narrow);
        }
        lab = d0 > d1 ? 1 : 0;
    }
    if (active) {
        if (ns[v].first || label[i] != lab) ns[v].changed = 1;
        label[i] = int8_t(lab);
    }
    if (uniform) {
        if (ns[s_node].done) return;  // the whole block agrees: no thread reaches a barrier below
        s_lab[threadIdx.x] = int8_t(active ? lab : -1);
        for (int k = threadIdx.x; k < 2 * d; k += blockDim.x) s_sum[k] = 0ull;
        if (active && lab == 1) atomicAdd(&s_cnt1, 1);
        __syncthreads();
        const int np = int(min(int64_t(blockDim.x), n - i0));
        for (int e = threadIdx.x; e < np * d; e += blockDim.x) {
            const int pnt = e / d, k = e - pnt * d;
            const int lb = s_lab[pnt];
            if (lb >= 0) atomicAdd(&s_sum[lb * d + k], (unsigned long long)q[(i0 + pnt) * d + k]);
        }
        __syncthreads();
        NodeState &S = ns[s_node];
        for (int k = threadIdx.x; k < d; k += blockDim.x) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&S.sum0[k]), s_sum[k]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&S.sum1[k]), s_sum[d + k]);
        }
        if (threadIdx.x == 0) atomicAdd(&S.cnt1, (unsigned long long)s_cnt1);
    } else if (active) {
        NodeState &S = ns[v];
        if (lab) atomicAdd(&S.cnt1, 1ull);
        int64_t *sum = lab ? S.sum1 : S.sum0;
        for (int k = 0; k < d; ++k)
            atomicAdd(reinterpret_cast<unsigned long long *>(&sum[k]), (unsigned long long)q[i * d + k]);
    }
}

// assign_kernel for wide rows (d >= kWarpDim, d <= 32 JS).  A block takes
// kWideRows consecutive points, each of its warps kWidePts of them one at
// a time, lanes over the coordinates.  Every coordinate of the point is
// loaded at once into registers (JS per lane, so the loads are all in
// flight together; as 32-bit words when NARROW: |q| <= 2^29 there, so the
// low word of the int64 is the value), the two distances are reduced
// across the warp, and the same registers are then added into the sums of
// the point's group: in shared memory ([2][d] int64, atomics) when the
// block's points are all one node, then one add per coordinate into the
// node; directly into the node's sums otherwise.  Each coordinate is read
// once per pass; integer sums, so the result is the same for any order.
// Dynamic shared memory: 2 d int64.
constexpr int kWidePts = 16;                           // points per warp
constexpr int kWideRows = (kTB / 32) * kWidePts;       // points per block

template <int JS, bool NARROW>
__global__ void __launch_bounds__(kTB) assign_wide_kernel(const int64_t *q, int d, int64_t n,
                                                          const int32_t *node_of, NodeState *ns, int8_t *label) {
    extern __shared__ unsigned long long s_acc[];  // [2][d]
    __shared__ int s_uniform;
    __shared__ int32_t s_node;
    __shared__ unsigned long long s_c1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = int64_t(blockIdx.x) * kWideRows;
    if (threadIdx.x == 0) {
        const int32_t v0 = i0 < n ? node_of[i0] : -1;
        const int64_t last = min(i0 + kWideRows - 1, n - 1);
        s_node = v0;
        s_uniform = (v0 >= 0 && node_of[last] == v0) ? 1 : 0;
        s_c1 = 0ull;
    }
    for (int k = threadIdx.x; k < 2 * d; k += kTB) s_acc[k] = 0ull;
    __syncthreads();
    const bool uniform = s_uniform != 0;
    if (uniform && ns[s_node].done) return;  // the whole block agrees: no thread reaches the barrier below
    using W = typename std::conditional<NARROW, int32_t, int64_t>::type;
    const W *qw = reinterpret_cast<const W *>(q);
    constexpr int kStride = NARROW ? 2 : 1;  // W words per coordinate
    unsigned long long c1 = 0;               // group-1 points of this warp (uniform blocks)
    const int64_t wbase = i0 + int64_t(warp) * kWidePts;
#pragma unroll 1
    for (int pl = 0; pl < kWidePts; ++pl) {
        const int64_t ip = wbase + pl;
        const int32_t vp = ip < n ? node_of[ip] : -1;  // the same for every lane
        if (vp < 0 || ns[vp].done) continue;
        NodeState &S = ns[vp];
        const W *row = qw + ip * d * kStride;
        W x[JS];
#pragma unroll
        for (int j = 0; j < JS; ++j) {
            const int k = lane + 32 * j;
            W xv = 0;
            if (k < d) xv = row[int64_t(k) * kStride];
            x[j] = xv;
        }
        long long d0 = 0, d1 = 0;
#pragma unroll
        for (int j = 0; j < JS; ++j) {
            const int k = lane + 32 * j;
            if (k < d) {
                if (NARROW) {
                    const int32_t a0 = int32_t(x[j]) - int32_t(S.c0[k]), a1 = int32_t(x[j]) - int32_t(S.c1[k]);
                    d0 += (long long)a0 * a0;
                    d1 += (long long)a1 * a1;
                } else {
                    const int64_t a0 = int64_t(x[j]) - S.c0[k], a1 = int64_t(x[j]) - S.c1[k];
                    d0 += a0 * a0;
                    d1 += a1 * a1;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        const int lab = d0 > d1 ? 1 : 0;  // the same for every lane
        if (lane == 0) {
            if (S.first || label[ip] != lab) S.changed = 1;
            label[ip] = int8_t(lab);
        }
        if (uniform) {
            c1 += unsigned(lab);
            unsigned long long *a = s_acc + (lab ? d : 0);
#pragma unroll
            for (int j = 0; j < JS; ++j) {
                const int k = lane + 32 * j;
                if (k < d) atomicAdd(a + k, (unsigned long long)(long long)x[j]);
            }
        } else {
            int64_t *sum = lab ? S.sum1 : S.sum0;
#pragma unroll
            for (int j = 0; j < JS; ++j) {
                const int k = lane + 32 * j;
                if (k < d) atomicAdd(reinterpret_cast<unsigned long long *>(sum + k), (unsigned long long)(long long)x[j]);
            }
            if (lane == 0 && lab) atomicAdd(&S.cnt1, 1ull);
        }
    }
    if (uniform) {
        if (lane == 0 && c1) atomicAdd(&s_c1, c1);
        __syncthreads();  // the block's sums are complete
        NodeState &S = ns[s_node];
        for (int k = threadIdx.x; k < 2 * d; k += kTB) {
            const unsigned long long t = s_acc[k];
            int64_t *dst = k < d ? &S.sum0[k] : &S.sum1[k - d];
            if (t) atomicAdd(reinterpret_cast<unsigned long long *>(dst), t);
        }
        if (threadIdx.x == 0 && s_c1) atomicAdd(&S.cnt1, s_c1);
    }
}

template <int JS, bool NARROW>
int launch_assign_wide_t(Ctx *c, const int64_t *q, int d, int64_t n, const int32_t *node_of, NodeState *ns,
                         int8_t *label) {
    const int bytes = 2 * d * int(sizeof(unsigned long long));  // <= 16 KB (d <= 1024)
    const unsigned grid = unsigned(cdiv(n, kWideRows));
    { assign_wide_kernel<JS, NARROW><<<grid, kTB, bytes, c->stream>>>(q, d, n, node_of, ns, label); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

template <bool NARROW>
int launch_assign_wide_n(Ctx *c, const int64_t *q, int d, int64_t n, const int32_t *node_of, NodeState *ns,
                         int8_t *label) {
    switch (wide_slots(d)) {
        case 4: return launch_assign_wide_t<4, NARROW>(c, q, d, n, node_of, ns, label);
        case 8: return launch_assign_wide_t<8, NARROW>(c, q, d, n, node_of, ns, label);
        case 16: return launch_assign_wide_t<16, NARROW>(c, q, d, n, node_of, ns, label);
        default: return launch_assign_wide_t<32, NARROW>(c, q, d, n, node_of, ns, label);
    }
}

int launch_assign_wide(Ctx *c, const int64_t *q, int d, int64_t n, const int32_t *node_of, NodeState *ns,
                       int8_t *label, bool narrow) {
    return narrow ? launch_assign_wide_n<true>(c, q, d, n, node_of, ns, label)
                  : launch_assign_wide_n<false>(c, q, d, n, node_of, ns, label);
}

// One CTA per node: stop test, centre update (threads over the
// coordinates), accumulator reset.
__global__ void update_kernel(int nn, int d, const int64_t *nsize, NodeState *ns, int *n_running) {
    const int v = blockIdx.x;
    if (v >= nn) return;
    NodeState &S = ns[v];
    if (S.done) return;  // the same for the whole block
    __shared__ int s_stop0, s_it;
    const int64_t m = nsize[v];
    const int64_t c1 = int64_t(S.cnt1), c0 = m - c1;
    if (threadIdx.x == 0) {
        s_stop0 = (!S.changed || c0 == 0 || c1 == 0) ? 1 : 0;
        s_it = S.it;
    }
    __syncthreads();
    const bool stop0 = s_stop0 != 0;
    const bool stop = stop0 || s_it + 1 == kMaxIter;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        if (!stop0) {
            S.c0[k] = floor_div(2 * S.sum0[k] + c0, 2 * c0);
            S.c1[k] = floor_div(2 * S.sum1[k] + c1, 2 * c1);
        }
        if (!stop) S.sum0[k] = S.sum1[k] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!stop0) S.it = s_it + 1;
        if (stop) {
            S.done = 1;
            if (c0 == 0 || c1 == 0) S.halved = 1;
        } else {
            S.cnt1 = 0;
            S.changed = 0;
            S.first = 0;
            atomicAdd(n_running, 1);
        }
    }
}

// Final labels (halves where required) and the per-point "goes left" flag.
__global__ void finalize_labels_kernel(int64_t n, const int32_t *node_of, const int64_t *nbeg, const int64_t *nsize,
                                       const NodeState *ns, int8_t *label, int32_t *zero_flag) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0) {
        zero_flag[i] = 0;
        return;
    }
    int lab = label[i];
    if (ns[v].halved) {
        lab = (i - nbeg[v]) >= nsize[v] / 2 ? 1 : 0;
        label[i] = int8_t(lab);
    }
    zero_flag[i] = lab == 0 ? 1 : 0;
}

// Exclusive prefix sum of int32 flags (three-phase: block sums, scan of
// block sums in one block, add back).
__global__ void scan_blocks_kernel(const int32_t *in, int64_t n, int64_t *out, int64_t *bsum) {
    __shared__ int64_t wsum[kTB / 32];
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t x = i < n ? in[i] : 0;
    const int64_t own = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    int64_t pre = 0;
    for (int w = 0; w < (threadIdx.x >> 5); ++w) pre += wsum[w];
    if (i < n) out[i] = pre + x - own;
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = pre + x;
}
__global__ void scan_sums_kernel(int64_t *bsum, int64_t nb) {
    // single block, sequential chunks
    __shared__ int64_t carry;
    __shared__ int64_t wsum[kTB / 32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int64_t x = i < nb ? bsum[i] : 0;
        const int64_t own = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        int64_t pre = 0;
        for (int w = 0; w < (threadIdx.x >> 5); ++w) pre += wsum[w];
        int64_t tot = 0;
        for (int w = 0; w < kTB / 32; ++w) tot += wsum[w];
        if (i < nb) bsum[i] = carry + pre + x - own;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}
__global__ void scan_add_kernel(int64_t *out, int64_t n, const int64_t *bsum, int64_t *total_out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
    if (i == n - 1 && total_out) *total_out = out[i];
}

// Stable partition of every active node; inactive rows copy through.
__global__ void partition_kernel(int64_t n, int d, const int32_t *node_of, const int64_t *nbeg, const int64_t *nsize,
                                 const int8_t *label, const int64_t *zscan, const int32_t *zflag, const int64_t *q,
                                 const int32_t *perm, int64_t *q2, int32_t *perm2, int64_t *cnt0_out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    int64_t dst = i;
    if (v >= 0) {
        const int64_t b = nbeg[v];
        const int64_t zb = zscan[b];
        const int64_t last = b + nsize[v] - 1;
        const int64_t c0 = zscan[last] + zflag[last] - zb;
        const int64_t zi = zscan[i] - zb;
        dst = label[i] == 0 ? b + zi : b + c0 + (i - b - zi);
        if (i == b) cnt0_out[v] = c0;
    }
    for (int k = 0; k < d; ++k) q2[dst * d + k] = q[i * d + k];
    perm2[dst] = perm[i];
}

// partition_kernel for wide rows (d >= kWarpDim): one warp per row, lanes
// over the coordinates, so each row moves in coalesced 256-byte pieces.
__global__ void partition_wide_kernel(int64_t n, int d, const int32_t *node_of, const int64_t *nbeg,
                                      const int64_t *nsize, const int8_t *label, const int64_t *zscan,
                                      const int32_t *zflag, const int64_t *q, const int32_t *perm, int64_t *q2,
                                      int32_t *perm2, int64_t *cnt0_out) {
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // the same for the whole warp
    const int32_t v = node_of[i];
    int64_t dst = i;
    if (v >= 0) {
        const int64_t b = nbeg[v];
        const int64_t zb = zscan[b];
        const int64_t last = b + nsize[v] - 1;
        const int64_t c0 = zscan[last] + zflag[last] - zb;
        const int64_t zi = zscan[i] - zb;
        dst = label[i] == 0 ? b + zi : b + c0 + (i - b - zi);
        if (i == b && lane == 0) cnt0_out[v] = c0;
    }
    for (int k = lane; k < d; k += 32) q2[dst * d + k] = q[i * d + k];
    if (lane == 0) perm2[dst] = perm[i];
}

__global__ void mark_nodes_kernel(int nn, const int64_t *nbeg, const int64_t *nsize, int32_t *node_of) {
    // one block per node, threads stride its rows
    const int v = blockIdx.x;
    if (v >= nn) return;
    for (int64_t i = nbeg[v] + threadIdx.x; i < nbeg[v] + nsize[v]; i += blockDim.x) node_of[i] = v;
}

// ------------------------------------------------ other orderings
// Section 4.3 compares two-means with no preprocessing (NP: halves in the
// natural order), a k-d tree (split along the coordinate of maximum spread
// at its mean, the median when that leaves one side 100 times larger) and
// the principal direction (split at the mean of the projections).  All
// three run on the same quantized coordinates and level loop as two-means.
// k-d: spread = max - min of the integer coordinates (lowest coordinate on
// ties), a point goes first iff q m <= sum q (exact).  PCA: a fixed
// sequence of round-to-nearest FP64 operations (no contraction into FMA),
// so the decision is the same in any implementation that follows it.

// Generic labels -> "goes first" flags; halves where flagged.
__global__ void finalize_generic_kernel(int64_t n, const int32_t *node_of, const int64_t *nbeg, const int64_t *nsize,
                                        const int *halved, int8_t *label, int32_t *zero_flag) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0) {
        zero_flag[i] = 0;
        return;
    }
    int lab = label[i];
    if (halved[v]) {
        lab = (i - nbeg[v]) >= nsize[v] / 2 ? 1 : 0;
        label[i] = int8_t(lab);
    }
    zero_flag[i] = lab == 0 ? 1 : 0;
}

__global__ void count_second_kernel(int64_t n, const int32_t *node_of, const int8_t *label, int *c1) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v >= 0 && label[i]) atomicAdd(&c1[v], 1);
}

// A split that leaves one side empty becomes halves.
__global__ void empty_side_kernel(int nn, const int64_t *nsize, const int *c1, int *halved) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nn) return;
    if (c1[v] == 0 || c1[v] == nsize[v]) halved[v] = 1;
}

__global__ void kd_stats_kernel(const int64_t *q, int d, int64_t n, const int32_t *node_of, long long *nmin,
                                long long *nmax, unsigned long long *nsum) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    const int64_t i = e / d;
    const int a = int(e % d);
    const int32_t v = node_of[i];
    if (v < 0) return;
    const long long x = q[e];
    atomicMin(&nmin[int64_t(v) * d + a], x);
    atomicMax(&nmax[int64_t(v) * d + a], x);
    atomicAdd(&nsum[int64_t(v) * d + a], static_cast<unsigned long long>(x));
}

__global__ void kd_choose_kernel(int nn, int d, const long long *nmin, const long long *nmax,
                                 const unsigned long long *nsum, int *kdim, long long *ksum, int *halved,
                                 long long *lo, long long *hi) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nn) return;
    long long best = -1;
    int bk = 0;
    for (int a = 0; a < d; ++a) {
        const long long sp = nmax[int64_t(v) * d + a] - nmin[int64_t(v) * d + a];
        if (sp > best) {
            best = sp;
            bk = a;
        }
    }
    kdim[v] = bk;
    ksum[v] = static_cast<long long>(nsum[int64_t(v) * d + bk]);
    halved[v] = best == 0 ? 1 : 0;
    lo[v] = nmin[int64_t(v) * d + bk];
    hi[v] = nmax[int64_t(v) * d + bk];
}

__global__ void kd_label_kernel(int64_t n, int d, const int64_t *q, const int32_t *node_of, const int64_t *nsize,
                                const int *kdim, const long long *ksum, int8_t *label, int *c1) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0) return;
    const long long x = q[i * d + kdim[v]];
    const int lab = x * nsize[v] <= ksum[v] ? 0 : 1;
    label[i] = int8_t(lab);
    if (lab) atomicAdd(&c1[v], 1);
}

// 100 x the smaller side below the larger one: the median split is needed.
__global__ void kd_balance_kernel(int nn, const int64_t *nsize, const int *c1, const int *halved, int *need,
                                  int *any) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nn) return;
    const int64_t c0 = nsize[v] - c1[v];
    const int64_t small = c0 < c1[v] ? c0 : c1[v], large = c0 < c1[v] ? c1[v] : c0;
    need[v] = (!halved[v] && 100 * small < large) ? 1 : 0;
    if (need[v]) atomicAdd(any, 1);
}

// Bisection for the smallest value v* with count(x <= v*) >= floor(m / 2)
// in the nodes that need the median (exact, order-free counts).
__global__ void kd_med_count_kernel(int64_t n, int d, const int64_t *q, const int32_t *node_of, const int *kdim,
                                    const int *need, const long long *lo, const long long *hi, int *cnt,
                                    int strict) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0 || !need[v]) return;
    const long long x = q[i * d + kdim[v]];
    // strict = 0: count x <= mid (mid = lo + (hi - lo) / 2); strict = 1: count x < lo
    const long long mid = lo[v] + ((hi[v] - lo[v]) >> 1);
    if (strict ? x < lo[v] : x <= mid) atomicAdd(&cnt[v], 1);
}
__global__ void kd_med_step_kernel(int nn, const int64_t *nsize, const int *need, long long *lo, long long *hi,
                                   int *cnt) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nn) return;
    if (need[v] && lo[v] < hi[v]) {
        const long long mid = lo[v] + ((hi[v] - lo[v]) >> 1);
        if (cnt[v] >= nsize[v] / 2) hi[v] = mid;
        else lo[v] = mid + 1;
    }
    cnt[v] = 0;
}
// flags of the rows equal to v* (ranked by a scan), then the median labels:
// x < v* first, and the first floor(m / 2) - count(x < v*) rows equal to v*
__global__ void kd_med_eq_kernel(int64_t n, int d, const int64_t *q, const int32_t *node_of, const int *kdim,
                                 const int *need, const long long *lo, int32_t *eq) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    eq[i] = (v >= 0 && need[v] && q[i * d + kdim[v]] == lo[v]) ? 1 : 0;
}
__global__ void kd_med_label_kernel(int64_t n, int d, const int64_t *q, const int32_t *node_of, const int64_t *nbeg,
                                    const int64_t *nsize, const int *kdim, const int *need, const long long *lo,
                                    const int *cless, const int64_t *eqscan, int8_t *label) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0 || !need[v]) return;
    const long long x = q[i * d + kdim[v]];
    const int64_t room = nsize[v] / 2 - cless[v];
    const int64_t rank = eqscan[i] - eqscan[nbeg[v]];
    label[i] = int8_t((x < lo[v] || (x == lo[v] && rank < room)) ? 0 : 1);
}

// Exact integer sums of one node's coordinates and their products: a CTA
// walks a contiguous range of rows (which may cross node boundaries) and
// adds its partial sums to the node at each boundary.  Entry p < d*d is
// the pair (p / d, p % d), entry d*d + a the coordinate a.
constexpr int kPcaRows = 1024;
constexpr int kPcaMaxD = 64;
__global__ void pca_sums_kernel(const int64_t *q, int d, int64_t n, const int32_t *node_of,
                                unsigned long long *sums) {
    const int64_t r0 = int64_t(blockIdx.x) * kPcaRows, r1 = min(n, r0 + kPcaRows);
    const int np = d * d + d;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int a = p < d * d ? p / d : p - d * d, b = p < d * d ? p % d : -1;
        long long acc = 0;
        int32_t cur = -1;
        for (int64_t i = r0; i < r1; ++i) {
            const int32_t v = node_of[i];
            if (v != cur) {
                if (cur >= 0 && acc) atomicAdd(&sums[int64_t(cur) * np + p], static_cast<unsigned long long>(acc));
                acc = 0;
                cur = v;
            }
            if (v < 0) continue;
            const long long x = q[i * d + a];
            acc += b < 0 ? x : x * q[i * d + b];
        }
        if (cur >= 0 && acc) atomicAdd(&sums[int64_t(cur) * np + p], static_cast<unsigned long long>(acc));
    }
}

// One CTA per node, thread a <-> coordinate a: mean, covariance and the
// power iteration in the prescribed order of rounded operations.
constexpr int kPcaIters = 64;
__global__ void pca_direction_kernel(int d, const int64_t *nsize, const unsigned long long *sums, double *mu_out,
                                     double *v_out, int *halved) {
    __shared__ double C[kPcaMaxD][kPcaMaxD + 1];
    __shared__ double mu[kPcaMaxD], v[kPcaMaxD], w[kPcaMaxD];
    __shared__ double nrm;
    __shared__ int zero;
    const int node = blockIdx.x, a = threadIdx.x;
    const int np = d * d + d;
    const unsigned long long *S = sums + int64_t(node) * np;
    const double m = double(nsize[node]);
    if (a == 0) zero = 1;
    if (a < d) mu[a] = __ddiv_rn(__ll2double_rn(static_cast<long long>(S[d * d + a])), m);
    __syncthreads();
    if (a < d) {
        for (int b = 0; b < d; ++b) {
            const double c = __dsub_rn(__ddiv_rn(__ll2double_rn(static_cast<long long>(S[a * d + b])), m),
                                       __dmul_rn(mu[a], mu[b]));
            C[a][b] = c;
            if (c != 0.0) zero = 0;
        }
        v[a] = a == 0 ? 1.0 : 0.0;
    }
    __syncthreads();
    if (zero) {
        if (a == 0) halved[node] = 1;
        return;
    }
    for (int it = 0; it < kPcaIters; ++it) {
        if (a < d) {
            double acc = 0.0;
            for (int b = 0; b < d; ++b) acc = __dadd_rn(acc, __dmul_rn(C[a][b], v[b]));
            w[a] = acc;
        }
        __syncthreads();
        if (a == 0) {
            double s2 = 0.0;
            for (int b = 0; b < d; ++b) s2 = __dadd_rn(s2, __dmul_rn(w[b], w[b]));
            nrm = s2;
        }
        __syncthreads();
        if (nrm == 0.0) break;  // uniform across the block
        const double r = __dsqrt_rn(nrm);
        if (a < d) v[a] = __ddiv_rn(w[a], r);
        __syncthreads();
    }
    if (a == 0) {
        int big = 0;
        for (int b = 1; b < d; ++b)
            if (fabs(v[b]) > fabs(v[big])) big = b;
        nrm = v[big] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    if (a < d) {
        mu_out[int64_t(node) * d + a] = mu[a];
        v_out[int64_t(node) * d + a] = nrm < 0.0 ? -v[a] : v[a];
    }
}

__global__ void pca_label_kernel(int64_t n, int d, const int64_t *q, const int32_t *node_of, const double *mu,
                                 const double *vdir, const int *halved, int8_t *label, int *c1) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = node_of[i];
    if (v < 0 || halved[v]) return;
    double p = 0.0;
    for (int a = 0; a < d; ++a)
        p = __dadd_rn(p, __dmul_rn(__dsub_rn(__ll2double_rn(q[i * d + a]), mu[int64_t(v) * d + a]),
                                   vdir[int64_t(v) * d + a]));
    const int lab = p > 0.0 ? 1 : 0;
    label[i] = int8_t(lab);
    if (lab) atomicAdd(&c1[v], 1);
}

}  // namespace

// Quantization exponent for m points in d dimensions with max |x| = maxabs:
// the largest k for which 4 d m (2^k max|x|)^2 stays below 2^63.
static int quant_exponent(float maxabs, int d, int64_t m) {
    int L = 0;
    uint64_t v = uint64_t(4) * uint64_t(d) * uint64_t(m) - 1;
    while (v) { ++L; v >>= 1; }
    const int t = (63 - L) / 2;
    if (!(maxabs > 0.f)) return 0;
    int e;
    std::frexp(double(maxabs), &e);
    return t - e;
}

int cluster(Ctx *c, const float *X, int64_t n, int d, int leaf, uint64_t seed, int32_t *perm_out,
            std::vector<int32_t> &tb, std::vector<int32_t> &te, std::vector<int32_t> &tl, std::vector<int32_t> &tr,
            std::vector<int32_t> &tp, std::vector<int32_t> &tv, const std::vector<int64_t> *segments, int method) {
    tb.clear(); te.clear(); tl.clear(); tr.clear(); tp.clear(); tv.clear();
    if (n == 0) return KRR_OK;
    if (d > kMaxD) return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_cluster: d > 1024");
    if (method < KRR_ORDER_TWO_MEANS || method > KRR_ORDER_PCA)
        return fail(KRR_ERR_INVALID_ARG, "krr_cluster: unknown ordering");
    if (method == KRR_ORDER_PCA && d > kPcaMaxD)
        return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_cluster: the principal-direction ordering supports d <= 64");
    cudaStream_t st = c->stream;
    // segments (one, the whole set, unless given)
    std::vector<int64_t> seg = segments ? *segments : std::vector<int64_t>{0, n};
    const int nseg = int(seg.size()) - 1;
    if (nseg < 1 || seg[0] != 0 || seg[nseg] != n) return fail(KRR_ERR_INVALID_ARG, "krr_cluster: bad segments");
    for (int p = 0; p < nseg; ++p)
        if (seg[p + 1] <= seg[p]) return fail(KRR_ERR_INVALID_ARG, "krr_cluster: empty segment");
    // --- quantization (per segment)
    DBuf<unsigned int> mx(c, nseg);
    DBuf<int> bad(c, 1), dkexp(c, nseg);
    DBuf<int64_t> dseg(c, nseg + 1);
    if (!mx.get() || !bad.get() || !dkexp.get() || !dseg.get()) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
    KRR_CUDA(cudaMemcpyAsync(dseg.get(), seg.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, st));
    KRR_CUDA(cudaMemsetAsync(mx.get(), 0, nseg * 4, st));
    KRR_CUDA(cudaMemsetAsync(bad.get(), 0, 4, st));
    int64_t longest = 0;
    for (int p = 0; p < nseg; ++p) longest = std::max(longest, seg[p + 1] - seg[p]);
    const dim3 sg(unsigned(std::min<int64_t>(1024, cdiv(longest * d, kTB))), unsigned(nseg));
    { absmax_seg_kernel<<<sg, kTB, 0, st>>>(X, d, dseg.get(), mx.get(), bad.get()); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    std::vector<unsigned int> hmx(nseg);
    int hbad = 0;
    KRR_CUDA(cudaMemcpyAsync(hmx.data(), mx.get(), nseg * 4, cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaMemcpyAsync(&hbad, bad.get(), 4, cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaStreamSynchronize(st));
    if (hbad) return fail(KRR_ERR_NONFINITE_INPUT, "krr_cluster: NaN or Inf in X");
    std::vector<int> hk(nseg);
    bool narrow = true;  // every segment has n d >= 3: differences fit in 32 bits
    for (int p = 0; p < nseg; ++p) narrow = narrow && (seg[p + 1] - seg[p]) * int64_t(d) >= 3;
    for (int p = 0; p < nseg; ++p) {
        float maxabs;
        std::memcpy(&maxabs, &hmx[p], 4);
        hk[p] = quant_exponent(maxabs, d, seg[p + 1] - seg[p]);
    }
    KRR_CUDA(cudaMemcpyAsync(dkexp.get(), hk.data(), nseg * 4, cudaMemcpyHostToDevice, st));
    DBuf<int64_t> q(c, size_t(n) * d), q2(c, size_t(n) * d);
    DBuf<int32_t> pa(c, n), pb(c, n), node_of(c, n), zflag(c, n);
    DBuf<int8_t> label(c, n);
    DBuf<int64_t> zscan(c, n), bsum(c, cdiv(n, kTB) + 1);
    if (!q.get() || !q2.get() || !pa.get() || !pb.get() || !node_of.get() || !zflag.get() || !label.get() ||
        !zscan.get() || !bsum.get())
        return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
    if (nseg == 1)
        { quantize_kernel<<<unsigned(cdiv(n * d, kTB)), kTB, 0, st>>>(X, n * d, std::ldexp(1.0, hk[0]), q.get()); ::krr::count_launch(); }
    else
        { quantize_seg_kernel<<<sg, kTB, 0, st>>>(X, d, dseg.get(), dkexp.get(), q.get()); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    {
        std::vector<int32_t> idp(n);
        for (int64_t i = 0; i < n; ++i) idp[i] = int32_t(i);
        KRR_CUDA(cudaMemcpyAsync(pa.get(), idp.data(), n * 4, cudaMemcpyHostToDevice, st));
        KRR_CUDA(cudaStreamSynchronize(st));
    }
    int64_t *qc = q.get(), *qn = q2.get();
    int32_t *pc = pa.get(), *pn = pb.get();

    // --- tree, created level by level (ids in creation order; postorder at the end)
    struct Node { int64_t b, m, base; int left, right, parent, level; };
    std::vector<Node> nodes;
    std::vector<int> active;
    // balanced binary tree over the segments; the segments' roots start the two-means recursion
    {
        struct Item { int s0, s1, node; };
        nodes.push_back({0, n, 0, -1, -1, -1, 0});
        std::vector<Item> todo{{0, nseg, 0}};
        while (!todo.empty()) {
            const Item it = todo.back();
            todo.pop_back();
            if (it.s1 - it.s0 == 1) {
                nodes[it.node].base = seg[it.s0];
                if (nodes[it.node].m > leaf) active.push_back(it.node);
                continue;
            }
            const int mid = (it.s0 + it.s1) / 2;
            const int li = int(nodes.size());
            const int lv = nodes[it.node].level + 1;
            nodes.push_back({seg[it.s0], seg[mid] - seg[it.s0], 0, -1, -1, it.node, lv});
            nodes.push_back({seg[mid], seg[it.s1] - seg[mid], 0, -1, -1, it.node, lv});
            nodes[it.node].left = li;
            nodes[it.node].right = li + 1;
            todo.push_back({mid, it.s1, li + 1});
            todo.push_back({it.s0, mid, li});
        }
        std::sort(active.begin(), active.end(), [&](int a, int b) { return nodes[a].b < nodes[b].b; });
    }
    DBuf<int32_t> running(c, 2);
    if (!running.get()) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
    // pinned host flags and events of the pipelined convergence check
    struct IterSync {
        int *pin = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~IterSync() {
            if (pin) cudaFreeHost(pin);
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
        }
    } isync;
    KRR_CUDA(cudaMallocHost(&isync.pin, 2 * sizeof(int)));
    KRR_CUDA(cudaEventCreateWithFlags(&isync.ev[0], cudaEventDisableTiming));
    KRR_CUDA(cudaEventCreateWithFlags(&isync.ev[1], cudaEventDisableTiming));
    int *hrun_pin = isync.pin;
    cudaEvent_t *iter_ev = isync.ev;
    DBuf<int32_t> eqflag;
    if (method == KRR_ORDER_KD && !eqflag.reset(c, n)) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
    DBuf<unsigned long long> sdist;  // wide rows: squared distance of each row to its node's first seed
    if (method == KRR_ORDER_TWO_MEANS && d >= kWarpDim && !sdist.reset(c, n))
        return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
    while (!active.empty()) {
        const int nn = int(active.size());
        std::vector<int64_t> hb(nn), hs(nn), hbase(nn);
        for (int k = 0; k < nn; ++k) {
            hb[k] = nodes[active[k]].b;
            hs[k] = nodes[active[k]].m;
            hbase[k] = nodes[active[k]].base;
        }
        DBuf<int64_t> db(c, nn), ds(c, nn), dbase(c, nn), dcnt0(c, nn);
        DBuf<NodeState> dns(c, nn);
        if (!db.get() || !ds.get() || !dbase.get() || !dcnt0.get() || !dns.get())
            return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
        KRR_CUDA(cudaMemcpyAsync(db.get(), hb.data(), nn * 8, cudaMemcpyHostToDevice, st));
        KRR_CUDA(cudaMemcpyAsync(ds.get(), hs.data(), nn * 8, cudaMemcpyHostToDevice, st));
        KRR_CUDA(cudaMemcpyAsync(dbase.get(), hbase.data(), nn * 8, cudaMemcpyHostToDevice, st));
        KRR_CUDA(cudaMemsetAsync(node_of.get(), 0xFF, n * 4, st));
        { mark_nodes_kernel<<<nn, kTB, 0, st>>>(nn, db.get(), ds.get(), node_of.get()); ::krr::count_launch(); }
        const int64_t nblk = cdiv(n, kTB);
        const unsigned gn = unsigned(cdiv(n, kTB)), gv = unsigned(cdiv(nn, 128));
        if (method == KRR_ORDER_TWO_MEANS) {
            if (d >= kWarpDim) {
                DBuf<unsigned long long> stot(c, nn);
                if (!stot.get()) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
                KRR_TRY(launch_seed_wide(c, nn, gn, qc, d, n, db.get(), ds.get(), dbase.get(), node_of.get(), dns.get(),
                                         seed, sdist.get(), stot.get(), narrow));
            } else {
                { seed_kernel<<<nn, kTB, 0, st>>>(qc, d, db.get(), ds.get(), dbase.get(), dns.get(), seed, narrow); ::krr::count_launch(); }
            }
            KRR_CUDA(cudaGetLastError());
            // The count of nodes still running is read one iteration late:
            // iteration t + 1 is queued before the host waits for t's count
            // (an iteration after the last is a no-op: every node is done).
            for (int iter = 0; iter <= kMaxIter; ++iter) {
                const int slot = iter & 1;
                KRR_CUDA(cudaMemsetAsync(running.get() + slot, 0, 4, st));
                if (d >= kWarpDim)
                    KRR_TRY(launch_assign_wide(c, qc, d, n, node_of.get(), dns.get(), label.get(), narrow));
                else
                    { assign_kernel<<<gn, kTB, size_t(2) * d * sizeof(unsigned long long), st>>>(qc, d, n, node_of.get(), dns.get(), label.get(), narrow); ::krr::count_launch(); }
                { update_kernel<<<nn, d >= kWarpDim ? kTB : 128, 0, st>>>(nn, d, ds.get(), dns.get(), running.get() + slot); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
                KRR_CUDA(cudaMemcpyAsync(hrun_pin + slot, running.get() + slot, 4, cudaMemcpyDeviceToHost, st));
                KRR_CUDA(cudaEventRecord(iter_ev[slot], st));
                if (iter > 0) {
                    KRR_CUDA(cudaEventSynchronize(iter_ev[slot ^ 1]));
                    if (hrun_pin[slot ^ 1] == 0) break;
                }
            }
            { finalize_labels_kernel<<<gn, kTB, 0, st>>>(n, node_of.get(), db.get(), ds.get(), dns.get(), label.get(),
                                                        zflag.get()); ::krr::count_launch(); }
        } else {
            DBuf<int> halved(c, nn), c1(c, nn);
            if (!halved.get() || !c1.get()) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
            KRR_CUDA(cudaMemsetAsync(c1.get(), 0, nn * 4, st));
            if (method == KRR_ORDER_NATURAL) {
                std::vector<int> ones(nn, 1);
                KRR_CUDA(cudaMemcpyAsync(halved.get(), ones.data(), nn * 4, cudaMemcpyHostToDevice, st));
            } else if (method == KRR_ORDER_KD) {
                DBuf<long long> nmin(c, size_t(nn) * d), nmax(c, size_t(nn) * d), ksum(c, nn), lo(c, nn), hi(c, nn);
                DBuf<unsigned long long> nsum(c, size_t(nn) * d);
                DBuf<int> kdim(c, nn), need(c, nn), cnt(c, nn), any(c, 1);
                if (!nmin.get() || !nmax.get() || !ksum.get() || !lo.get() || !hi.get() || !nsum.get() || !kdim.get() ||
                    !need.get() || !cnt.get() || !any.get())
                    return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
                std::vector<long long> big(size_t(nn) * d, 0x7FFFFFFFFFFFFFFFll), small(size_t(nn) * d, -0x7FFFFFFFFFFFFFFFll - 1);
                KRR_CUDA(cudaMemcpyAsync(nmin.get(), big.data(), big.size() * 8, cudaMemcpyHostToDevice, st));
                KRR_CUDA(cudaMemcpyAsync(nmax.get(), small.data(), small.size() * 8, cudaMemcpyHostToDevice, st));
                KRR_CUDA(cudaMemsetAsync(nsum.get(), 0, size_t(nn) * d * 8, st));
                KRR_CUDA(cudaMemsetAsync(any.get(), 0, 4, st));
                KRR_CUDA(cudaMemsetAsync(cnt.get(), 0, nn * 4, st));
                { kd_stats_kernel<<<unsigned(cdiv(n * d, kTB)), kTB, 0, st>>>(qc, d, n, node_of.get(), nmin.get(), nmax.get(), nsum.get()); ::krr::count_launch(); }
                { kd_choose_kernel<<<gv, 128, 0, st>>>(nn, d, nmin.get(), nmax.get(), nsum.get(), kdim.get(), ksum.get(),
                                                       halved.get(), lo.get(), hi.get()); ::krr::count_launch(); }
                { kd_label_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), ds.get(), kdim.get(), ksum.get(), label.get(), c1.get()); ::krr::count_launch(); }
                { kd_balance_kernel<<<gv, 128, 0, st>>>(nn, ds.get(), c1.get(), halved.get(), need.get(), any.get()); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
                int hany = 0;
                KRR_CUDA(cudaMemcpyAsync(&hany, any.get(), 4, cudaMemcpyDeviceToHost, st));
                KRR_CUDA(cudaStreamSynchronize(st));
                if (hany) {
                    // bisection on the value (64 halvings cover any int64 range)
                    for (int it = 0; it < 64; ++it) {
                        { kd_med_count_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), kdim.get(), need.get(), lo.get(), hi.get(), cnt.get(), 0); ::krr::count_launch(); }
                        { kd_med_step_kernel<<<gv, 128, 0, st>>>(nn, ds.get(), need.get(), lo.get(), hi.get(), cnt.get()); ::krr::count_launch(); }
                    }
                    { kd_med_count_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), kdim.get(), need.get(), lo.get(), hi.get(), cnt.get(), 1); ::krr::count_launch(); }
                    { kd_med_eq_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), kdim.get(), need.get(), lo.get(), eqflag.get()); ::krr::count_launch(); }
                    { scan_blocks_kernel<<<unsigned(nblk), kTB, 0, st>>>(eqflag.get(), n, zscan.get(), bsum.get()); ::krr::count_launch(); }
                    { scan_sums_kernel<<<1, kTB, 0, st>>>(bsum.get(), nblk); ::krr::count_launch(); }
                    { scan_add_kernel<<<unsigned(nblk), kTB, 0, st>>>(zscan.get(), n, bsum.get(), nullptr); ::krr::count_launch(); }
                    { kd_med_label_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), db.get(), ds.get(), kdim.get(), need.get(), lo.get(), cnt.get(), zscan.get(), label.get()); ::krr::count_launch(); }
                    KRR_CUDA(cudaGetLastError());
                    // the median labels replace the mean ones: recount the second side
                    KRR_CUDA(cudaMemsetAsync(c1.get(), 0, nn * 4, st));
                    { count_second_kernel<<<gn, kTB, 0, st>>>(n, node_of.get(), label.get(), c1.get()); ::krr::count_launch(); }
                }
            } else {  // KRR_ORDER_PCA
                const int np = d * d + d;
                DBuf<unsigned long long> sums(c, size_t(nn) * np);
                DBuf<double> mu(c, size_t(nn) * d), vdir(c, size_t(nn) * d);
                if (!sums.get() || !mu.get() || !vdir.get()) return fail(KRR_ERR_OOM, "krr_cluster: out of memory");
                KRR_CUDA(cudaMemsetAsync(sums.get(), 0, size_t(nn) * np * 8, st));
                KRR_CUDA(cudaMemsetAsync(halved.get(), 0, nn * 4, st));
                { pca_sums_kernel<<<unsigned(cdiv(n, kPcaRows)), kTB, 0, st>>>(qc, d, n, node_of.get(), sums.get()); ::krr::count_launch(); }
                { pca_direction_kernel<<<nn, kPcaMaxD, 0, st>>>(d, ds.get(), sums.get(), mu.get(), vdir.get(), halved.get()); ::krr::count_launch(); }
                { pca_label_kernel<<<gn, kTB, 0, st>>>(n, d, qc, node_of.get(), mu.get(), vdir.get(), halved.get(), label.get(), c1.get()); ::krr::count_launch(); }
                KRR_CUDA(cudaGetLastError());
            }
            if (method != KRR_ORDER_NATURAL)
                { empty_side_kernel<<<gv, 128, 0, st>>>(nn, ds.get(), c1.get(), halved.get()); ::krr::count_launch(); }
            { finalize_generic_kernel<<<gn, kTB, 0, st>>>(n, node_of.get(), db.get(), ds.get(), halved.get(), label.get(),
                                                         zflag.get()); ::krr::count_launch(); }
            KRR_CUDA(cudaGetLastError());
            KRR_CUDA(cudaStreamSynchronize(st));  // the level's scratch is freed at the end of this block
        }
        { scan_blocks_kernel<<<unsigned(nblk), kTB, 0, st>>>(zflag.get(), n, zscan.get(), bsum.get()); ::krr::count_launch(); }
        { scan_sums_kernel<<<1, kTB, 0, st>>>(bsum.get(), nblk); ::krr::count_launch(); }
        { scan_add_kernel<<<unsigned(nblk), kTB, 0, st>>>(zscan.get(), n, bsum.get(), nullptr); ::krr::count_launch(); }
        if (d >= kWarpDim)
            { partition_wide_kernel<<<unsigned(cdiv(n * 32, kTB)), kTB, 0, st>>>(n, d, node_of.get(), db.get(), ds.get(),
                                                                              label.get(), zscan.get(), zflag.get(), qc,
                                                                              pc, qn, pn, dcnt0.get()); ::krr::count_launch(); }
        else
            { partition_kernel<<<unsigned(nblk), kTB, 0, st>>>(n, d, node_of.get(), db.get(), ds.get(), label.get(),
                                                              zscan.get(), zflag.get(), qc, pc, qn, pn, dcnt0.get()); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
        std::vector<int64_t> hc0(nn);
        KRR_CUDA(cudaMemcpyAsync(hc0.data(), dcnt0.get(), nn * 8, cudaMemcpyDeviceToHost, st));
        KRR_CUDA(cudaStreamSynchronize(st));
        std::swap(qc, qn);
        std::swap(pc, pn);
        std::vector<int> next;
        for (int k = 0; k < nn; ++k) {
            const int v = active[k];
            const Node par = nodes[v];
            const int64_t c0 = hc0[k];
            const int li = int(nodes.size());
            nodes.push_back({par.b, c0, par.base, -1, -1, v, par.level + 1});
            nodes.push_back({par.b + c0, par.m - c0, par.base, -1, -1, v, par.level + 1});
            nodes[v].left = li;
            nodes[v].right = li + 1;
            if (c0 > leaf) next.push_back(li);
            if (par.m - c0 > leaf) next.push_back(li + 1);
        }
        active.swap(next);
    }
    KRR_CUDA(cudaMemcpyAsync(perm_out, pc, n * 4, cudaMemcpyDeviceToDevice, st));
    KRR_CUDA(cudaStreamSynchronize(st));

    // --- postorder numbering (left subtree, right subtree, node)
    const int N = int(nodes.size());
    std::vector<int> post(N, -1), order;
    order.reserve(N);
    std::vector<std::pair<int, int>> stack;
    stack.push_back({0, 0});
    while (!stack.empty()) {
        auto &top = stack.back();
        const Node &nd = nodes[top.first];
        if (nd.left < 0 || top.second == 2) {
            post[top.first] = int(order.size());
            order.push_back(top.first);
            stack.pop_back();
        } else {
            const int child = top.second == 0 ? nd.left : nd.right;
            top.second += 1;
            stack.push_back({child, 0});
        }
    }
    tb.resize(N); te.resize(N); tl.resize(N); tr.resize(N); tp.resize(N); tv.resize(N);
    for (int k = 0; k < N; ++k) {
        const Node &nd = nodes[order[k]];
        tb[k] = int32_t(nd.b);
        te[k] = int32_t(nd.b + nd.m);
        tl[k] = nd.left < 0 ? -1 : post[nd.left];
        tr[k] = nd.right < 0 ? -1 : post[nd.right];
        tp[k] = nd.parent < 0 ? -1 : post[nd.parent];
        tv[k] = nd.level;
    }
    return KRR_OK;
}

}  // namespace krr

using namespace krr;

static int cluster_entry(krr_ctx *k, const float *X, int64_t n, int32_t d, int32_t leaf, uint64_t seed,
                         int32_t *perm, int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes,
                         const std::vector<int64_t> *seg, int method = KRR_ORDER_TWO_MEANS) {
    if (!k || (n > 0 && (!X || !perm)) || n < 0 || d <= 0 || leaf < 1 || !n_nodes)
        return fail(KRR_ERR_INVALID_ARG, "krr_cluster: bad arguments");
    if (n > 0x7FFFFFFF) return fail(KRR_ERR_INVALID_ARG, "krr_cluster: n too large");
    std::vector<int32_t> tb, te, tl, tr, tp, tv;
    KRR_TRY(cluster(&k->c, X, n, d, leaf, seed, perm, tb, te, tl, tr, tp, tv, seg, method));
    const int N = int(tb.size());
    *n_nodes = N;
    if (N > max_nodes) return fail(KRR_ERR_INVALID_ARG, "krr_cluster: max_nodes too small");
    if (N > 0 && (!tree.begin || !tree.end || !tree.left || !tree.right || !tree.parent || !tree.level))
        return fail(KRR_ERR_INVALID_ARG, "krr_cluster: tree arrays are NULL");
    for (int i = 0; i < N; ++i) {
        tree.begin[i] = tb[i];
        tree.end[i] = te[i];
        tree.left[i] = tl[i];
        tree.right[i] = tr[i];
        tree.parent[i] = tp[i];
        tree.level[i] = tv[i];
    }
    return KRR_OK;
}

extern "C" int krr_cluster(krr_ctx *k, const float *X, int64_t n, int32_t d, int32_t leaf, uint64_t seed,
                           int32_t *perm, int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes) {
    return cluster_entry(k, X, n, d, leaf, seed, perm, max_nodes, tree, n_nodes, nullptr);
}

extern "C" int krr_cluster_batched(krr_ctx *k, const float *X, int64_t n, int32_t d, int32_t nprob,
                                   const int64_t *offsets, int32_t leaf, uint64_t seed, int32_t *perm,
                                   int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes) {
    if (nprob < 1 || !offsets) return fail(KRR_ERR_INVALID_ARG, "krr_cluster_batched: bad arguments");
    std::vector<int64_t> seg(offsets, offsets + nprob + 1);
    return cluster_entry(k, X, n, d, leaf, seed, perm, max_nodes, tree, n_nodes, &seg);
}

extern "C" int krr_order(krr_ctx *k, const float *X, int64_t n, int32_t d, int32_t leaf, int32_t ordering,
                         uint64_t seed, int32_t *perm, int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes) {
    return cluster_entry(k, X, n, d, leaf, seed, perm, max_nodes, tree, n_nodes, nullptr, ordering);
}
