// Data-preparation kernels: feature standardization, row gathers, the
// augmented FP16 operands of the fused product, FP16 transposes, and the
// method's random block (Philox4x64-10 + Box-Muller).
#include <algorithm>

#include "common.cuh"
#include "prep.cuh"

namespace krr {

// ----------------------------------------------------- standardization
// Column mean / population std in FP64 (Section 5.2 normalization).
// One block per column; each block reduces its column in a fixed order
// (strided partial sums, then a tree), so results are deterministic.
__global__ void col_stats_kernel(const float *X, int64_t n, int d, double *mean, double *stdv) {
    const int col = blockIdx.x;
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += double(X[i * d + col]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double mu = sh[0] / double(n);
    __syncthreads();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = double(X[i * d + col]) - mu;
        v += t * t;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = sqrt(sh[0] / double(n));
        mean[col] = mu;
        stdv[col] = sd > 0.0 ? sd : 1.0;
    }
}

__global__ void apply_standardize_kernel(float *X, int64_t n, int d, const double *mean, const double *stdv) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * d) return;
    const int col = int(k % d);
    X[k] = float((double(X[k]) - mean[col]) / stdv[col]);
}

int standardize(Ctx *c, float *X, int64_t n, int d, float *Xt, int64_t m, double *mean, double *stdv) {
    DBuf<double> mb, sb;
    double *mu = mean, *sd = stdv;
    if (!mu) {
        if (!mb.reset(c, d)) return fail(KRR_ERR_OOM, "standardize: out of memory");
        mu = mb.get();
    }
    if (!sd) {
        if (!sb.reset(c, d)) return fail(KRR_ERR_OOM, "standardize: out of memory");
        sd = sb.get();
    }
    { col_stats_kernel<<<d, 256, 0, c->stream>>>(X, n, d, mu, sd); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    if (Xt && m > 0) {
        { apply_standardize_kernel<<<unsigned(cdiv(m * d, 256)), 256, 0, c->stream>>>(Xt, m, d, mu, sd); ::krr::count_launch(); }
        KRR_CUDA(cudaGetLastError());
    }
    { apply_standardize_kernel<<<unsigned(cdiv(n * d, 256)), 256, 0, c->stream>>>(X, n, d, mu, sd); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// ----------------------------------------------------------- gathers
template <class Tin, class Tout>
__global__ void gather_rows_kernel(const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols,
                                   Tout *dst, int64_t ldd) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * cols) return;
    const int64_t i = k / cols;
    const int c = int(k % cols);
    dst[i * ldd + c] = Tout(src[int64_t(perm[i]) * lds + c]);
}

template <class Tin, class Tout>
__global__ void scatter_rows_kernel(const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols,
                                    Tout *dst, int64_t ldd) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * cols) return;
    const int64_t i = k / cols;
    const int c = int(k % cols);
    dst[int64_t(perm[i]) * ldd + c] = Tout(src[i * lds + c]);
}

template <class Tin, class Tout>
int gather_rows(Ctx *c, const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols, Tout *dst,
                int64_t ldd) {
    if (n * cols == 0) return KRR_OK;
    { gather_rows_kernel<Tin, Tout><<<unsigned(cdiv(n * cols, 256)), 256, 0, c->stream>>>(src, lds, perm, n, cols,
                                                                                          dst, ldd); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}
template <class Tin, class Tout>
int scatter_rows(Ctx *c, const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols, Tout *dst,
                 int64_t ldd) {
    if (n * cols == 0) return KRR_OK;
    { scatter_rows_kernel<Tin, Tout><<<unsigned(cdiv(n * cols, 256)), 256, 0, c->stream>>>(src, lds, perm, n, cols,
                                                                                           dst, ldd); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}
template int gather_rows<float, float>(Ctx *, const float *, int64_t, const int32_t *, int64_t, int, float *, int64_t);
template int gather_rows<float, double>(Ctx *, const float *, int64_t, const int32_t *, int64_t, int, double *,
                                        int64_t);
template int gather_rows<double, double>(Ctx *, const double *, int64_t, const int32_t *, int64_t, int, double *,
                                         int64_t);
template int scatter_rows<double, double>(Ctx *, const double *, int64_t, const int32_t *, int64_t, int, double *,
                                          int64_t);

__global__ void widen_kernel(const float *src, int64_t n, double *dst) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = double(src[k]);
}
int widen(Ctx *c, const float *src, int64_t n, double *dst) {
    if (n == 0) return KRR_OK;
    { widen_kernel<<<unsigned(cdiv(n, 256)), 256, 0, c->stream>>>(src, n, dst); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// ------------------------------------------- augmented FP16 operands
// Row i of the A operand (role 0) or the B operand (role 1) of the
// distance GEMM; see sample_tc.cu for the layout.  All splits are done in
// FP64 so every part is the correctly rounded remainder.
__global__ void augment_kernel(const float *X, int64_t rows, int d, double c, int role, __half *out, int kpad,
                               DevStatus *st) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float *x = X + i * d;
    __half *o = out + i * kpad;
    double nrm = 0.0;
    for (int k = 0; k < d; ++k) nrm += double(x[k]) * double(x[k]);
    // norms use the FP32 coordinates exactly as stored
    const double a = -c * nrm;
    bool overflow = fabs(a) > 60000.0;
    for (int k = 0; k < d; ++k) {
        if (role == 0) {
            const double v = double(x[k]);
            const __half hv = __double2half(v);
            const __half lv = __double2half(v - double(__half2float(hv)));
            o[k] = hv;
            o[d + k] = hv;
            o[2 * d + k] = lv;
        } else {
            const double v = 2.0 * c * double(x[k]);
            overflow |= fabs(v) > 60000.0;
            const __half hv = __double2half(v);
            const __half lv = __double2half(v - double(__half2float(hv)));
            o[k] = hv;
            o[d + k] = lv;
            o[2 * d + k] = hv;
        }
    }
    const __half h1 = __double2half(a);
    const double r1 = a - double(__half2float(h1));
    const __half h2 = __double2half(r1);
    const __half h3 = __double2half(r1 - double(__half2float(h2)));
    const __half one = __float2half(1.0f);
    const int base = 3 * d;
    if (role == 0) {
        o[base + 0] = h1;
        o[base + 1] = h2;
        o[base + 2] = h3;
        o[base + 3] = one;
        o[base + 4] = one;
        o[base + 5] = one;
    } else {
        o[base + 0] = one;
        o[base + 1] = one;
        o[base + 2] = one;
        o[base + 3] = h1;
        o[base + 4] = h2;
        o[base + 5] = h3;
    }
    for (int k = base + 6; k < kpad; ++k) o[k] = __float2half(0.0f);
    if (overflow) dev_fail(st, KRR_ERR_INVALID_ARG, 100);
}

int augment(Ctx *c, const float *X, int64_t rows, int d, double h, int role, __half *out, int kpad) {
    if (rows == 0) return KRR_OK;
    const double cc = 1.4426950408889634 / (2.0 * h * h);  // log2(e) / (2 h^2)
    { augment_kernel<<<unsigned(cdiv(rows, 128)), 128, 0, c->stream>>>(X, rows, d, cc, role, out, kpad, c->status); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// R (float, n x r, ldr) -> RT (FP16, rpad x ldrt); rows r..rpad-1 zero.
__global__ void transpose_half_kernel(const float *R, int64_t n, int r, int64_t ldr, __half *RT, int rpad,
                                      int64_t ldrt) {
    __shared__ float tile[32][33];
    const int64_t j0 = int64_t(blockIdx.x) * 32;
    const int c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t j = j0 + y;
        const int cc = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (j < n && cc < r) ? R[j * ldr + cc] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int cc = c0 + y;
        const int64_t j = j0 + threadIdx.x;
        if (cc < rpad && j < ldrt) RT[int64_t(cc) * ldrt + j] = __float2half(j < n ? tile[threadIdx.x][y] : 0.f);
    }
}

int transpose_half(Ctx *c, const float *R, int64_t n, int r, int64_t ldr, __half *RT, int rpad, int64_t ldrt) {
    dim3 grid(unsigned(cdiv(ldrt, 32)), unsigned(cdiv(rpad, 32)));
    { transpose_half_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(R, n, r, ldr, RT, rpad, ldrt); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

// S(i, c) += lambda * round16(R(i, c)) (mixed) or lambda * R(i, c).
template <class T>
__global__ void add_lambda_kernel(T *S, int64_t lds, const T *R, int64_t ldr, int64_t n, int r, double lambda,
                                  int round16) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * r) return;
    const int64_t i = k / r;
    const int c = int(k % r);
    double v = double(R[i * ldr + c]);
    if (round16) v = double(__half2float(__double2half(v)));
    S[i * lds + c] = T(double(S[i * lds + c]) + lambda * v);
}
template <class T>
int add_lambda(Ctx *c, T *S, int64_t lds, const T *R, int64_t ldr, int64_t n, int r, double lambda, bool round16) {
    if (lambda == 0.0 || n * r == 0) return KRR_OK;
    { add_lambda_kernel<T><<<unsigned(cdiv(n * r, 256)), 256, 0, c->stream>>>(S, lds, R, ldr, n, r, lambda,
                                                                            round16 ? 1 : 0); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}
template int add_lambda<float>(Ctx *, float *, int64_t, const float *, int64_t, int64_t, int, double, bool);
template int add_lambda<double>(Ctx *, double *, int64_t, const double *, int64_t, int64_t, int, double, bool);

// --------------------------------------------------------- random block
// Element (j, col) of R: Philox4x64-10 with key (seed, 0x52) at counter
// (j, col / 4, 0, 0); words (w0, w1) give columns 4g, 4g+1 and (w2, w3)
// give 4g+2, 4g+3 by Box-Muller with u = ((w >> 11) + 0.5) 2^-53.
__device__ __forceinline__ double u01(uint64_t w) { return (double(w >> 11) + 0.5) * 1.1102230246251565e-16; }

template <class T>
__global__ void random_block_kernel(int64_t n, int r, int col0, uint64_t seed, int round16, T *out, int64_t ld) {
    const int ng = (r + 3) / 4;
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * ng) return;
    const int64_t j = k / ng;
    const int g = int(k % ng);
    const U64x4 w = philox4x64_10(uint64_t(j), uint64_t(col0 / 4 + g), 0, 0, seed, kStreamR);
    double z[4];
    for (int p = 0; p < 2; ++p) {
        const double u1 = u01(w.v[2 * p]), u2 = u01(w.v[2 * p + 1]);
        const double rho = sqrt(-2.0 * log(u1));
        double s, cth;
        sincospi(2.0 * u2, &s, &cth);
        z[2 * p] = rho * cth;
        z[2 * p + 1] = rho * s;
    }
    for (int t = 0; t < 4; ++t) {
        const int cc = 4 * g + t;
        if (cc >= r) break;
        double v = z[t];
        if (round16) v = double(__half2float(__double2half(v)));
        out[j * ld + cc] = T(v);
    }
}

// The mixed path stores every element rounded to FP16, so FP32 arithmetic
// suffices wherever the value is not close to an FP16 rounding boundary.
// Same counters and words as random_block_kernel; the Box-Muller steps in
// FP32 with the argument reductions done exactly in integers:
//   u1 = (2 m1 + 1) 2^-54:  ln u1 = logf(u1) for u1 <= 1/2, else
//                           log1pf(-(1 - u1)) with 1 - u1 = (2^54 - 2 m1 - 1) 2^-54;
//   2 pi u2 = pi t 2^-53, t = 2 m2 + 1:  quadrant q = t >> 52 and the
//                           remainder f (or 1/2 - f, the octant's mirror) in
//                           [0, 1/4], then sincospif and a quarter-turn rotation.
// Each value is then within a few FP32 ulps of the exact one.  A value
// within 2^-19 (relative) of an FP16 rounding boundary is listed and
// recomputed by the FP64 steps (random_fix_kernel), so the stored FP16
// values are those of the FP64 computation.
__device__ __forceinline__ void box_muller_f32(uint64_t w1, uint64_t w2, float &z0, float &z1) {
    const uint64_t m1 = w1 >> 11, m2 = w2 >> 11;
    const uint64_t t1 = 2 * m1 + 1;  // u1 = t1 2^-54
    float L;
    if (t1 <= (uint64_t(1) << 53)) L = logf(__ull2float_rn(t1) * 5.551115123125783e-17f);  // 2^-54
    else L = log1pf(-(__ull2float_rn((uint64_t(1) << 54) - t1) * 5.551115123125783e-17f));
    const float rho = sqrtf(-2.f * L);
    const uint64_t t2 = 2 * m2 + 1;  // 2 u2 = t2 2^-53
    const int q = int(t2 >> 52);
    const uint64_t rem = t2 - (uint64_t(q) << 52);  // f = rem 2^-53 in [0, 1/2)
    float sf, cf;  // sin(pi f), cos(pi f)
    if (rem <= (uint64_t(1) << 51)) {
        sincospif(__ull2float_rn(rem) * 1.1102230246251565e-16f, &sf, &cf);  // 2^-53
    } else {
        float sg, cg;
        sincospif(__ull2float_rn((uint64_t(1) << 52) - rem) * 1.1102230246251565e-16f, &sg, &cg);
        sf = cg;
        cf = sg;
    }
    float c, sn;  // cos and sin of pi (q / 2 + f)
    if (q == 0) { c = cf; sn = sf; }
    else if (q == 1) { c = -sf; sn = cf; }
    else if (q == 2) { c = -cf; sn = -sf; }
    else { c = sf; sn = -cf; }
    z0 = rho * c;
    z1 = rho * sn;
}

__device__ __forceinline__ bool near_half_tie(float z) {
    const float e = 1.9073486328125e-06f;  // 2^-19
    return __float2half_rn(z * (1.f + e)) != __float2half_rn(z * (1.f - e));
}

__device__ __forceinline__ double box_muller_f64(const U64x4 &w, int t) {
    const int pr = t >> 1;
    const double u1 = u01(w.v[2 * pr]), u2 = u01(w.v[2 * pr + 1]);
    const double rho = sqrt(-2.0 * log(u1));
    double sv, cv;
    sincospi(2.0 * u2, &sv, &cv);
    return (t & 1) ? rho * sv : rho * cv;
}

__global__ void random_block16_kernel(int64_t n, int r, int col0, uint64_t seed, float *out, int64_t ld,
                                      uint64_t *fix, unsigned *nfix, unsigned cap) {
    const int ng = (r + 3) / 4;
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n * ng) return;
    const int64_t j = k / ng;
    const int g = int(k % ng);
    const U64x4 w = philox4x64_10(uint64_t(j), uint64_t(col0 / 4 + g), 0, 0, seed, kStreamR);
    float z[4];
    box_muller_f32(w.v[0], w.v[1], z[0], z[1]);
    box_muller_f32(w.v[2], w.v[3], z[2], z[3]);
    for (int t = 0; t < 4; ++t) {
        const int cc = 4 * g + t;
        if (cc >= r) break;
        if (near_half_tie(z[t])) {
            const unsigned slot = atomicAdd(nfix, 1u);
            if (slot < cap) fix[slot] = (uint64_t(j) << 24) | uint64_t(cc);
        }
        out[j * ld + cc] = __half2float(__float2half_rn(z[t]));
    }
}

// The listed values by the FP64 steps of random_block_kernel (every value
// when the list overflowed).
__global__ void random_fix_kernel(int64_t n, int r, int col0, uint64_t seed, float *out, int64_t ld,
                                  const uint64_t *fix, const unsigned *nfix, unsigned cap) {
    const unsigned cnt = *nfix;
    const int64_t total = cnt <= cap ? int64_t(cnt) : n * r;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t j;
        int cc;
        if (cnt <= cap) {
            j = int64_t(fix[e] >> 24);
            cc = int(fix[e] & 0xFFFFFFu);
        } else {
            j = e / r;
            cc = int(e % r);
        }
        const U64x4 w = philox4x64_10(uint64_t(j), uint64_t(col0 / 4 + cc / 4), 0, 0, seed, kStreamR);
        out[j * ld + cc] = __half2float(__double2half(box_muller_f64(w, cc & 3)));
    }
}

int random_block(Ctx *c, int64_t n, int r, int col0, uint64_t seed, int precision, void *out, int64_t ld) {
    if (col0 % 4 != 0) return fail(KRR_ERR_INVALID_ARG, "random_block: col0 must be a multiple of 4");
    if (n == 0 || r == 0) return KRR_OK;
    const int ng = (r + 3) / 4;
    const unsigned grid = unsigned(cdiv(n * ng, 256));
    if (precision == KRR_FP64)
        { random_block_kernel<double><<<grid, 256, 0, c->stream>>>(n, r, col0, seed, 0, static_cast<double *>(out), ld); ::krr::count_launch(); }
    else if (r >= (1 << 24))
        { random_block_kernel<float><<<grid, 256, 0, c->stream>>>(n, r, col0, seed, 1, static_cast<float *>(out), ld); ::krr::count_launch(); }
    else {
        // FP32 steps, the values near an FP16 rounding boundary redone in FP64
        // (about 1 % expected; a list of 1/16 of the block, all redone if it overflows)
        const unsigned cap = unsigned(std::min<int64_t>(int64_t(1) << 30, std::max<int64_t>(4096, n * r / 16)));
        DBuf<uint64_t> fix(c, cap);
        DBuf<unsigned> nfix(c, 1);
        if (!fix.get() || !nfix.get()) return fail(KRR_ERR_OOM, "random_block: out of memory");
        KRR_CUDA(cudaMemsetAsync(nfix.get(), 0, sizeof(unsigned), c->stream));
        { random_block16_kernel<<<grid, 256, 0, c->stream>>>(n, r, col0, seed, static_cast<float *>(out), ld, fix.get(), nfix.get(), cap); ::krr::count_launch(); }
        { random_fix_kernel<<<unsigned(2 * c->num_sms), 256, 0, c->stream>>>(n, r, col0, seed, static_cast<float *>(out), ld, fix.get(), nfix.get(), cap); ::krr::count_launch(); }
    }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

}  // namespace krr
