// FP64 fused kernel x block product on the CUDA cores: the "plain"
// comparator of the tensor-core path.  Same operation,
//     S(i, :) = sum_j w_ij exp(-||xa_i - xb_j||^2 / (2 h^2)) R(j, :),
// with the kernel evaluated in the difference form (paper Eq. (1)) and
// never stored: each CTA owns 64 rows x 64 columns of S and streams
// 32-row tiles of Xb and R through shared memory.
#include "common.cuh"
#include "prep.cuh"

namespace krr {

namespace {
constexpr int F_BM = 64, F_BC = 64, F_BJ = 32, F_MAXD = 64;

__global__ void __launch_bounds__(256) sample_f64_kernel(const double *Xa, int64_t ma, const double *Xb, int64_t nb,
                                                         int d, double inv2h2, const double *R, int r, int64_t ldr,
                                                         const int32_t *leaf_a, const int32_t *leaf_b, double *S,
                                                         int64_t lds, const int32_t *grp_a, const int32_t *grp_b,
                                                         const int64_t *off_b) {
    __shared__ double sxa[F_BM][F_MAXD + 1];
    __shared__ double sxb[F_BJ][F_MAXD + 1];
    __shared__ double sk[F_BM][F_BJ + 1];
    __shared__ double sr[F_BJ][F_BC + 1];
    const int64_t i0 = int64_t(blockIdx.x) * F_BM;
    const int c0 = blockIdx.y * F_BC;
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;  // 4x4 outputs per thread
    double acc[4][4] = {};
    for (int k = tid; k < F_BM * d; k += 256) {
        const int ii = k / d, kk = k % d;
        sxa[ii][kk] = (i0 + ii < ma) ? Xa[(i0 + ii) * d + kk] : 0.0;
    }
    // block-diagonal product: only the columns of the problems of this row block
    int64_t jlo = 0, jhi = nb;
    if (grp_a) {
        jlo = off_b[grp_a[i0]];
        jhi = off_b[grp_a[min(i0 + F_BM, ma) - 1] + 1];
    }
    for (int64_t j0 = jlo; j0 < jhi; j0 += F_BJ) {
        __syncthreads();
        for (int k = tid; k < F_BJ * d; k += 256) {
            const int jj = k / d, kk = k % d;
            sxb[jj][kk] = (j0 + jj < jhi) ? Xb[(j0 + jj) * d + kk] : 0.0;
        }
        for (int k = tid; k < F_BJ * F_BC; k += 256) {
            const int jj = k / F_BC, cc = k % F_BC;
            sr[jj][cc] = (j0 + jj < jhi && c0 + cc < r) ? R[(j0 + jj) * ldr + c0 + cc] : 0.0;
        }
        __syncthreads();
        for (int k = tid; k < F_BM * F_BJ; k += 256) {
            const int ii = k / F_BJ, jj = k % F_BJ;
            double s = 0.0;
            for (int kk = 0; kk < d; ++kk) {
                const double t = sxa[ii][kk] - sxb[jj][kk];
                s += t * t;
            }
            double kv = exp(-s * inv2h2);
            const int64_t i = i0 + ii, j = j0 + jj;
            if (j >= jhi || i >= ma) kv = 0.0;
            else if (leaf_a && leaf_b && leaf_a[i] == leaf_b[j]) kv = 0.0;
            else if (grp_a && grp_a[i] != grp_b[j]) kv = 0.0;
            sk[ii][jj] = kv;
        }
        __syncthreads();
        for (int jj = 0; jj < F_BJ; ++jj) {
            double kv[4], rv[4];
            for (int a = 0; a < 4; ++a) kv[a] = sk[tr * 4 + a][jj];
            for (int b = 0; b < 4; ++b) rv[b] = sr[jj][tc * 4 + b];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(kv[a], rv[b], acc[a][b]);
        }
    }
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + tr * 4 + a;
        if (i >= ma) continue;
        for (int b = 0; b < 4; ++b) {
            const int cc = c0 + tc * 4 + b;
            if (cc < r) S[i * lds + cc] = acc[a][b];
        }
    }
}
}  // namespace

int launch_sample_f64(Ctx *c, const double *Xa, int64_t ma, const double *Xb, int64_t nb, int d, double h,
                      const double *R, int r, int64_t ldr, const int32_t *leaf_a, const int32_t *leaf_b, double *S,
                      int64_t lds, const BlockDiag *bd) {
    if (d > F_MAXD) return fail(KRR_ERR_NOT_IMPLEMENTED, "sample_f64: d > 64");
    if (ma == 0 || r == 0) return KRR_OK;
    dim3 grid(unsigned(cdiv(ma, F_BM)), unsigned(cdiv(r, F_BC)));
    { sample_f64_kernel<<<grid, 256, 0, c->stream>>>(Xa, ma, Xb, nb, d, 1.0 / (2.0 * h * h), R, r, ldr, leaf_a, leaf_b,
                                                   S, lds, bd ? bd->grp_a : nullptr,
                                                   bd ? bd->grp_b : nullptr, bd ? bd->off_b : nullptr); ::krr::count_launch(); }
    KRR_CUDA(cudaGetLastError());
    return KRR_OK;
}

}  // namespace krr
