/*
 * Oracle: plain FP64 evaluation of the Gaussian kernel (Eq. (1) of the
 * paper, Section 1; the same formula is Step 1 of Algorithm 1) and of
 * products with it.  TEST INFRASTRUCTURE ONLY: the CUDA path never links
 * or calls this file.
 *
 * Every entry is evaluated in the difference form
 *     K(a, b) = exp( -sum_k (a_k - b_k)^2 / (2 h^2) ),
 * with the sum taken sequentially over k, so K(a, b) == K(b, a) bit for
 * bit and K(a, a) == 1 exactly.  Loops over output rows are split across
 * OpenMP threads; each output entry is summed sequentially over j, so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

static double kval(const double *a, const double *b, int d, double inv2h2) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        s += t * t;
    }
    return exp(-s * inv2h2);
}

/* K(Xa, Xb): ma x nb, row-major into K. */
void okrr_kernel_matrix(const double *Xa, int64_t ma, const double *Xb,
                        int64_t nb, int d, double h, double *K) {
    const double inv2h2 = 1.0 / (2.0 * h * h);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ma; ++i)
        for (int64_t j = 0; j < nb; ++j)
            K[i * nb + j] = kval(Xa + i * d, Xb + j * d, d, inv2h2);
}

/* Squared distances D(i, j) = sum_k (Xa_ik - Xb_jk)^2 (the exponent of
 * Eq. (1) times -2 h^2), ma x nb row-major, difference form. */
void okrr_sqdist_matrix(const double *Xa, int64_t ma, const double *Xb,
                        int64_t nb, int d, double *D) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ma; ++i)
        for (int64_t j = 0; j < nb; ++j) {
            const double *a = Xa + i * d, *b = Xb + j * d;
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
                double t = a[k] - b[k];
                s += t * t;
            }
            D[i * nb + j] = s;
        }
}

/*
 * S(i, :) = sum_j w_ij K(Xa_i, Xb_j) R(j, :) for the rows listed in rows[]
 * (rows == NULL means all ma rows, in order).  w_ij = 0 when both leaf
 * arrays are given and leaf_a[i] == leaf_b[j] (the product restricted to
 * the off-diagonal leaf blocks), else 1.  If Sabs != NULL it receives the
 * same product with |R| in place of R, which bounds the rounding error of
 * any evaluation that perturbs each K entry by a relative amount.
 * R is nb x r row-major; S and Sabs are nrows x r row-major.
 */
void okrr_kernel_product(const double *Xa, int64_t ma, const double *Xb,
                         int64_t nb, int d, double h, const double *R, int r,
                         const int32_t *leaf_a, const int32_t *leaf_b,
                         const int64_t *rows, int64_t nrows, double *S,
                         double *Sabs) {
    const double inv2h2 = 1.0 / (2.0 * h * h);
    if (rows == NULL) nrows = ma;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t i = rows ? rows[t] : t;
        double *s = S + t * r;
        double *sa = Sabs ? Sabs + t * r : NULL;
        for (int c = 0; c < r; ++c) {
            s[c] = 0.0;
            if (sa) sa[c] = 0.0;
        }
        for (int64_t j = 0; j < nb; ++j) {
            if (leaf_a && leaf_b && leaf_a[i] == leaf_b[j]) continue;
            const double kij = kval(Xa + i * d, Xb + j * d, d, inv2h2);
            const double *rj = R + j * r;
            for (int c = 0; c < r; ++c) s[c] += kij * rj[c];
            if (sa)
                for (int c = 0; c < r; ++c) sa[c] += kij * fabs(rj[c]);
        }
    }
}

int okrr_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
