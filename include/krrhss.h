/*
 * krrhss: Gaussian-kernel ridge regression through a randomized HSS
 * approximation of K + lambda I, on one GB300 GPU (sm_103a).
 *
 * Method (arXiv:1803.10274, "A Study of Clustering Techniques and
 * Hierarchical Matrix Formats for Kernel Ridge Regression"):
 *   Algorithm 1 (Section 2): order the training points (step 0), form the
 *   Gaussian kernel K_ij = exp(-||x_i - x_j||^2 / (2 h^2)) (Eq. (1), step 1),
 *   solve (K + lambda I) w = y (step 2), predict sign(w^T K'(i)) (steps 3-4).
 *   Step 0 is recursive two-means (Sections 4.2-4.3).  Step 2 uses an HSS
 *   approximation (Section 3.1) built by randomized sampling from products
 *   with K and selected entries of K (Section 1.1, "partially matrix-free"),
 *   then a ULV factorization and solve (Section 3.1).
 *
 * Conventions shared by every call:
 *   - Matrices are row-major; "device" pointers are CUDA global memory of
 *     the current device, "host" pointers are ordinary host memory.
 *   - The caller owns every buffer it passes.  Opaque handles (krr_ctx,
 *     krr_hss) are owned by the library and freed by their destroy call.
 *   - All device work is enqueued on the context's stream.  A call returns
 *     after enqueueing unless its description says it synchronizes.
 *   - Return value: KRR_OK or a krr_status error code; krr_last_error()
 *     gives a message for the calling thread.  No C++ exception crosses
 *     this interface.
 *   - Device-side failures (a wait that ran past its limit, a zero pivot)
 *     are latched in the context and reported by the next synchronizing
 *     call.
 */
#ifndef KRRHSS_H
#define KRRHSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KRR_OK = 0,
    KRR_ERR_INVALID_ARG = 1,     /* bad size, pointer, option or layout   */
    KRR_ERR_NONFINITE_INPUT = 2, /* NaN or Inf in X                       */
    KRR_ERR_OOM = 3,             /* device allocation failed              */
    KRR_ERR_SINGULAR = 4,        /* zero pivot in a ULV block factorization */
    KRR_ERR_RANK_BUDGET = 5,     /* ranks not revealed within r_max samples */
    KRR_ERR_TIMEOUT = 6,         /* a device wait ran past its limit       */
    KRR_ERR_CUDA = 7,            /* CUDA runtime/driver error              */
    KRR_ERR_NOT_IMPLEMENTED = 8,
    KRR_ERR_NO_CONVERGENCE = 9   /* refinement did not reach the tolerance */
} krr_status;

/* Arithmetic of the compression / factor / solve path. */
typedef enum {
    KRR_MIXED = 0, /* kernel products on tcgen05 tensor cores: FP16 operands
                      (split into hi/lo parts for the distances), FP32
                      accumulation; other steps in FP32                     */
    KRR_FP64 = 1,  /* every step in FP64 on the CUDA cores                  */
    KRR_MIXED_F64 = 2 /* kernel products on tensor cores as KRR_MIXED; the
                      interpolative decompositions, the factorization and
                      the ULV solve in FP64 (for smooth kernels, whose
                      blocks are large next to lambda)                     */
} krr_precision;

/* Optional device-memory allocator (e.g. a framework's caching allocator).
 * alloc(bytes, user) returns device memory aligned to 256 bytes or NULL;
 * free(ptr, user) releases it.  Both are called on the context's stream
 * order.  Pass NULL to krr_create to use cudaMallocAsync/cudaFreeAsync. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} krr_allocator;

typedef struct krr_ctx krr_ctx;
typedef struct krr_hss krr_hss;

/* Create a context on the current CUDA device.  stream: a cudaStream_t
 * (NULL = the legacy default stream).  The allocator struct is copied. */
int krr_create(krr_ctx **ctx, const krr_allocator *alloc, void *stream);
void krr_destroy(krr_ctx *ctx);

/* Message for the last failing call on this thread ("" if none). */
const char *krr_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (a diagnostic for profiling and benchmarks). */
long long krr_launch_count(void);

/* Measured throughput of one arithmetic pipe of the context's GPU (a
 * diagnostic: the denominators of the fused product's secondary bounds and
 * of the FP64 comparator).  which: 0 = FP32 FMA (flop/s, 2 per FMA),
 * 1 = FP64 FMA (flop/s), 2 = ex2.approx.ftz.f32 on the SFU (results/s),
 * 3 = cvt.rn.f16x2.f32 (converted values/s, 2 per instruction).  Runs
 * independent chains in a full grid, best of three timed launches after a
 * warm-up.  Synchronizes. */
int krr_probe_rate(krr_ctx *ctx, int32_t which, double *ops_per_second);

/* Batched FP32 products C_b = alpha op(A_b) op(B_b) + beta C_b, b < batch,
 * through the library's grouped product (the interpolative decompositions'
 * and the factorization's node products use the same code).  A_b = A + b sA
 * is M x K (ta = 0: row-major, element (i, k) at A_b[i lda + k]) or stored
 * K x M (ta = 1: element (i, k) at A_b[k lda + i]); B_b = B + b sB is K x N
 * (tb = 0: B_b[k ldb + j]) or stored N x K (tb = 1: B_b[j ldb + k]);
 * C_b = C + b sC is M x N row-major (C_b[i ldc + j]).  All device float
 * pointers; C must not overlap A or B.  path: 0 = the library's choice,
 * 1 = tensor cores (tcgen05 kind::tf32, each operand split into two TF32
 * parts, three products: about FP32 accuracy), 2 = CUDA cores (FP32 FMA).
 * Asynchronous on the context's stream. */
int krr_gemm_f32_batched(krr_ctx *ctx, int32_t batch, int32_t M, int32_t N,
                         int32_t K, float alpha, const float *A, int64_t lda,
                         int64_t sA, int32_t ta, const float *B, int64_t ldb,
                         int64_t sB, int32_t tb, float beta, float *C,
                         int64_t ldc, int64_t sC, int32_t path);

/* Wait for the context's stream and return (and clear) any latched device
 * error.  Synchronizes. */
int krr_sync(krr_ctx *ctx);

/* Autotuning of the fused product's launch variant (enable = 1; 0, the
 * default, uses fixed rules).  The variants: pairs of row tiles in
 * clusters of two CTAs sharing every column tile's loads, or one row tile
 * per CTA; one or two threads issuing the tensor-core MMAs.  With the
 * autotuner on, the first launch of a shape class (device, feature
 * chunks, column width, split K, leaf masks, log2 of the tile count) on any
 * context times every allowed variant on that call (synchronizing) and
 * caches the fastest for the process; later launches of the class use it.
 * Skipped while the context's stream is being captured.  The results of
 * the variants differ only in the order of floating-point additions. */
int krr_set_autotune(krr_ctx *ctx, int32_t enable);

/* Limit, in SM clock cycles, of each hand-off wait inside the pipelined
 * tensor-core kernels (the fused products) that this context launches from
 * now on; cycles <= 0 restores the default (4e9 cycles, about two seconds).
 * When a wait runs past the limit the kernel stops its pipeline, lets the
 * copies and tensor-core operations it already issued finish, frees its
 * tensor memory and returns; the context latches KRR_ERR_TIMEOUT, which the
 * next synchronizing call (krr_sync, a compression, a solve) returns and
 * clears.  The outputs of that launch are then undefined; the context stays
 * usable.  Failure detection (the paper has no counterpart): a stalled
 * pipeline ends with an error status instead of a hung GPU. */
int krr_set_wait_limit(krr_ctx *ctx, int64_t cycles);

/* ---------------------------------------------------------------------
 * Feature standardization (Section 5.2: zero mean, unit standard
 * deviation per column; test data use the training statistics; a column
 * with zero spread is divided by 1).
 *   X   device float, n x d, standardized in place (training set)
 *   Xt  device float, m x d, in place with X's statistics (may be NULL, m=0)
 *   mean, std  device double[d] outputs (may be NULL)
 * Statistics are accumulated in FP64.
 * ------------------------------------------------------------------- */
int krr_standardize(krr_ctx *ctx, float *X, int64_t n, int32_t d, float *Xt,
                    int64_t m, double *mean, double *std);

/* ---------------------------------------------------------------------
 * Recursive two-means ordering (Algorithm 1 step 0; Sections 4.2-4.3).
 *   X      device float, n x d, read only
 *   leaf   split while a node holds more than `leaf` rows (>= 1)
 *   seed   seeds the counter-based draws of the first and second
 *          representatives (Philox4x64-10, counter (begin, size, 0, 0))
 *   perm   device int32[n] output: perm[new] = old row
 *   tree   host int32 arrays of capacity max_nodes (>= 2*ceil(n/1)-1 is
 *          always enough; 2*n is safe): node begin/end (row range in the
 *          new order), left/right child (-1 at a leaf), parent (-1 at the
 *          root), level (root 0).  Nodes are numbered in postorder
 *          (Figure 2), so the root is node n_nodes-1.
 *   n_nodes host output
 * Arithmetic is exact (quantized 64-bit integer coordinates), so the
 * result does not depend on thread scheduling.  Synchronizes.
 * ------------------------------------------------------------------- */
typedef struct {
    int32_t *begin, *end, *left, *right, *parent, *level;
} krr_tree_arrays;

int krr_cluster(krr_ctx *ctx, const float *X, int64_t n, int32_t d,
                int32_t leaf, uint64_t seed, int32_t *perm,
                int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes);

/* The orderings Section 4.3 compares (same outputs and conventions as
 * krr_cluster, which is ordering KRR_ORDER_TWO_MEANS):
 *   KRR_ORDER_NATURAL  no preprocessing (NP): the input order, every node
 *                      split into halves (first floor(m/2) rows first);
 *   KRR_ORDER_KD       k-d tree: split along the coordinate of maximum
 *                      spread (max - min of the quantized coordinates,
 *                      lowest coordinate on ties) at its mean (a row goes
 *                      first iff its value <= the mean, exact in integers);
 *                      when 100 x the smaller side < the larger side, at
 *                      the median (the floor(m/2) smallest values first,
 *                      ties in row order);
 *   KRR_ORDER_PCA      principal direction: split at the mean of the
 *                      projections onto the node's first principal
 *                      direction (covariance from exact integer sums, 64
 *                      power iterations from e_0, fixed round-to-nearest FP64
 *                      operation order, largest entry made positive; a row
 *                      goes first iff its projection <= 0); d <= 64.
 * A split that leaves one side empty becomes halves; seed is used by
 * two-means only.  Synchronizes. */
#define KRR_ORDER_TWO_MEANS 0
#define KRR_ORDER_NATURAL 1
#define KRR_ORDER_KD 2
#define KRR_ORDER_PCA 3
int krr_order(krr_ctx *ctx, const float *X, int64_t n, int32_t d, int32_t leaf,
              int32_t ordering, uint64_t seed, int32_t *perm,
              int32_t max_nodes, krr_tree_arrays tree, int32_t *n_nodes);

/* Batched form: the rows of X split into nprob contiguous problems
 * (offsets: host int64[nprob + 1], offsets[0] = 0, offsets[nprob] = n, every
 * problem non-empty).  The top of the tree is a balanced binary tree over
 * the problems; below, every problem is ordered exactly as krr_cluster
 * orders it alone (quantization and seed counters are per problem), and
 * perm keeps every row inside its problem.  One set of launches serves all
 * problems.  Synchronizes. */
int krr_cluster_batched(krr_ctx *ctx, const float *X, int64_t n, int32_t d,
                        int32_t nprob, const int64_t *offsets, int32_t leaf,
                        uint64_t seed, int32_t *perm, int32_t max_nodes,
                        krr_tree_arrays tree, int32_t *n_nodes);

/* ---------------------------------------------------------------------
 * Fused kernel-times-block product (the HSS sampling step, Section 1.1
 * and Section 3.1: the randomized construction needs A R for a block R of
 * random vectors; Section 5.6 shows it dominates construction time):
 *     S(i, :) = sum_j w_ij K(xa_i, xb_j) R(j, :)  + lambda * R(i, :)
 * without storing K.  w_ij = 0 when leaf_a and leaf_b are both given and
 * leaf_a[i] == leaf_b[j] (the product restricted to the off-diagonal leaf
 * blocks, which is what the compression samples), else 1.  lambda must be
 * 0 unless Xa and Xb are the same rows (ma == nb).
 *   Xa device float ma x d;  Xb device float nb x d
 *   R  device float nb x r (row stride ldr >= r)
 *   S  device float ma x r output (row stride lds >= r), overwritten
 *   leaf_a, leaf_b  device int32[ma], int32[nb] or both NULL
 * KRR_MIXED: R is rounded to FP16; distances use an FP16 hi/lo split with
 * FP32 accumulation on tcgen05 tensor cores, exp2 on the SFU, K rounded to
 * FP16, K R accumulated in FP32 in tensor memory.  Requires d <= 1024
 * (rows longer than four 64-element chunks, d > 82, stream through shared
 * memory chunk by chunk instead of staying resident),
 * 1 <= r and max |x|^2 / h^2 small enough for FP16 (else INVALID_ARG).
 * ------------------------------------------------------------------- */
int krr_sample(krr_ctx *ctx, const float *Xa, int64_t ma, const float *Xb,
               int64_t nb, int32_t d, double h, double lambda, const float *R,
               int32_t r, int64_t ldr, const int32_t *leaf_a,
               const int32_t *leaf_b, float *S, int64_t lds);

/* krr_sample without device-memory allocation, for callers that cannot
 * allocate at the point of the call: a process that runs under a fixed
 * device-memory budget, one that has no allocator to hand to the library,
 * or a latency-critical loop that must not enter an allocator.  The paper
 * has no counterpart: this is an interface convenience.
 * Same arguments, result and precision as krr_sample (KRR_MIXED).  Its
 * scratch lives in one fixed device array inside the library (about
 * 12.6 MB, reserved on every GPU that loads the library until the process
 * exits), so sizes are limited to max(ma, nb) <= 16384, r <= 256 and
 * d <= 19; larger sizes return KRR_ERR_INVALID_ARG.  The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture.  Every call reuses the same array: calls that may
 * overlap on the GPU (other streams or unordered threads) race on it. */
int krr_sample_noalloc(krr_ctx *ctx, const float *Xa, int64_t ma,
                       const float *Xb, int64_t nb, int32_t d, double h,
                       double lambda, const float *R, int32_t r, int64_t ldr,
                       const int32_t *leaf_a, const int32_t *leaf_b, float *S,
                       int64_t lds);

/* Same product in FP64 on the CUDA cores (the "plain" comparator):
 * Xa, Xb device double; R, S device double.  No size limit on d. */
int krr_sample_f64(krr_ctx *ctx, const double *Xa, int64_t ma,
                   const double *Xb, int64_t nb, int32_t d, double h,
                   double lambda, const double *R, int32_t r, int64_t ldr,
                   const int32_t *leaf_a, const int32_t *leaf_b, double *S,
                   int64_t lds);

/* Columns [col0, col0 + r) of the method's random block, N(0,1) by
 * Philox4x64-10 (key (seed, 0x52), counter (row, col/4, 0, 0)) and
 * Box-Muller, as FP32 (KRR_MIXED: rounded to FP16 and widened back, so
 * the tensor-core path uses it exactly) or FP64.  out: device, n x r with
 * row stride ld.  col0 must be a multiple of 4. */
int krr_random_block(krr_ctx *ctx, int64_t n, int32_t r, int32_t col0,
                     uint64_t seed, int precision, void *out, int64_t ld);

/* ---------------------------------------------------------------------
 * HSS compression / factorization / solve / prediction.
 * ------------------------------------------------------------------- */
typedef struct {
    double h;          /* Gaussian width (Eq. (1))                          */
    double lambda;     /* ridge parameter (> 0)                             */
    double eps_c;      /* relative tolerance of the interpolative
                          decompositions: a pivot is kept while
                          |R_jj| > eps_c |R_11|                             */
    double eps_abs;    /* absolute pivot floor (0 = none)                   */
    int32_t leaf;      /* leaf size of the two-means tree                   */
    int32_t r0;        /* initial number of random columns (multiple of 16) */
    int32_t p;         /* oversampling: ranks must stay <= r - p            */
    int32_t r_max;     /* cap on random columns                             */
    uint64_t seed;     /* seeds clustering and the random block             */
    int32_t precision; /* krr_precision                                     */
    int32_t flags;     /* KRR_TRUNCATE_AT_RMAX | KRR_LAMBDA_TOL, or 0       */
    int32_t ordering;  /* KRR_ORDER_* (default two-means, Section 4.3)      */
    int32_t pad;
} krr_options;

/* krr_options.flags: when the ranks are not revealed within r_max samples,
 * keep every decomposition truncated at the budget (rank r_max - 16 - p + 1
 * at most; a coarser approximation, still a usable preconditioner for the
 * refined solve) instead of failing with KRR_ERR_RANK_BUDGET. */
#define KRR_TRUNCATE_AT_RMAX 1
/* krr_options.flags: measure the decompositions' accuracy against lambda as
 * well: a decomposition stops only when its next pivot is below
 * eps_c * min(|R_11|, lambda sqrt(s)), s the sample columns it uses (a pivot
 * is about sigma sqrt(s) for a singular value sigma of the block).  For
 * smooth kernels, whose blocks are large next to lambda, this keeps the
 * approximation error of K + lambda I below about eps_c lambda per block, so
 * the factorization stays a good preconditioner. */
#define KRR_LAMBDA_TOL 2

/* Fill opts with defaults: eps_c 0.03, eps_abs 0, leaf 128, r0 64, p 10,
 * r_max 2048, seed 1, KRR_MIXED, flags 0, two-means ordering; h and lambda
 * set to 1. */
void krr_default_options(krr_options *opts);

/* Cluster X (device float n x d, original order, already standardized if
 * wanted) and build the HSS approximation of K + lambda I in that order.
 * Synchronizes (the adaptive sampling reads ranks back per level). */
int hss_compress(krr_ctx *ctx, const float *X, int64_t n, int32_t d,
                 const krr_options *opts, krr_hss **out);

/* Many independent problems in one handle (batching): problem p owns rows
 * [offsets[p], offsets[p+1]) of X (host int64[nprob + 1], offsets[0] = 0,
 * offsets[nprob] = n, every problem non-empty) and has the Gaussian width
 * h[p] (host double[nprob]); opts->h is ignored, lambda and the other
 * options are shared.  The handle holds the block-diagonal matrix
 * diag(K_p + lambda I): one tree over all problems (krr_cluster_batched),
 * every fused product one persistent launch over the tiles of the
 * diagonal blocks only, every level of the compression, factorization and
 * solve one set of launches over the nodes of all problems.  Problems that
 * share their points but differ in h are passed as separate problems.
 * hss_factor, hss_solve (alpha in original row order, i.e. problem by
 * problem; the tolerance applies to each right-hand side over the whole
 * batch), hss_stats and hss_destroy work as for one problem; predict
 * with krr_predict_batched.  Synchronizes. */
int hss_compress_batched(krr_ctx *ctx, const float *X, int64_t n, int32_t d,
                         int32_t nprob, const int64_t *offsets,
                         const double *h, const krr_options *opts,
                         krr_hss **out);

/* Decision values of a batched handle: test rows [test_offsets[p],
 * test_offsets[p+1]) of Xt (device float m x d) against problem p's
 * training points and weights only (test_offsets: host int64[nprob + 1],
 * nondecreasing, from 0 to m; a problem may have no test rows). */
int krr_predict_batched(krr_hss *H, const float *Xt, int64_t m,
                        const int64_t *test_offsets, const double *alpha,
                        int32_t nrhs, int64_t lda, double *out, int64_t ldo);

/* Change lambda without recompressing (Section 5.3: only the diagonal
 * changes).  Invalidates the factorization; call hss_factor again. */
int hss_update_lambda(krr_hss *H, double lambda);

/* ULV factorization of the HSS matrix (Section 3.1), level by level. */
int hss_factor(krr_hss *H);

/* Solve (K + lambda I) alpha = y.
 *   y      device double, n x nrhs (row stride ldy), original row order
 *   alpha  device double, n x nrhs (row stride lda), original row order
 *   tol    stop refinement when max_c ||(K+lambda I) a_c - y_c|| / ||y_c||
 *          <= tol (the residual uses the fused product, exact up to the
 *          precision mode); tol <= 0: one ULV solve, no refinement
 *   max_refine  cap on refinement steps
 *   resid  host double[1] out (may be NULL): final relative residual
 *          (max over columns), or -1 when no refinement ran
 * Each refinement step is one fused product with the current iterate and
 * one ULV solve (the HSS factor as a preconditioner).  Synchronizes when
 * tol > 0. */
int hss_solve(krr_hss *H, const double *y, int32_t nrhs, int64_t ldy,
              double *alpha, int64_t lda, double tol, int32_t max_refine,
              double *resid);

/* y = H x for the HSS matrix H that the compression built (Section 3.1:
 * leaf blocks D = K(I, I) + lambda I, nested interpolative bases U and
 * sibling blocks B = K(J_a, J_b)), applied from those generators in FP64.
 *   x, y   device double, n x nrhs (row strides ldx, ldy >= nrhs), original
 *          row order; 1 <= nrhs <= 64
 * The ULV factorization eliminates exactly this matrix, so hss_solve with
 * tol <= 0 applied to H x returns x up to rounding, and
 * (H - (K + lambda I)) x measures the compression error.  Works before or
 * after hss_factor.  Single-problem handles only (batched handles return
 * KRR_ERR_NOT_IMPLEMENTED).  Synchronizes. */
int hss_matvec(krr_hss *H, const double *x, int32_t nrhs, int64_t ldx,
               double *y, int64_t ldy);

/* Decision values out = K(Xt, X) alpha (Algorithm 1 steps 3-4; the label
 * is sign(out) with sign(0) = +1).  Xt device float m x d (standardized
 * like X), alpha device double n x nrhs (original order), out device
 * double m x nrhs. */
int krr_predict(krr_hss *H, const float *Xt, int64_t m, const double *alpha,
                int32_t nrhs, int64_t lda, double *out, int64_t ldo);

/* ---------------------------------------------------------------------
 * Multi-class prediction by one-vs-all (Section 2, after Algorithm 1): one
 * binary classifier per class, all c solved as right-hand sides of one
 * hss_solve, and the class of a test point is the argmax of its c
 * confidences.  The paper prints the confidence as |w(c)^T K'(i)|; read
 * literally, a point far on the "not c" side would count as confident in
 * c, so the default takes the signed value w(c)^T K'(i) (absolute = 0) and
 * absolute = 1 gives the printed form.
 * ------------------------------------------------------------------- */
/* Right-hand sides of the c binary problems: Y(i, k) = +1 if cls[i] == k,
 * else -1 (a class outside [0, c) gives -1 in every column).
 *   cls  device int32[n];  Y  device double n x c (row stride ldy >= c)
 * c >= 2. */
int krr_one_vs_all(krr_ctx *ctx, const int32_t *cls, int64_t n, int32_t c,
                   double *Y, int64_t ldy);

/* Decision values dec = K(Xt, X) alpha (m x c, as krr_predict) and
 * labels[i] = argmax_k score(i, k), the lowest k on ties, with score the
 * decision value (absolute = 0) or its magnitude (absolute = 1).
 *   alpha   device double n x c (row stride lda), 2 <= c <= 64
 *   dec     device double m x c (row stride ldd >= c) output, or NULL
 *   labels  device int32[m] output */
int krr_predict_classes(krr_hss *H, const float *Xt, int64_t m,
                        const double *alpha, int32_t c, int64_t lda,
                        int32_t absolute, double *dec, int64_t ldd,
                        int32_t *labels);

/* ---------------------------------------------------------------------
 * Held-out squared-error loss and its gradient in h, lambda and the
 * training points: the quantities Section 5.3 tunes (h and lambda of
 * Eq. (1) and Algorithm 1, chosen on held-out data) made differentiable.
 * With alpha = (K + lambda I)^{-1} y (solved through H as hss_solve with
 * tol) and g = K(Xt, X) alpha - yt:
 *     L = 1/2 sum_k g_k^2.
 * With a = K(Xt, X)^T g and z = (K + lambda I)^{-1} a (a second solve; K
 * is symmetric), the adjoint gives
 *     dL/dlambda = -z . alpha
 *     dL/dh      = h^-3 [ g^T (Kt o Dt) alpha - z^T (K o D) alpha ]
 *     dL/dx_p    = h^-2 [ alpha_p sum_k g_k Kt_kp (xt_k - x_p)
 *                  - sum_j (z_p alpha_j + z_j alpha_p) K_pj (x_j - x_p) ]
 * where D and Dt hold squared distances.  Each sum over kernel entries is
 * one fused product (the kernel recomputed, never stored) against the
 * augmented columns [v, v |x|^2, v x] of the expansion
 * |u - v|^2 = |u|^2 - 2 u.v + |v|^2, on coordinates centred on the training
 * mean.  The arithmetic follows H's precision (KRR_MIXED: tensor-core
 * products with FP16 hi/lo splits of the kernel and of the columns, FP64
 * accumulation of the sums; KRR_FP64: FP64 throughout).
 *   H        compressed at X, h, lambda (hss_compress; lambda as last set by
 *            hss_update_lambda); factored here if needed
 *   Xt       device float m x d held-out points (scaled like X), m >= 1
 *   y        device double[n] training targets, original row order
 *   yt       device double[m] held-out targets
 *   tol, max_refine  as hss_solve, for each of the two solves
 *   loss     host double[1] out
 *   dh, dlambda  host double[1] outs, or NULL
 *   dX       device double n x d out (row stride lddx >= d), original row
 *            order, or NULL
 *   alpha    device double[n] out (original order), or NULL
 *   resid    host double[1] out (may be NULL): the larger final residual
 *            of the two solves
 * With dh, dlambda and dX all NULL only the first solve and the held-out
 * product run.  Returns KRR_ERR_NO_CONVERGENCE (outputs still written)
 * when a solve stops above tol.  Synchronizes. */
int krr_heldout_grad(krr_hss *H, const float *Xt, int64_t m, const double *y,
                     const double *yt, double tol, int32_t max_refine,
                     double *loss, double *dh, double *dlambda, double *dX,
                     int64_t lddx, double *alpha, double *resid);

/* Block partition of an H matrix over a cluster tree (Section 3.2, the H
 * matrix representation: only well-separated sub-blocks are compressed,
 * strong admissibility).  Host only: needs no context and no GPU.
 *   n_nodes, left, right  the tree in postorder (host int32[n_nodes]; the
 *          root is n_nodes - 1; left[v] = right[v] = -1 for a leaf, else
 *          both children have ids below v)
 *   d, lo, hi  host double n_nodes x d (row-major): each node's bounding box
 *   eta    admissibility parameter >= 0: (t, s) is admissible when the
 *          boxes are apart and min(diam t, diam s) <= eta dist(t, s), with
 *          diam the box diagonal and dist the distance between the boxes
 *          (sums of squares in coordinate order, one square root)
 *   near, far  host int32[2 cap_near], int32[2 cap_far]: node pairs (t, s)
 *          of the dense and of the admissible blocks, in depth-first order
 *          from (root, root), left child first (a pair that is neither is
 *          split into its children's pairs: both nodes when both have
 *          children, else the inner one)
 *   n_near, n_far  out: numbers of pairs
 * Returns KRR_ERR_INVALID_ARG for a bad tree or arguments, and when a list
 * is longer than its capacity (counts still returned; nothing written past
 * a capacity). */
int krr_h_partition(int32_t n_nodes, const int32_t *left, const int32_t *right,
                    int32_t d, const double *lo, const double *hi, double eta,
                    int32_t *near, int64_t cap_near, int64_t *n_near,
                    int32_t *far, int64_t cap_far, int64_t *n_far);

typedef struct {
    int64_t n;
    int32_t n_nodes, n_levels, max_rank, samples, rounds, refine_steps;
    int64_t memory_bytes; /* D, U and B generators (Section 4.2 metric) */
    double t_cluster_ms, t_sample_ms, t_compress_ms, t_factor_ms, t_solve_ms;
    int32_t truncated;    /* 1: ranks kept at the r_max budget
                             (KRR_TRUNCATE_AT_RMAX)                      */
    int32_t pad;
} krr_hss_stats;

int hss_stats(const krr_hss *H, krr_hss_stats *st);

/* Row order of the compressed matrix: perm[new] = old (device int32[n]). */
const int32_t *hss_permutation(const krr_hss *H);

void hss_destroy(krr_hss *H);

#ifdef __cplusplus
}
#endif
#endif /* KRRHSS_H */
