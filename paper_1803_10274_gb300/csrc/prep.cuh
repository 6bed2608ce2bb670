// Declarations of the data-preparation kernels (prep.cu) and of the
// launchers of the fused products (sample_tc.cu, sample_f64.cu).
#pragma once
#include "common.cuh"

namespace krr {

int standardize(Ctx *c, float *X, int64_t n, int d, float *Xt, int64_t m, double *mean, double *stdv);
template <class Tin, class Tout>
int gather_rows(Ctx *c, const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols, Tout *dst,
                int64_t ldd);
template <class Tin, class Tout>
int scatter_rows(Ctx *c, const Tin *src, int64_t lds, const int32_t *perm, int64_t n, int cols, Tout *dst,
                 int64_t ldd);
int widen(Ctx *c, const float *src, int64_t n, double *dst);
int augment(Ctx *c, const float *X, int64_t rows, int d, double h, int role, __half *out, int kpad);
int transpose_half(Ctx *c, const float *R, int64_t n, int r, int64_t ldr, __half *RT, int rpad, int64_t ldrt);
template <class T>
int add_lambda(Ctx *c, T *S, int64_t lds, const T *R, int64_t ldr, int64_t n, int r, double lambda, bool round16);
int random_block(Ctx *c, int64_t n, int r, int col0, uint64_t seed, int precision, void *out, int64_t ld);

// Augmented-operand geometry of the tensor-core product for feature
// dimension d: 3d + 6 used FP16 elements, padded to 64-element chunks.
inline int aug_used(int d) { return 3 * d + 6; }
inline int aug_kmma(int d) { return int(cdiv(aug_used(d), 16)); }
inline int aug_chunks(int d) { return int(cdiv(aug_used(d), 64)); }
// d <= 8 (3d + 6 <= 32): one 32-element chunk of 64-byte rows (64-byte
// swizzle), half the shared-memory bytes of a 64-element chunk
inline bool aug_narrow(int d) { return aug_used(d) <= 32; }
inline int aug_kpad(int d) { return aug_narrow(d) ? 32 : 64 * aug_chunks(d); }
constexpr int kMaxResidentDim = 82;  // 3d + 6 <= 256: rows resident in shared memory (four chunks)
constexpr int kMaxMixedDim = 1024;   // above kMaxResidentDim the rows stream chunk by chunk

// A block-diagonal product: many independent problems whose rows are
// contiguous ranges of A and of B; a pair (i, j) is kept only when
// grp_a[i] == grp_b[j].  The tensor-core kernel walks only the 128 x 128
// tiles that meet a diagonal block: row tile rt covers column tiles
// [tl_lo[rt], tl_hi[rt]], numbered from tl_off[rt] (tl_off has one entry
// per row tile plus the total).  off_b (nprob + 1 entries) gives the first
// row of each problem in B, for the FP64 kernel.  All device arrays.
constexpr int kTcTile = 128;  // rows and columns of one tile of the tensor-core product

struct BlockDiag {
    const int32_t *grp_a = nullptr, *grp_b = nullptr;
    const int64_t *off_b = nullptr;
    const int32_t *tl_lo = nullptr, *tl_hi = nullptr;
    const int64_t *tl_off = nullptr;
    int64_t tiles = 0;
};

int launch_sample_tc(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int nchunk, int kmma,
                     const __half *RT, int rpad, int64_t ldrt, int r_valid, const int32_t *leaf_a,
                     const int32_t *leaf_b, float *S, int64_t lds, bool split_k = false,
                     const BlockDiag *bd = nullptr);
int launch_sample_tc_wide(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int nchunk, int kmma,
                          const __half *RT, int rpad, int64_t ldrt, int r_valid, const int32_t *leaf_a,
                          const int32_t *leaf_b, float *S, int64_t lds, bool split_k, const BlockDiag *bd);
int launch_sample_f64(Ctx *c, const double *Xa, int64_t ma, const double *Xb, int64_t nb, int d, double h,
                      const double *R, int r, int64_t ldr, const int32_t *leaf_a, const int32_t *leaf_b, double *S,
                      int64_t lds, const BlockDiag *bd = nullptr);

// Mixed-precision product on already-prepared operands: S = W o K R over
// any number of columns (split into launches of <= 256 columns).  S is
// zeroed here.  RT holds r_total rows (ldrt each).  split_k evaluates K
// as an FP16 pair K_hi + K_lo (about 2^-22 relative instead of 2^-11).
int sample_mixed_prepared(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int d,
                          const __half *RT, int r_total, int64_t ldrt, const int32_t *leaf_a,
                          const int32_t *leaf_b, float *S, int64_t lds, bool split_k = false,
                          const BlockDiag *bd = nullptr);

}  // namespace krr
