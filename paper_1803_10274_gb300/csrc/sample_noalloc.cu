// krr_sample_noalloc: the fused kernel-times-block product without any
// device-memory allocation.
//
// krr_sample stages three scratch operands (the augmented FP16 rows of Xa
// and Xb and the FP16 transpose of R) in memory it allocates per call.
// Some callers cannot allocate device memory at that point: code running
// under a fixed device-memory budget, code without access to an allocator
// it could hand to the library, or latency-critical loops that must not
// enter an allocator.  This
// variant keeps the scratch in one file-scope device array of fixed size
// instead, so a call only launches kernels and clears S.
//
// Limits: max(ma, nb) <= 16384 rows, r <= 256 columns, d <= 19 features
// (one 64-element augmented chunk); larger problems are rejected with
// KRR_ERR_INVALID_ARG.  The array (about 12.6 MB) is reserved on every GPU
// that loads the library, until the process exits.  All calls share it
// and it keeps the previous call's contents, so two calls that overlap on
// the GPU (different streams, or different threads without ordering) race
// on it; calls on one stream are ordered and safe.
#include <mutex>

#include "common.cuh"
#include "prep.cuh"

namespace krr {
namespace {

constexpr int64_t kNoAllocMaxRows = 16384;
constexpr int kNoAllocMaxCols = 256;
constexpr int kNoAllocKpad = 64;
constexpr int kNoAllocMaxDim = 19;  // 3 * 19 + 6 = 63 augmented elements: one chunk
constexpr size_t kXaOff = 0;
constexpr size_t kXbOff = size_t(kNoAllocMaxRows) * kNoAllocKpad;
constexpr size_t kRtOff = 2 * size_t(kNoAllocMaxRows) * kNoAllocKpad;
constexpr size_t kScratchHalves = kRtOff + size_t(kNoAllocMaxCols) * kNoAllocMaxRows;

__device__ __align__(256) __half g_noalloc_scratch[kScratchHalves];

// Device address of the scratch array, looked up once per device with
// that device current.  In host code the array's name is only a stand-in
// symbol, never a usable device pointer.
int scratch_address(__half **out) {
    static std::mutex mu;
    static void *addr[256] = {};
    int dev = 0;
    KRR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(KRR_ERR_CUDA, "krr_sample_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        addr[dev] = p;
    }
    *out = static_cast<__half *>(addr[dev]);
    return KRR_OK;
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" int krr_sample_noalloc(krr_ctx *k, const float *Xa, int64_t ma, const float *Xb, int64_t nb, int32_t d,
                                  double h, double lambda, const float *R, int32_t r, int64_t ldr,
                                  const int32_t *leaf_a, const int32_t *leaf_b, float *S, int64_t lds) {
    if (!k || !Xa || !Xb || !R || !S || ma < 0 || nb < 0 || d <= 0 || r <= 0 || ldr < r || lds < r || !(h > 0))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample_noalloc: bad arguments");
    if ((leaf_a == nullptr) != (leaf_b == nullptr))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample_noalloc: give both leaf arrays or neither");
    if (lambda != 0.0 && ma != nb) return fail(KRR_ERR_INVALID_ARG, "krr_sample_noalloc: lambda needs Xa == Xb");
    // d is tested before aug_kpad(d) (3d + 6 must not overflow): 3d + 6 <= 64
    if (ma > kNoAllocMaxRows || nb > kNoAllocMaxRows || r > kNoAllocMaxCols || d > kNoAllocMaxDim ||
        aug_kpad(d) > kNoAllocKpad)
        return fail(KRR_ERR_INVALID_ARG,
                    "krr_sample_noalloc: size beyond the fixed scratch (rows <= 16384, r <= 256, d <= 19)");
    Ctx *c = &k->c;
    __half *scratch = nullptr;
    KRR_TRY(scratch_address(&scratch));
    const int kpad = aug_kpad(d);
    const int64_t ldrt = round_up(nb > 0 ? nb : 1, 8);
    const int rpad = int(round_up(r, 64));
    __half *xa = scratch + kXaOff, *xb = scratch + kXbOff, *rt = scratch + kRtOff;
    KRR_TRY(augment(c, Xa, ma, d, h, 0, xa, kpad));
    KRR_TRY(augment(c, Xb, nb, d, h, 1, xb, kpad));
    KRR_TRY(transpose_half(c, R, nb, r, ldr, rt, rpad, ldrt));
    KRR_TRY(sample_mixed_prepared(c, xa, ma, xb, nb, d, rt, r, ldrt, leaf_a, leaf_b, S, lds));
    KRR_TRY(add_lambda<float>(c, S, lds, R, ldr, ma, r, lambda, true));
    return KRR_OK;
}
