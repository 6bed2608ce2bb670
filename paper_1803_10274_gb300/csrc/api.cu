// C-ABI entry points: context, errors, standardization, the fused
// products and the random block.  The HSS entry points live in hss_api.cu.
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "prep.cuh"

namespace krr {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }
int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}
int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    std::string where;
    if (file) {
        const char *b = std::strrchr(file, '/');
        where = " (" + std::string(b ? b + 1 : file) + ":" + std::to_string(line) + ")";
    }
    set_error(std::string(what) + ": " + cudaGetErrorString(e) + where);
    return e == cudaErrorMemoryAllocation ? KRR_ERR_OOM : KRR_ERR_CUDA;
}

void *dalloc(Ctx *c, size_t bytes) {
    if (bytes == 0) return nullptr;
    bytes = (bytes + 255) & ~size_t(255);
    if (c->has_alloc) return c->alloc.alloc(bytes, c->alloc.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void dfree(Ctx *c, void *p) {
    if (!p) return;
    if (c->has_alloc)
        c->alloc.free(p, c->alloc.user);
    else
        cudaFreeAsync(p, c->stream);
}

int sample_mixed_prepared(Ctx *c, const __half *XA, int64_t ma, const __half *XB, int64_t nb, int d,
                          const __half *RT, int r_total, int64_t ldrt, const int32_t *leaf_a,
                          const int32_t *leaf_b, float *S, int64_t lds, bool split_k, const BlockDiag *bd) {
    if (ma == 0 || r_total == 0) return KRR_OK;
    KRR_CUDA(cudaMemset2DAsync(S, size_t(lds) * 4, 0, size_t(r_total) * 4, size_t(ma), c->stream));
    if (nb == 0) return KRR_OK;
    const int nchunk = aug_chunks(d);
    // resident rows (up to four chunks): launches of up to 256 / 128 / 64
    // columns as tensor memory and shared memory allow; wider rows stream
    // chunk by chunk in launches of up to 128 columns
    const bool wide = nchunk > 4;
    const int rmax = wide ? 128 : nchunk == 1 ? 256 : nchunk <= 3 ? 128 : 64;
    for (int col = 0; col < r_total; col += rmax) {
        const int rv = r_total - col < rmax ? r_total - col : rmax;
        // the product MMA is 32 columns wide for up to 32 columns (the
        // streamed wide-row kernel keeps multiples of 64)
        const int rpad = !wide && rv <= 32 ? 32 : int(round_up(rv, 64));
        if (wide)
            KRR_TRY(launch_sample_tc_wide(c, XA, ma, XB, nb, nchunk, aug_kmma(d), RT + int64_t(col) * ldrt, rpad, ldrt,
                                          rv, leaf_a, leaf_b, S + col, lds, split_k, bd));
        else
            KRR_TRY(launch_sample_tc(c, XA, ma, XB, nb, nchunk, aug_kmma(d), RT + int64_t(col) * ldrt, rpad, ldrt, rv,
                                     leaf_a, leaf_b, S + col, lds, split_k, bd));
    }
    return KRR_OK;
}

}  // namespace krr

using namespace krr;

extern "C" {

const char *krr_last_error(void) { return g_last_error.c_str(); }

long long krr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int krr_create(krr_ctx **out, const krr_allocator *alloc, void *stream) {
    if (!out) return fail(KRR_ERR_INVALID_ARG, "krr_create: out is NULL");
    *out = nullptr;
    krr_ctx *k = new (std::nothrow) krr_ctx();
    if (!k) return fail(KRR_ERR_OOM, "krr_create: host allocation failed");
    Ctx &c = k->c;
    if (alloc && alloc->alloc && alloc->free) {
        c.alloc = *alloc;
        c.has_alloc = true;
    }
    c.stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (e == cudaSuccess) e = cudaMalloc(&c.status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(c.status, 0, sizeof(DevStatus));
    if (e != cudaSuccess) {
        delete k;
        return cuda_fail(e, "krr_create");
    }
    *out = k;
    return KRR_OK;
}

void krr_destroy(krr_ctx *k) {
    if (!k) return;
    cudaStreamSynchronize(k->c.stream);
    if (k->c.status) cudaFree(k->c.status);
    delete k;
}

int krr_set_wait_limit(krr_ctx *k, int64_t cycles) {
    if (!k) return fail(KRR_ERR_INVALID_ARG, "krr_set_wait_limit: ctx is NULL");
    k->c.wait_cycles = cycles > 0 ? (long long)cycles : kDefaultWaitCycles;
    return KRR_OK;
}

int krr_set_autotune(krr_ctx *k, int32_t enable) {
    if (!k || (enable != 0 && enable != 1)) return fail(KRR_ERR_INVALID_ARG, "krr_set_autotune: bad arguments");
    k->c.autotune = enable != 0;
    return KRR_OK;
}

int krr_sync(krr_ctx *k) {
    if (!k) return fail(KRR_ERR_INVALID_ARG, "krr_sync: ctx is NULL");
    KRR_CUDA(cudaStreamSynchronize(k->c.stream));
    DevStatus st{};
    KRR_CUDA(cudaMemcpy(&st, k->c.status, sizeof st, cudaMemcpyDeviceToHost));
    if (st.code != 0) {
        KRR_CUDA(cudaMemset(k->c.status, 0, sizeof(DevStatus)));
        return fail(st.code, "device error latched (site " + std::to_string(st.where) + ")");
    }
    return KRR_OK;
}

int krr_standardize(krr_ctx *k, float *X, int64_t n, int32_t d, float *Xt, int64_t m, double *mean, double *std) {
    if (!k || !X || n <= 0 || d <= 0 || m < 0 || (m > 0 && !Xt))
        return fail(KRR_ERR_INVALID_ARG, "krr_standardize: bad arguments");
    return standardize(&k->c, X, n, d, Xt, m, mean, std);
}

int krr_random_block(krr_ctx *k, int64_t n, int32_t r, int32_t col0, uint64_t seed, int precision, void *out,
                     int64_t ld) {
    if (!k || n < 0 || r < 0 || col0 < 0 || (n > 0 && r > 0 && !out) || ld < r ||
        (precision != KRR_MIXED && precision != KRR_FP64))
        return fail(KRR_ERR_INVALID_ARG, "krr_random_block: bad arguments");
    return random_block(&k->c, n, r, col0, seed, precision, out, ld);
}

int krr_sample(krr_ctx *k, const float *Xa, int64_t ma, const float *Xb, int64_t nb, int32_t d, double h,
               double lambda, const float *R, int32_t r, int64_t ldr, const int32_t *leaf_a, const int32_t *leaf_b,
               float *S, int64_t lds) {
    if (!k || !Xa || !Xb || !R || !S || ma < 0 || nb < 0 || d <= 0 || r <= 0 || ldr < r || lds < r || !(h > 0))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample: bad arguments");
    if ((leaf_a == nullptr) != (leaf_b == nullptr))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample: give both leaf arrays or neither");
    if (lambda != 0.0 && ma != nb) return fail(KRR_ERR_INVALID_ARG, "krr_sample: lambda needs Xa == Xb");
    if (d > kMaxMixedDim) return fail(KRR_ERR_NOT_IMPLEMENTED, "krr_sample: mixed path supports d <= 1024");
    Ctx *c = &k->c;
    const int kpad = aug_kpad(d);
    const int64_t ldrt = round_up(nb > 0 ? nb : 1, 8);
    const int rpad = int(round_up(r, 64));
    DBuf<__half> xa(c, size_t(ma) * kpad), xb(c, size_t(nb) * kpad), rt(c, size_t(rpad) * ldrt);
    if ((ma && !xa.get()) || (nb && !xb.get()) || !rt.get()) return fail(KRR_ERR_OOM, "krr_sample: out of memory");
    KRR_TRY(augment(c, Xa, ma, d, h, 0, xa.get(), kpad));
    KRR_TRY(augment(c, Xb, nb, d, h, 1, xb.get(), kpad));
    KRR_TRY(transpose_half(c, R, nb, r, ldr, rt.get(), rpad, ldrt));
    KRR_TRY(sample_mixed_prepared(c, xa.get(), ma, xb.get(), nb, d, rt.get(), r, ldrt, leaf_a, leaf_b, S, lds));
    KRR_TRY(add_lambda<float>(c, S, lds, R, ldr, ma, r, lambda, true));
    return KRR_OK;
}

int krr_sample_f64(krr_ctx *k, const double *Xa, int64_t ma, const double *Xb, int64_t nb, int32_t d, double h,
                   double lambda, const double *R, int32_t r, int64_t ldr, const int32_t *leaf_a,
                   const int32_t *leaf_b, double *S, int64_t lds) {
    if (!k || !Xa || !Xb || !R || !S || ma < 0 || nb < 0 || d <= 0 || r <= 0 || ldr < r || lds < r || !(h > 0))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample_f64: bad arguments");
    if ((leaf_a == nullptr) != (leaf_b == nullptr))
        return fail(KRR_ERR_INVALID_ARG, "krr_sample_f64: give both leaf arrays or neither");
    if (lambda != 0.0 && ma != nb) return fail(KRR_ERR_INVALID_ARG, "krr_sample_f64: lambda needs Xa == Xb");
    Ctx *c = &k->c;
    KRR_TRY(launch_sample_f64(c, Xa, ma, Xb, nb, d, h, R, r, ldr, leaf_a, leaf_b, S, lds));
    KRR_TRY(add_lambda<double>(c, S, lds, R, ldr, ma, r, lambda, false));
    return KRR_OK;
}

}  // extern "C"
