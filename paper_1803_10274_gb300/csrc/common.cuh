// Internal helpers shared by the krrhss CUDA sources: error latching, the
// context, device memory, and the counter-based generator.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/krrhss.h"

namespace krr {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file = nullptr, int line = 0);

#define KRR_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return ::krr::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define KRR_TRY(call)                 \
    do {                              \
        int s_ = (call);              \
        if (s_ != KRR_OK) return s_;  \
    } while (0)

// Device status word layout (latched by kernels, read by krr_sync):
// first nonzero error code wins; the second word records where.
struct DevStatus {
    int code;
    int where;
};

// ---------------------------------------------------------------- context
// Default limit of one device-side wait of the pipelined kernels (about two
// seconds of SM clock); krr_set_wait_limit changes it per context.
constexpr long long kDefaultWaitCycles = 4000000000ll;

struct Ctx {
    krr_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    DevStatus *status = nullptr;  // device
    long long wait_cycles = kDefaultWaitCycles;
    bool autotune = false;  // time the fused product's launch variants per shape class
};

// A kernel's dynamic shared-memory limit is an attribute of the device's
// context, so it is raised once per device (and again if a larger size is
// asked for).  Threads may race here; the call is idempotent.
constexpr int kMaxDevices = 64;
struct SmemLimitOnce {
    std::atomic<int> bytes[kMaxDevices];
};
template <class F>
inline cudaError_t raise_smem_limit(SmemLimitOnce &once, int device, F *kernel, int bytes) {
    const bool cached = device >= 0 && device < kMaxDevices;
    if (cached && once.bytes[device].load(std::memory_order_acquire) >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && cached) once.bytes[device].store(bytes, std::memory_order_release);
    return e;
}

void *dalloc(Ctx *c, size_t bytes);
void dfree(Ctx *c, void *p);

// RAII device buffer tied to a context.
template <class T>
struct DBuf {
    Ctx *c = nullptr;
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(Ctx *ctx, size_t count) { reset(ctx, count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : c(o.c), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); c = o.c; p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    bool reset(Ctx *ctx, size_t count) {
        release();
        c = ctx;
        n = count;
        p = count ? static_cast<T *>(dalloc(ctx, count * sizeof(T))) : nullptr;
        return count == 0 || p != nullptr;
    }
    void release() {
        if (p) dfree(c, p);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
};

// Latch an error code from device code (first one wins).
__device__ __forceinline__ void dev_fail(DevStatus *st, int code, int where) {
    if (st && atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Count of kernel launches made by this library (all threads); kernels
// replayed from a captured CUDA graph count once per replay.
void count_launch();
void count_launches(long long k);
long long launches_so_far();
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// --------------------------------------------------- Philox4x64-10 (device)
// Salmon et al., SC'11.  Round multipliers and Weyl key increments are
// the published Philox4x64 constants.
struct U64x4 {
    uint64_t v[4];
};

__host__ __device__ __forceinline__ void mulhilo64(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    lo = (uint64_t)p;
    hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                       uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, hi0, lo0);
        mulhilo64(M1, c2, hi1, lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    U64x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

constexpr uint64_t kStreamR = 0x52;
constexpr uint64_t kStreamCluster = 0x43;

}  // namespace krr

struct krr_ctx {
    krr::Ctx c;
};
