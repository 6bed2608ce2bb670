// Throughput probes of the GPU's arithmetic pipes, the denominators of the
// fused product's secondary bounds: FP32 FMA, FP64 FMA, the SFU's ex2 and
// the FP32 -> FP16x2 conversion the epilogue rounds K with.  Each probe runs
// independent dependency chains in every thread of a full grid (8 warps per
// SM scheduler) so the pipe, not latency, sets the time; the rate is the
// number of per-lane operations divided by the CUDA-event time.
#include "common.cuh"

namespace krr {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_fma32(int iters, float seed, float *sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + float(threadIdx.x + c);
    const float m = 0.999f, b = 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_fma64(int iters, double seed, double *sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + double(threadIdx.x + c);
    const double m = 0.999, b = 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[c]) : "d"(m), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[0] = s;
}

// x <- 2^x stays in [0, 2] for a start in [-1, 1]: no overflow or NaN.
__global__ void __launch_bounds__(kProbeThreads) probe_ex2(int iters, float seed, float *sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed - 0.01f * float((threadIdx.x + c) & 63);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678f) sink[0] = s;
}

// One cvt.rn.f16x2.f32 per step and chain, each feeding an XOR into the
// chain's accumulator (an integer op of a faster pipe).
__global__ void __launch_bounds__(kProbeThreads) probe_cvt(int iters, float seed, float *sink) {
    float x[kChains];
    uint32_t acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = seed + 0.37f * float(threadIdx.x + c);
        acc[c] = 0u;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                uint32_t h;
                asm volatile("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x[c]), "f"(__uint_as_float(acc[c])));
                acc[c] ^= h;
            }
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= acc[c];
    if (s == 0x12345678u) sink[0] = float(s);
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" int krr_probe_rate(krr_ctx *k, int32_t which, double *ops_per_second) {
    if (!k || !ops_per_second || which < 0 || which > 3) return fail(KRR_ERR_INVALID_ARG, "krr_probe_rate: bad arguments");
    Ctx *c = &k->c;
    DBuf<double> sink(c, 1);
    if (!sink.get()) return fail(KRR_ERR_OOM, "krr_probe_rate: out of memory");
    const int blocks = 4 * c->num_sms;  // 4 x 512 threads: 64 warps per SM
    const int iters = which == 1 ? 256 : 2048;
    cudaEvent_t e0, e1;
    KRR_CUDA(cudaEventCreate(&e0));
    KRR_CUDA(cudaEventCreate(&e1));
    float best = 0.f;
    for (int rep = 0; rep < 4; ++rep) {  // first launch warms up
        KRR_CUDA(cudaEventRecord(e0, c->stream));
        float *fs = reinterpret_cast<float *>(sink.get());
        switch (which) {
            case 0: probe_fma32<<<blocks, kProbeThreads, 0, c->stream>>>(iters, 0.5f, fs); break;
            case 1: probe_fma64<<<blocks, kProbeThreads, 0, c->stream>>>(iters, 0.5, sink.get()); break;
            case 2: probe_ex2<<<blocks, kProbeThreads, 0, c->stream>>>(iters, 0.5f, fs); break;
            default: probe_cvt<<<blocks, kProbeThreads, 0, c->stream>>>(iters, 0.5f, fs); break;
        }
        count_launch();
        KRR_CUDA(cudaGetLastError());
        KRR_CUDA(cudaEventRecord(e1, c->stream));
        KRR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        KRR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // per-lane operations: FMA counts 2 flops; a packed conversion 2 values
    const double lanes = double(blocks) * kProbeThreads * double(iters) * 16.0 * kChains;
    const double per_op = (which == 0 || which == 1 || which == 3) ? 2.0 : 1.0;
    *ops_per_second = lanes * per_op / (double(best) * 1e-3);
    return KRR_OK;
}
