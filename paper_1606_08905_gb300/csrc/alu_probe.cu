// alu_probe.cu -- throughput of the FP32 and FP64 FMA pipes on this GPU
// (knor_probe_alu in include/knor.h).
//
// The plain Lloyd scan at larger k is bound by FP32 arithmetic, not by
// memory, so its roofline needs the FMA rate of the chip.  This probe
// measures it: every thread runs eight independent FMA chains (enough to
// cover the pipe latency), so the kernel issues nothing but FMAs.
#include "knor.h"
#include "knor_internal.cuh"

#include <string>

namespace knor {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

__device__ __forceinline__ unsigned long long probe_fma2(unsigned long long a, unsigned long long b,
                                                         unsigned long long c) {
    unsigned long long r;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// kind 0: FP32 fma.rn.f32; 1: packed fma.rn.f32x2 (two FP32 FMAs); 2: FP64.
template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int iters, float seed, double *sink, int store) {
    if constexpr (KIND == 0) {
        float a[PROBE_CHAINS];
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = seed + threadIdx.x + q;
        const float m = 0.999f, c = 1e-3f * seed;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = __fmaf_rn(a[q], m, c);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) s += a[q];
        if (store) sink[threadIdx.x] = s;
    } else if constexpr (KIND == 1) {
        unsigned long long a[PROBE_CHAINS];
        const float x0 = seed + threadIdx.x;
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) {
            const float lo = x0 + q, hi = x0 - q;
            asm("mov.b64 %0, {%1, %2};" : "=l"(a[q]) : "f"(lo), "f"(hi));
        }
        unsigned long long m, c;
        const float mf = 0.999f, cf = 1e-3f * seed;
        asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(mf));
        asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(cf));
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = probe_fma2(a[q], m, c);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[q]));
            s += lo + hi;
        }
        if (store) sink[threadIdx.x] = s;
    } else {
        double a[PROBE_CHAINS];
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = (double)seed + threadIdx.x + q;
        const double m = 0.999, c = 1e-3 * seed;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = __fma_rn(a[q], m, c);
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) s += a[q];
        if (store) sink[threadIdx.x] = s;
    }
}

template <int KIND>
cudaError_t probe_launch(int grid, int iters, double *sink, cudaStream_t s) {
    k_probe_fma<KIND><<<grid, PROBE_THREADS, 0, s>>>(iters, 1.0f, sink, 0);
    return cudaGetLastError();
}

} // namespace
} // namespace knor

extern "C" knor_status knor_probe_alu(int32_t kind, double *tflops_out, float *ms_out) {
    using namespace knor;
    set_global_error("");
    if (kind < 0 || kind > 2 || !tflops_out) {
        set_global_error("knor_probe_alu: kind must be 0, 1 or 2 and tflops_out non-NULL");
        return KNOR_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // eight CTAs of 256 threads per SM; FP64 runs far fewer iterations
    const int grid = 8 * sms;
    const int iters = kind == 2 ? 1 << 12 : 1 << 16;
    auto launch = [&]() {
        return kind == 0 ? probe_launch<0>(grid, iters, nullptr, s)
               : kind == 1 ? probe_launch<1>(grid, iters, nullptr, s)
                           : probe_launch<2>(grid, iters, nullptr, s);
    };
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) { // rep 0 warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        set_global_error((std::string("knor_probe_alu: ") + cudaGetErrorString(e)).c_str());
        return KNOR_ERR_CUDA;
    }
    const double fmas = (double)grid * PROBE_THREADS * PROBE_CHAINS * iters * (kind == 1 ? 2.0 : 1.0);
    *tflops_out = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return KNOR_OK;
}
