// k_peaks.cu -- measured FP32 issue peaks of the device (instrumentation for
// the filter's roofline; the paper has no counterpart): independent chains
// of scalar FMA, paired FMA (fma.rn.f32x2) and ex2.approx in every thread
// of a grid that fills the GPU, timed with CUDA events.
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float seed, float *sink) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + (float)(threadIdx.x + k);
    const float m = 0.999999f, c = 1e-7f;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma2(float seed, float *sink) {
    unsigned long long a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float v = seed + (float)(threadIdx.x + k);
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(v), "f"(v + 1.f));
    }
    unsigned long long m, c;
    asm("mov.b64 %0, {%1, %2};" : "=l"(m) : "f"(0.999999f), "f"(0.999999f));
    asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(1e-7f), "f"(1e-7f));
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(m), "l"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
        s += x + y;
    }
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

// ex2 chains kept in range by one FMA each: x <- 0.25 - 0.5 * 2^x stays in
// [-0.35, 0]; the FMA issues on another pipe.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(float seed, float *sink) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = -seed * (float)(k + 1) * 1e-3f - 1e-6f * (float)threadIdx.x;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
            a[k] = fmaf(y, -0.5f, 0.25f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

template <typename K>
float time_kernel(K kernel, int grid, float *sink, cudaStream_t s, cudaError_t &e) {
    cudaEvent_t a = nullptr, b = nullptr;
    float best = 0.f;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
        e = cudaEventRecord(a, s);
        kernel<<<grid, kPeakThreads, 0, s>>>(1.0f, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return best;
}

}  // namespace
}  // namespace afr

// Measured FP32 rates of the current device: out_host[0] = scalar FMA
// TFLOP/s (2 FLOP each), out_host[1] = paired FMA (fma.rn.f32x2) TFLOP/s,
// out_host[2] = ex2.approx Tops/s, out_host[3] = SM count. Synchronises.
extern "C" AfrStatus afr_measure_alu_peaks(float *out_host) {
    using namespace afr;
    if (!out_host) return AFR_ERR_INVALID_ARG;
    const int sms = device_sms();
    const int grid = sms * 8;   // 8 blocks of 256 threads per SM: full occupancy at these register counts
    float *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * kPeakThreads);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? AFR_ERR_OOM : AFR_ERR_CUDA;
    }
    const double threads = (double)grid * kPeakThreads, ops = threads * kChains * kIters;
    const float ms1 = time_kernel(k_peak_fma, grid, sink, 0, e);
    float ms2 = 0.f, ms3 = 0.f;
    if (e == cudaSuccess) ms2 = time_kernel(k_peak_fma2, grid, sink, 0, e);
    if (e == cudaSuccess) ms3 = time_kernel(k_peak_ex2, grid, sink, 0, e);
    cudaFree(sink);
    if (e != cudaSuccess || ms1 <= 0.f || ms2 <= 0.f || ms3 <= 0.f) {
        cudaGetLastError();
        return AFR_ERR_CUDA;
    }
    out_host[0] = (float)(2.0 * ops / (ms1 * 1e-3) / 1e12);
    out_host[1] = (float)(4.0 * ops / (ms2 * 1e-3) / 1e12);
    out_host[2] = (float)(ops / (ms3 * 1e-3) / 1e12);
    out_host[3] = (float)sms;
    return AFR_OK;
}
