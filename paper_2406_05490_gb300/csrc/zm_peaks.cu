// zm_peaks.cu -- CUDA-core throughput probes used as roofline denominators for the
// Birkhoff-Rott kernels (FP32 FMA, FP64 FMA and MUFU rsqrt issue rates of this GPU, measured
// with CUDA events; the copy bandwidth and tensor peaks come from elsewhere).  The paper has no
// counterpart: it reports no single-GPU rates.
#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kPeakTpb = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(kPeakTpb) ffma_probe(int iters, float a, float b, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 12345.678f) sink[0] = s;  // never true for the probe inputs; keeps the work alive
}

__global__ void __launch_bounds__(kPeakTpb) dfma_probe(int iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 12345.678) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakTpb) rsqrt_probe(int iters, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0f + threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = dev::rsqrt_approx(x[k]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace
}  // namespace zm

using namespace zm;

extern "C" int zm_measure_peak(int kind, double *ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 2) return set_error(ZM_ERR_INVALID, "zm_measure_peak: bad argument");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return set_error(ZM_ERR_NOMEM, "zm_measure_peak: alloc");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8;
    const int iters = (kind == 1) ? 64 : 2048;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        if (kind == 0) ffma_probe<<<blocks, kPeakTpb>>>(iters, 0.999f, 1e-3f, (float *)sink);
        else if (kind == 1) dfma_probe<<<blocks, kPeakTpb>>>(iters, 0.999, 1e-3, (double *)sink);
        else rsqrt_probe<<<blocks, kPeakTpb>>>(iters, (float *)sink);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    const double ops = (double)blocks * kPeakTpb * iters * 16.0 * kChains;
    // FMA probes report flops (FMA = 2); the rsqrt probe reports operations
    *ops_per_s = (kind == 2 ? 1.0 : 2.0) * ops / (best * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return cuda_check(cudaGetLastError(), "zm_measure_peak");
}
