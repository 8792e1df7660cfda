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

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// packed FP32x2 FMA (two FMAs per lane per instruction)
__global__ void __launch_bounds__(kPeakTpb) ffma2_probe(int iters, float a, float b, float *sink)
{
    unsigned long long x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    const unsigned long long ua = *reinterpret_cast<const unsigned long long *>(&a2);
    const unsigned long long ub = *reinterpret_cast<const unsigned long long *>(&b2);
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float2 v = make_float2(threadIdx.x * 1e-3f + k, threadIdx.x * 2e-3f + k);
        x[k] = *reinterpret_cast<unsigned long long *>(&v);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = ffma2(x[k], ua, ub);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float2 v = *reinterpret_cast<float2 *>(&x[k]);
        s += v.x + v.y;
    }
    if (s == 12345.678f) sink[0] = s;
}

// packed FP32x2 FMA chains interleaved with scalar FMA chains (4 + 4): shows whether scalar
// FMAs run beside packed ones
__global__ void __launch_bounds__(kPeakTpb) mixed_probe(int iters, float a, float b, float *sink)
{
    unsigned long long x[kChains / 2];
    float y[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    const unsigned long long ua = *reinterpret_cast<const unsigned long long *>(&a2);
    const unsigned long long ub = *reinterpret_cast<const unsigned long long *>(&b2);
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) {
        float2 v = make_float2(threadIdx.x * 1e-3f + k, threadIdx.x * 2e-3f + k);
        x[k] = *reinterpret_cast<unsigned long long *>(&v);
        y[k] = threadIdx.x * 3e-3f + k;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) {
                x[k] = ffma2(x[k], ua, ub);
                y[k] = fmaf(y[k], a, b);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) {
        float2 v = *reinterpret_cast<float2 *>(&x[k]);
        s += v.x + v.y + y[k];
    }
    if (s == 12345.678f) sink[0] = s;
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

// One CTA waits on a shared-memory mbarrier phase with the same bounded try-wait the
// Birkhoff-Rott kernels use for their bulk copies.  With arrive = 0 nothing ever arrives (the
// flag that nothing sets), so the wait gives up after max_polls polls and the kernel records
// kErrTimeout in *status and returns; with arrive = 1 one thread arrives first and the wait
// completes.  Nothing is left in flight either way.
__global__ void wait_selftest_kernel(long long max_polls, int arrive, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dev::smem_u32(&bar)) : "memory");
    __syncthreads();
    bool done = false;
    for (long long it = 0; it < max_polls && !done; ++it) done = dev::mbar_try_wait(&bar, 0);
    __syncthreads();
    if (threadIdx.x == 0) *status = done ? 0 : kErrTimeout;
}

}  // namespace
}  // namespace zm

using namespace zm;

extern "C" int zm_wait_selftest(int64_t max_polls, int32_t arrive, double *elapsed_ms)
{
    if (max_polls < 1 || max_polls > ((int64_t)1 << 34) || (arrive != 0 && arrive != 1))
        return set_error(ZM_ERR_INVALID, "zm_wait_selftest: max_polls in [1, 2^34], arrive 0 or 1");
    int *status = nullptr;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "zm_wait_selftest: alloc");
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    wait_selftest_kernel<<<1, 32>>>((long long)max_polls, arrive, status);
    cudaEventRecord(b);
    int rc = cuda_check(cudaGetLastError(), "zm_wait_selftest launch");
    int h = 0;
    if (!rc) rc = cuda_check(cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost), "zm_wait_selftest");
    float ms = 0.f;
    if (!rc) cudaEventElapsedTime(&ms, a, b);
    if (elapsed_ms) *elapsed_ms = ms;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(status);
    if (!rc && (h & kErrTimeout))
        rc = set_error(ZM_ERR_TIMEOUT, "zm_wait_selftest: the bounded device-side wait gave up (as intended)");
    return rc;
}

extern "C" int64_t zm_wait_poll_limit(void) { return (int64_t)dev::kSpinLimit; }

extern "C" int zm_checked_build(void) { return ZM_CHECKS ? 1 : 0; }

extern "C" int zm_bounds_status(uint32_t *hits, int64_t *first_index, int32_t *source_line, int32_t clear)
{
    if (!hits) return set_error(ZM_ERR_INVALID, "zm_bounds_status: null hits");
    if (cudaDeviceSynchronize() != cudaSuccess) return set_error(ZM_ERR_CUDA, "zm_bounds_status: device error");
    unsigned int h = 0;
    long long f = -1;
    int line = 0;
    int (*const readers[])(unsigned int *, long long *, int *, int) = {
        bounds_api, bounds_batch, bounds_br, bounds_br32, bounds_br32tc, bounds_fft, bounds_lowdf, bounds_lowdf_mix,
        bounds_stencil};
    for (auto rd : readers)
        if (rd(&h, &f, &line, clear ? 1 : 0) != 0) return set_error(ZM_ERR_CUDA, "zm_bounds_status: read failed");
    *hits = h;
    if (first_index) *first_index = h ? f : -1;
    if (source_line) *source_line = h ? line : 0;
    return ZM_OK;
}

extern "C" int zm_measure_peak(int kind, double *ops_per_s)
{
    if (!ops_per_s || kind < 0 || kind > 4) return set_error(ZM_ERR_INVALID, "zm_measure_peak: bad argument");
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
        else if (kind == 2) rsqrt_probe<<<blocks, kPeakTpb>>>(iters, (float *)sink);
        else if (kind == 3) ffma2_probe<<<blocks, kPeakTpb>>>(iters, 0.999f, 1e-3f, (float *)sink);
        else mixed_probe<<<blocks, kPeakTpb>>>(iters, 0.999f, 1e-3f, (float *)sink);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    const double ops = (double)blocks * kPeakTpb * iters * 16.0 * kChains;
    // FMA probes report flops (FMA = 2; a packed x2 FMA = 4; the mixed probe does one packed and
    // one scalar FMA per chain pair = 6 flops per 2 chain steps); the rsqrt probe reports operations
    const double per = (kind == 2) ? 1.0 : (kind == 3) ? 4.0 : (kind == 4) ? 3.0 : 2.0;
    *ops_per_s = per * ops / (best * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return cuda_check(cudaGetLastError(), "zm_measure_peak");
}
