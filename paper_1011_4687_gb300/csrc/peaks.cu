// Pipe-throughput microbenchmarks: the denominators of the potential kernels'
// rooflines on the GPU at hand.
//
// The paper estimates the peaks of its CPU and GPU from unit counts and
// clocks (Table performances) and compares its kernel against them.  Here the
// peaks are measured: every thread runs kChains independent dependency chains
// of one instruction kind, enough warps per SM to hide each pipe's latency,
// timed with CUDA events after a warm-up launch.  The rate is reported in
// instructions per second summed over all lanes ("lane ops"), the unit in
// which the potential kernels' algorithmic FP32 / FP64 counts are stated.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/esp.h"
#include "esp_ctx.h"

using namespace esp;

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) ffma_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = float(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = fmaf(x[k], a, b);
    }
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        acc += x[k];
    if (acc == 12345.678f) // never true for the arguments used; keeps the chains live
        out[blockIdx.x] = acc;
}

// Packed FP32 pairs (sm_100 and later): one instruction does two lanes' FMAs.
__global__ void __launch_bounds__(kThreads) ffma2_kernel(float *out, int iters, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        x[k] = make_float2(float(threadIdx.x + k) * 1e-3f, float(threadIdx.x + 2 * k) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k)
                x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        acc += x[k].x + x[k].y;
    if (acc == 12345.678f)
        out[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) dfma_kernel(double *out, int iters, double a, double b)
{
    double x[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        x[k] = double(threadIdx.x + k) * 1e-3;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k)
                x[k] = fma(x[k], a, b);
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
        acc += x[k];
    if (acc == 12345.678)
        out[blockIdx.x] = acc;
}

// MUFU reciprocal square root: x <- rsqrt(x) converges to 1, no special values.
__global__ void __launch_bounds__(kThreads) rsqrt_kernel(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = 1.5f + float(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = rsqrtf(x[k]);
    }
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        acc += x[k];
    if (acc == 12345.678f)
        out[blockIdx.x] = acc;
}

// MUFU base-2 exponential: x <- 2^-x converges near 0.64.
__device__ __forceinline__ float ex2_neg(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

__global__ void __launch_bounds__(kThreads) ex2_kernel(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        x[k] = 0.5f + float(threadIdx.x + k) * 1e-4f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                x[k] = ex2_neg(x[k]);
    }
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        acc += x[k];
    if (acc == 12345.678f)
        out[blockIdx.x] = acc;
}

// Times `launch` (one warm-up, then `reps` launches between two events) and
// returns the rate of `ops_per_launch` in ops per second.
template <typename F>
esp_status time_rate(F launch, double ops_per_launch, int reps, double *rate, double *ms_out)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return cuda_fail(e, "creating timing events");
    }
    launch();
    e = cudaEventRecord(e0, 0);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return cuda_fail(e, "timing a microbenchmark");
    *rate = ops_per_launch * reps / (double(ms) * 1e-3);
    *ms_out = ms / reps;
    return ESP_OK;
}

} // namespace

extern "C" esp_status esp_measure_peaks(int32_t device, esp_peaks *out)
{
    last_error().clear();
    if (!out)
        return fail(ESP_ERR_INVALID, "out is NULL");
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
        return fail(ESP_ERR_CUDA, "no CUDA device");
    DeviceGuard dg(dev);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", dev);
    int sms = 0, clock_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    if (sms <= 0)
        return fail(ESP_ERR_CUDA, "cannot read the SM count of device %d", dev);
    float *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, size_t(sms) * kBlocksPerSm * sizeof(double));
    if (e != cudaSuccess)
        return cuda_fail(e, "allocating microbenchmark scratch");
    const int grid = sms * kBlocksPerSm;
    const double lanes = double(grid) * kThreads;
    esp_peaks p;
    std::memset(&p, 0, sizeof(p));
    p.num_sms = sms;
    p.clock_khz = clock_khz;
    const int it32 = 4096, it64 = 64, itmufu = 512;
    esp_status st = time_rate([&] { ffma_kernel<<<grid, kThreads>>>(scratch, it32, 0.999f, 1e-3f); },
                              lanes * it32 * 8 * kChains, 5, &p.fp32_fma_per_s, &p.fp32_ms);
    if (st == ESP_OK)
        st = time_rate([&] { ffma2_kernel<<<grid, kThreads>>>(scratch, it32, 0.999f, 1e-3f); },
                       lanes * it32 * 8 * kChains, 5, &p.fp32x2_fma_per_s, &p.fp32x2_ms);
    if (st == ESP_OK)
        st = time_rate([&] { dfma_kernel<<<grid, kThreads>>>(reinterpret_cast<double *>(scratch), it64, 0.999, 1e-3); },
                       lanes * it64 * 8 * (kChains / 2), 5, &p.fp64_fma_per_s, &p.fp64_ms);
    if (st == ESP_OK)
        st = time_rate([&] { rsqrt_kernel<<<grid, kThreads>>>(scratch, itmufu); }, lanes * itmufu * 8 * kChains, 5,
                       &p.mufu_rsqrt_per_s, &p.rsqrt_ms);
    if (st == ESP_OK)
        st = time_rate([&] { ex2_kernel<<<grid, kThreads>>>(scratch, itmufu); }, lanes * itmufu * 8 * kChains, 5,
                       &p.mufu_ex2_per_s, &p.ex2_ms);
    cudaFree(scratch);
    if (st != ESP_OK)
        return st;
    *out = p;
    return ESP_OK;
}
