// Work census: how many (distribution, position) terms of an evaluation fall
// in each regime of the Boys function, by total angular momentum L.
//
// The potential kernels evaluate every term by McMurchie-Davidson (the
// generalisation of one cell term of Eq. ElectrostaticField, Sec. II.B):
// Boys F_0..F_L(T) at T = p |P - C|^2, then the Hermite recursion and
// contraction.  How many operations a term needs depends on T: at and above
// T = 30 (FP32 path) or 45 (FP64 path) the asymptotic form applies, below it
// the Taylor table with downward recursion.  The census gives the mix for a
// sample of positions, from which the algorithmic operation count of a launch
// (the numerator of its roofline) follows.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/esp.h"
#include "esp_ctx.h"

using namespace esp;

namespace {

constexpr int kCensusThreads = 128;
constexpr int kCensusMaxPositions = ESP_CENSUS_MAX_POSITIONS; // 48 KB of positions in shared memory

// counts layout: [(L + 5 * short) * 3 + band] for band 0: T < 30, 1: 30 <= T < 45,
// 2: T >= 45; [30]: FP64 point-charge terms; [31]: FP32 point-charge terms
__global__ void __launch_bounds__(kCensusThreads) census_kernel(const TileMeta *__restrict__ tiles,
                                                                const double *__restrict__ rec64,
                                                                const float *__restrict__ pos, int n,
                                                                unsigned long long *__restrict__ counts)
{
    __shared__ float s_pos[kCensusMaxPositions * 3];
    __shared__ unsigned long long s_cnt[32];
    for (int i = threadIdx.x; i < n * 3; i += kCensusThreads)
        s_pos[i] = pos[i];
    if (threadIdx.x < 32)
        s_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    const TileMeta m = tiles[blockIdx.x];
    if (is_point_class(m.cls)) {
        if (threadIdx.x == 0)
            atomicAdd(&s_cnt[m.cls == kClassPoint ? 30 : 31], (unsigned long long)m.n * (unsigned long long)n);
    } else {
        const int L = m.cls & 7;
        const int base = (L + ((m.cls & kClassShortBit) ? 5 : 0)) * 3;
        const int st = rec64_stride(L);
        for (int j = threadIdx.x; j < m.n; j += kCensusThreads) {
            const double *r = rec64 + m.off64 + (size_t)j * st;
            const float px = float(r[0]), py = float(r[1]), pz = float(r[2]);
            const float p = float(r[3] * r[3]);
            unsigned c0 = 0, c1 = 0;
            for (int i = 0; i < n; ++i) {
                const float dx = px - s_pos[3 * i], dy = py - s_pos[3 * i + 1], dz = pz - s_pos[3 * i + 2];
                const float T = p * (dx * dx + dy * dy + dz * dz);
                c0 += T < 30.0f;
                c1 += T >= 30.0f && T < 45.0f;
            }
            atomicAdd(&s_cnt[base], (unsigned long long)c0);
            atomicAdd(&s_cnt[base + 1], (unsigned long long)c1);
            atomicAdd(&s_cnt[base + 2], (unsigned long long)(n - c0 - c1));
        }
    }
    __syncthreads();
    if (threadIdx.x < 32 && s_cnt[threadIdx.x])
        atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

} // namespace

extern "C" esp_status esp_work_census(esp_ctx *ctx, const double *positions, int64_t n, int64_t *counts)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!counts || n < 0 || n > kCensusMaxPositions || (n > 0 && !positions))
        return fail(ESP_ERR_INVALID, "census takes a host array of 0..%d positions and a counts array",
                    kCensusMaxPositions);
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(ctx->device);
    if (!dg.ok)
        return fail(ESP_ERR_CUDA, "cannot select device %d", ctx->device);
    if (classify(positions, ctx->device) != Space::Host)
        return fail(ESP_ERR_INVALID, "census positions must be host memory");
    std::vector<float> rel(size_t(n) * 3);
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            rel[size_t(i) * 3 + d] = float(positions[3 * i + d] - ctx->opt.qm_center[d]);
    float *d_pos = nullptr;
    unsigned long long *d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_pos, std::max<size_t>(rel.size(), 1) * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&d_cnt, 32 * sizeof(unsigned long long));
    cudaStream_t s = ctx->stream;
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(d_pos, rel.data(), rel.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_cnt, 0, 32 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && n > 0 && ctx->n_tiles > 0) {
        census_kernel<<<ctx->n_tiles, kCensusThreads, 0, s>>>(static_cast<const TileMeta *>(ctx->tiles.p),
                                                               static_cast<const double *>(ctx->rec64.p), d_pos,
                                                               int(n), d_cnt);
        e = cudaGetLastError();
    }
    unsigned long long h[32] = {0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (d_pos)
        cudaFree(d_pos);
    if (d_cnt)
        cudaFree(d_cnt);
    if (e != cudaSuccess)
        return cuda_fail(e, "work census");
    for (int k = 0; k < 32; ++k)
        counts[k] = int64_t(h[k]);
    return ESP_OK;
}
