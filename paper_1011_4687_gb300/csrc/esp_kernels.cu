// Staging, reduction and dispatch of the potential kernels for sm_103a.
//
// The potential kernels themselves are templates in esp_potential.cuh; each
// launch shape is compiled into its own object from esp_shape.cu, and the
// dispatchers below pick the shape's launcher.
#include "esp_potential.cuh"
#include "esp_shapes.h"

#include <algorithm>

namespace esp {

namespace {

// ---------------------------------------------------------------------------
// staging: recentre in FP64, split into FP32 hi + lo
// ---------------------------------------------------------------------------
__global__ void stage_kernel(const double *__restrict__ pos, int n, double cx, double cy, double cz, double q,
                             Staged st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double x = pos[3 * i] - cx, y = pos[3 * i + 1] - cy, z = pos[3 * i + 2] - cz;
    st.x64[i] = x;
    st.y64[i] = y;
    st.z64[i] = z;
    // hi words on the environment's coordinate grid q (see the pair builder)
    double xh = nearbyint(x / q) * q, yh = nearbyint(y / q) * q, zh = nearbyint(z / q) * q;
    st.xh[i] = (float)xh;
    st.yh[i] = (float)yh;
    st.zh[i] = (float)zh;
    st.xl[i] = (float)(x - xh);
    st.yl[i] = (float)(y - yh);
    st.zl[i] = (float)(z - zh);
}

__global__ void batch_stage_kernel(const BatchHeader *__restrict__ hdr, const SysDesc *__restrict__ sys)
{
    const int total = hdr->n_pos_total, n_sys = hdr->n_sys;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const SysDesc &d = sys[find_sys(sys, n_sys, g, false)];
        const int i = g - d.pos_begin;
        double x = d.pos_in[3 * i] - d.qm[0], y = d.pos_in[3 * i + 1] - d.qm[1], z = d.pos_in[3 * i + 2] - d.qm[2];
        d.st.x64[i] = x;
        d.st.y64[i] = y;
        d.st.z64[i] = z;
        const double q = d.quantum;
        double xh = nearbyint(x / q) * q, yh = nearbyint(y / q) * q, zh = nearbyint(z / q) * q;
        d.st.xh[i] = (float)xh;
        d.st.yh[i] = (float)yh;
        d.st.zh[i] = (float)zh;
        d.st.xl[i] = (float)(x - xh);
        d.st.yl[i] = (float)(y - yh);
        d.st.zl[i] = (float)(z - zh);
    }
}

__global__ void batch_reduce_kernel(const BatchHeader *__restrict__ hdr, const SysDesc *__restrict__ sys)
{
    const int total = hdr->n_pos_total, n_sys = hdr->n_sys;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const SysDesc &d = sys[find_sys(sys, n_sys, g, false)];
        const int i = g - d.pos_begin;
        double s = 0.0, c = 0.0;
        if (d.n_tiles > 0)
            for (int k = 0; k < d.splits; ++k)
                two_sum_acc(s, c, d.partial[(size_t)k * d.n_pos + i]);
        d.V_out[i] = s + c;
    }
}

// ---------------------------------------------------------------------------
// few positions per call (the paper's call pattern: one r_new per Metropolis
// move).  The roles of the main kernels turn back to the paper's: threads
// take environment entries (cells, point charges, distributions), every
// thread evaluates its entries at all n <= kSmallN positions in FP64, the CTA
// reduces per position in a fixed order, and CTA b writes partial[b][q].
// Tiles are dealt round-robin to the CTAs; entries are read straight from the
// FP64 records (each once per call).
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 64; // one thread per entry of a full tile

__global__ void __launch_bounds__(kSmallThreads) small_n_kernel(SmallArgs a)
{
    __shared__ double s_pos[kSmallN][3];
    __shared__ double s_red[kSmallThreads / 32][kSmallN];
    const int n = a.n_pos;
    for (int i = threadIdx.x; i < n * 3; i += kSmallThreads)
        s_pos[i / 3][i % 3] = (i % 3 == 0 ? a.x64 : i % 3 == 1 ? a.y64 : a.z64)[i / 3];
    __syncthreads();
    double acc[kSmallN];
#pragma unroll
    for (int q = 0; q < kSmallN; ++q)
        acc[q] = 0.0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const TileMeta m = a.tiles[t];
        const bool pts = m.cls == kClassPoint;
        const int st = pts ? kPointStride64 : rec64_stride(m.cls & 7);
        for (int j = threadIdx.x; j < m.n; j += kSmallThreads) {
            const double *r = a.rec64 + m.off64 + (size_t)j * st;
#pragma unroll
            for (int q = 0; q < kSmallN; ++q) {
                if (q >= n)
                    break;
                if (pts) {
                    const double dx = r[0] - s_pos[q][0], dy = r[1] - s_pos[q][1], dz = r[2] - s_pos[q][2];
                    acc[q] += r[3] * esp_rsqrt(dx * dx + dy * dy + dz * dz);
                } else {
                    acc[q] += tile_f64_one_any(m.cls, r, 1, s_pos[q][0], s_pos[q][1], s_pos[q][2], a.boys64);
                }
            }
        }
    }
    // fixed-order reduction per position: warp shuffles, then the warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kSmallN; ++q) {
        if (q >= n)
            break;
        double v = acc[q];
        for (int o = 16; o; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            s_red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        double v = 0.0;
        for (int w = 0; w < kSmallThreads / 32; ++w)
            v += s_red[w][threadIdx.x];
        a.partial[(size_t)blockIdx.x * n + threadIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Many partials for few positions: one CTA per position, strided TwoSum per
// thread, then a fixed-order tree over the threads' (sum, compensation) pairs.
constexpr int kWideThreads = 256;

__global__ void __launch_bounds__(kWideThreads) reduce_wide_kernel(const double *__restrict__ partial, int n_splits,
                                                                    int n, double *__restrict__ V)
{
    __shared__ double s_s[kWideThreads], s_c[kWideThreads];
    const int q = blockIdx.x, t = threadIdx.x;
    double sum = 0.0, cmp = 0.0;
    for (int k = t; k < n_splits; k += kWideThreads)
        two_sum_acc(sum, cmp, partial[(size_t)k * n + q]);
    s_s[t] = sum;
    s_c[t] = cmp;
    __syncthreads();
    for (int o = kWideThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
            double a = s_s[t], c = s_c[t] + s_c[t + o];
            two_sum_acc(a, c, s_s[t + o]);
            s_s[t] = a;
            s_c[t] = c;
        }
        __syncthreads();
    }
    if (t == 0)
        V[q] = s_s[0] + s_c[0];
}

__global__ void reduce_kernel(const double *__restrict__ partial, int n_splits, int n, double *__restrict__ V)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double s = 0.0, c = 0.0;
    for (int k = 0; k < n_splits; ++k)
        two_sum_acc(s, c, partial[(size_t)k * n + i]);
    V[i] = s + c;
}

__global__ void walker_kernel(const double *__restrict__ V, int n_walkers, int n_elec, double *__restrict__ E)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_walkers)
        return;
    double s = 0.0, c = 0.0;
    for (int e = 0; e < n_elec; ++e)
        two_sum_acc(s, c, -V[(size_t)w * n_elec + e]);
    E[w] = s + c;
}

} // namespace

bool potential_shape_supported(int precision, int threads, int ppt)
{
#define ESP_SHAPE_IS(NT, PPT) || (threads == NT && ppt == PPT)
    if (precision == 0)
        return false ESP_F64_SHAPES(ESP_SHAPE_IS);
    return false ESP_F32C_SHAPES(ESP_SHAPE_IS);
#undef ESP_SHAPE_IS
}

size_t potential_smem_bytes(int precision, int tile_size)
{
    if (precision == 0)
        return (size_t)tile_size * 40 * sizeof(double);
    return (size_t)tile_size * kRec32MaxStride * sizeof(float) + (size_t)kBoys32Rows * kBoys32Row * sizeof(float);
}

cudaError_t launch_stage(const double *pos_in, int n, const double center[3], double quantum, const Staged &st,
                         cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    stage_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos_in, n, center[0], center[1], center[2], quantum, st);
    return cudaGetLastError();
}

cudaError_t launch_potential(int precision, const EvalArgs &a, int threads, int ppt, cudaStream_t s)
{
    if (a.n_pos <= 0)
        return cudaSuccess;
    const int per_cta = threads * ppt;
    dim3 grid((a.n_pos + per_cta - 1) / per_cta, a.n_splits);
    size_t smem = potential_smem_bytes(precision, a.tile_size);
#define ESP_LAUNCH_F64(NT, PPT) \
    if (threads == NT && ppt == PPT) return launch_f64_shape<NT, PPT>(a, grid, smem, s);
#define ESP_LAUNCH_F32C(NT, PPT) \
    if (threads == NT && ppt == PPT) return launch_f32c_shape<NT, PPT>(a, grid, smem, s);
    if (precision == 0) {
        ESP_F64_SHAPES(ESP_LAUNCH_F64)
    } else {
        ESP_F32C_SHAPES(ESP_LAUNCH_F32C)
    }
#undef ESP_LAUNCH_F64
#undef ESP_LAUNCH_F32C
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_batch(int precision, const BatchHeader *hdr, const SysDesc *sys, int *counter, int max_items,
                         const float *boys32, const double *boys64, int tile_cap, int threads, int ppt,
                         int num_sms, int max_pos_total, cudaStream_t s)
{
    const int sgrid = std::max(1, std::min(4 * num_sms, (max_pos_total + 255) / 256));
    batch_stage_kernel<<<sgrid, 256, 0, s>>>(hdr, sys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t smem = potential_smem_bytes(precision, tile_cap);
    bool launched = false;
#define ESP_BLAUNCH(NT, PPT, PR)                                                                                \
    if (!launched && threads == NT && ppt == PPT && precision == PR) {                                        \
        e = launch_batch_shape<NT, PPT, PR>(hdr, sys, counter, max_items, boys32, boys64, tile_cap, num_sms, smem, s); \
        launched = true;                                                                                      \
    }
    ESP_BATCH_SHAPES(ESP_BLAUNCH)
#undef ESP_BLAUNCH
    if (!launched)
        return cudaErrorInvalidConfiguration;
    if (e != cudaSuccess)
        return e;
    batch_reduce_kernel<<<sgrid, 256, 0, s>>>(hdr, sys);
    return cudaGetLastError();
}

bool batch_shape_supported(int precision, int threads, int ppt)
{
#define ESP_BSHAPE_IS(NT, PPT, PR) || (threads == NT && ppt == PPT && precision == PR)
    return false ESP_BATCH_SHAPES(ESP_BSHAPE_IS);
#undef ESP_BSHAPE_IS
}

int small_n_splits(int n_tiles, int num_sms) { return std::max(1, std::min(n_tiles, 8 * num_sms)); }

cudaError_t launch_small_n(const SmallArgs &a, int n_splits, double *V, cudaStream_t s)
{
    if (a.n_pos <= 0 || a.n_pos > kSmallN)
        return cudaErrorInvalidValue;
    small_n_kernel<<<n_splits, kSmallThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    reduce_wide_kernel<<<a.n_pos, kWideThreads, 0, s>>>(a.partial, n_splits, a.n_pos, V);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partial, int n_splits, int n, double *V, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, n_splits, n, V);
    return cudaGetLastError();
}

cudaError_t launch_walkers(const double *V, int n_walkers, int n_elec, double *E, cudaStream_t s)
{
    if (n_walkers <= 0)
        return cudaSuccess;
    walker_kernel<<<(n_walkers + 127) / 128, 128, 0, s>>>(V, n_walkers, n_elec, E);
    return cudaGetLastError();
}

} // namespace esp
