// Potential kernels for sm_103a.
//
// The paper's kernel (Sec. III, Eq. blockSum and Eq. coalease) splits the cell
// sum over N_B blocks of N_th threads, each thread striding through the cell
// array so that neighbouring threads read neighbouring cells (coalescing), and
// reduces per block in shared memory; one position r_new sits in constant
// memory.  Here many positions are evaluated per launch, so the roles turn
// around: each thread keeps PPT positions in registers, a CTA stages one tile
// of distributions at a time in shared memory with coalesced 16-byte loads,
// and every warp reads the tile's records as same-address broadcasts.  Tiles
// are dealt round-robin to `n_splits` CTAs per position block; each split
// writes its own FP64 partial, and a separate kernel sums the partials in a
// fixed order (deterministic, no atomics on the result).
#include "esp_eval_core.h"
#include "esp_kernels.h"

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

__device__ __forceinline__ void copy_tile(float4 *__restrict__ dst, const float4 *__restrict__ src, int nvec)
{
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
        dst[i] = __ldg(src + i);
}

// ---------------------------------------------------------------------------
// FP32C kernel
// ---------------------------------------------------------------------------
// One CTA's work in the FP32C kernel: position block bx against the tiles of
// split `split` (tiles split, split + n_splits, ...).  The Boys table is
// already in shared memory (s_boys); s_tile4 holds one staged tile.
template <int NT, int PPT>
__device__ __forceinline__ void cta_f32c(const EvalArgs &a, int bx, int split, float4 *s_tile4,
                                         const float *s_boys)
{
    const int base = bx * NT * PPT + threadIdx.x;
    float ch[PPT][3], cl[PPT][3];
    float S[PPT], Cc[PPT];
    double acc64[PPT];
    int idx[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int i = base + q * NT;
        idx[q] = i;
        int ic = min(i, a.n_pos - 1);
        ch[q][0] = a.pos.xh[ic];
        ch[q][1] = a.pos.yh[ic];
        ch[q][2] = a.pos.zh[ic];
        cl[q][0] = a.pos.xl[ic];
        cl[q][1] = a.pos.yl[ic];
        cl[q][2] = a.pos.zl[ic];
        S[q] = 0.0f;
        Cc[q] = 0.0f;
        acc64[q] = 0.0;
    }
    const float near_r = a.near_r;
    for (int t = split; t < a.n_tiles; t += a.n_splits) {
        const TileMeta m = a.tiles[t];
        __syncthreads(); // previous tile fully consumed
        const bool pts = m.cls == kClassPoint;
        const float4 *src = pts ? reinterpret_cast<const float4 *>(a.rec64 + m.off64)
                                : reinterpret_cast<const float4 *>(a.rec32 + m.off32);
        const int nvec = pts ? m.n * 2 : (m.n * rec32_stride(m.cls & 7)) / 4;
        copy_tile(s_tile4, src, nvec);
        __syncthreads();
        if (pts) {
            double c64[PPT][3];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                int ic = min(idx[q], a.n_pos - 1);
                c64[q][0] = a.pos.x64[ic];
                c64[q][1] = a.pos.y64[ic];
                c64[q][2] = a.pos.z64[ic];
            }
            tile_points_f64<PPT>(reinterpret_cast<const double *>(s_tile4), m.n, c64, acc64);
            continue;
        }
        bool nearq[PPT];
        bool any_near = false, lane_far = true;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            bool f;
            classify_tile(m, ch[q][0], ch[q][1], ch[q][2], near_r, nearq[q], f);
            any_near |= nearq[q];
            lane_far &= f;
        }
        const bool far = __all_sync(0xffffffffu, lane_far);
        const float *s_rec = reinterpret_cast<const float *>(s_tile4);
#define ESP_TILE(CLS, LL, SH)                                                           \
    case CLS:                                                                           \
        if (far)                                                                        \
            tile_f32c<LL, PPT, true, SH>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys);     \
        else                                                                            \
            tile_f32c<LL, PPT, false, SH>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys);    \
        break;
        switch (m.cls) {
            ESP_TILE(0, 0, false)
            ESP_TILE(1, 1, false)
            ESP_TILE(2, 2, false)
            ESP_TILE(3, 3, false)
            ESP_TILE(4, 4, false)
            ESP_TILE(8, 0, true)
            ESP_TILE(9, 1, true)
            ESP_TILE(10, 2, true)
            ESP_TILE(11, 3, true)
            default:
            ESP_TILE(12, 4, true)
        }
#undef ESP_TILE
        if (any_near) {
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (nearq[q]) {
                    int ic = min(idx[q], a.n_pos - 1);
                    acc64[q] += tile_f64_one_any(m.cls, a.rec64 + m.off64, m.n, a.pos.x64[ic], a.pos.y64[ic],
                                                 a.pos.z64[ic], a.boys64);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (idx[q] < a.n_pos)
            a.partial[(size_t)split * a.n_pos + idx[q]] = ((double)S[q] + (double)Cc[q]) + acc64[q];
}

template <int NT, int PPT>
__global__ void __launch_bounds__(NT) potential_f32c_kernel(EvalArgs a)
{
    extern __shared__ float4 smem4[];
    float4 *s_tile4 = smem4;
    float *s_boys = reinterpret_cast<float *>(smem4 + (a.tile_size * kRec32MaxStride) / 4);
    for (int i = threadIdx.x; i < kBoys32Rows * kBoys32Row; i += NT)
        s_boys[i] = a.boys32[i];
    cta_f32c<NT, PPT>(a, blockIdx.x, blockIdx.y, s_tile4, s_boys);
}

// ---------------------------------------------------------------------------
// FP64 kernel
// ---------------------------------------------------------------------------
template <int L, int PPT, bool SHORT>
__device__ __forceinline__ void tile_f64(const double *__restrict__ s_rec, int n, const double (&c)[PPT][3],
                                         double (&tacc)[PPT], const double *__restrict__ boys64)
{
    constexpr int st = rec64_stride(L);
    for (int j = 0; j < n; ++j) {
        const double *r = s_rec + j * st;
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            tacc[q] += dist_f64<L, SHORT>(r, c[q][0], c[q][1], c[q][2], boys64);
    }
}

template <int NT, int PPT>
__device__ __forceinline__ void cta_f64(const EvalArgs &a, int bx, int split, float4 *smem4)
{
    const double *s_rec = reinterpret_cast<const double *>(smem4);
    const int base = bx * NT * PPT + threadIdx.x;
    double c[PPT][3], S[PPT], Cc[PPT];
    int idx[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int i = base + q * NT;
        idx[q] = i;
        int ic = min(i, a.n_pos - 1);
        c[q][0] = a.pos.x64[ic];
        c[q][1] = a.pos.y64[ic];
        c[q][2] = a.pos.z64[ic];
        S[q] = 0.0;
        Cc[q] = 0.0;
    }
    for (int t = split; t < a.n_tiles; t += a.n_splits) {
        const TileMeta m = a.tiles[t];
        __syncthreads();
        const bool pts = m.cls == kClassPoint;
        const int nvec = pts ? m.n * 2 : (m.n * rec64_stride(m.cls & 7)) / 2;
        copy_tile(smem4, reinterpret_cast<const float4 *>(a.rec64 + m.off64), nvec);
        __syncthreads();
        double tacc[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            tacc[q] = 0.0;
        if (pts) {
            tile_points_f64<PPT>(s_rec, m.n, c, tacc);
        } else {
            switch (m.cls) {
            case 0: tile_f64<0, PPT, false>(s_rec, m.n, c, tacc, a.boys64); break;
            case 1: tile_f64<1, PPT, false>(s_rec, m.n, c, tacc, a.boys64); break;
            case 2: tile_f64<2, PPT, false>(s_rec, m.n, c, tacc, a.boys64); break;
            case 3: tile_f64<3, PPT, false>(s_rec, m.n, c, tacc, a.boys64); break;
            case 4: tile_f64<4, PPT, false>(s_rec, m.n, c, tacc, a.boys64); break;
            case 8: tile_f64<0, PPT, true>(s_rec, m.n, c, tacc, a.boys64); break;
            case 9: tile_f64<1, PPT, true>(s_rec, m.n, c, tacc, a.boys64); break;
            case 10: tile_f64<2, PPT, true>(s_rec, m.n, c, tacc, a.boys64); break;
            case 11: tile_f64<3, PPT, true>(s_rec, m.n, c, tacc, a.boys64); break;
            default: tile_f64<4, PPT, true>(s_rec, m.n, c, tacc, a.boys64); break;
            }
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            two_sum_acc(S[q], Cc[q], tacc[q]);
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (idx[q] < a.n_pos)
            a.partial[(size_t)split * a.n_pos + idx[q]] = S[q] + Cc[q];
}

template <int NT, int PPT>
__global__ void __launch_bounds__(NT) potential_f64_kernel(EvalArgs a)
{
    extern __shared__ float4 smem4[];
    cta_f64<NT, PPT>(a, blockIdx.x, blockIdx.y, smem4);
}

// ---------------------------------------------------------------------------
// Batched systems: persistent kernel over (system, position block, split)
// work items taken from an atomic counter, plus grid-stride staging and
// reduction over every system's positions.  All sizes and pointers come from
// the device-side table (BatchHeader + SysDesc[]), so one captured CUDA graph
// serves every call whose work fits the allocated capacity.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_sys(const SysDesc *__restrict__ sys, int n_sys, int key, bool by_item)
{
    int lo = 0, hi = n_sys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int v = by_item ? sys[mid].item_begin : sys[mid].pos_begin;
        if (v <= key)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ EvalArgs args_of(const SysDesc &d, const float *boys32, const double *boys64)
{
    EvalArgs a;
    a.n_pos = d.n_pos;
    a.n_splits = d.splits;
    a.n_tiles = d.n_tiles;
    a.tile_size = d.tile_size;
    a.pos = d.st;
    a.tiles = d.tiles;
    a.rec32 = d.rec32;
    a.rec64 = d.rec64;
    a.boys32 = boys32;
    a.boys64 = boys64;
    a.partial = d.partial;
    a.near_r = d.near_r;
    return a;
}

template <int NT, int PPT, int PREC>
__global__ void __launch_bounds__(NT) batch_potential_kernel(const BatchHeader *__restrict__ hdr,
                                                             const SysDesc *__restrict__ sys, int *counter,
                                                             const float *boys32, const double *boys64,
                                                             int tile_cap)
{
    extern __shared__ float4 smem4[];
    __shared__ int s_item;
    float *s_boys = reinterpret_cast<float *>(smem4 + (tile_cap * kRec32MaxStride) / 4);
    if (PREC == 1)
        for (int i = threadIdx.x; i < kBoys32Rows * kBoys32Row; i += NT)
            s_boys[i] = boys32[i];
    const int n_items = hdr->n_items, n_sys = hdr->n_sys;
    for (;;) {
        __syncthreads(); // s_item and the tile buffer are free again
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items)
            break;
        const int k = find_sys(sys, n_sys, item, true);
        const SysDesc &d = sys[k];
        const int local = item - d.item_begin;
        const EvalArgs a = args_of(d, boys32, boys64);
        if (PREC == 1)
            cta_f32c<NT, PPT>(a, local / d.splits, local % d.splits, smem4, s_boys);
        else
            cta_f64<NT, PPT>(a, local / d.splits, local % d.splits, smem4);
    }
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
// reductions
// ---------------------------------------------------------------------------
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

template <typename K>
cudaError_t launch_with_smem(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const EvalArgs &a)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kernel<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

} // namespace

bool potential_shape_supported(int precision, int threads, int ppt)
{
    if (precision == 0)
        return (threads == 64 || threads == 128 || threads == 256) && (ppt == 1 || ppt == 2);
    if (threads == 64)
        return ppt == 2 || ppt == 4;
    if (threads == 128)
        return ppt == 1 || ppt == 2 || ppt == 4;
    return threads == 256 && (ppt == 1 || ppt == 2);
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
    dim3 block(threads);
    size_t smem = potential_smem_bytes(precision, a.tile_size);
#define ESP_LAUNCH(KER, NT, PPT) \
    if (threads == NT && ppt == PPT) return launch_with_smem(KER<NT, PPT>, grid, block, smem, s, a)
    if (precision == 0) {
        ESP_LAUNCH(potential_f64_kernel, 64, 1);
        ESP_LAUNCH(potential_f64_kernel, 64, 2);
        ESP_LAUNCH(potential_f64_kernel, 128, 1);
        ESP_LAUNCH(potential_f64_kernel, 128, 2);
        ESP_LAUNCH(potential_f64_kernel, 256, 1);
        ESP_LAUNCH(potential_f64_kernel, 256, 2);
    } else {
        ESP_LAUNCH(potential_f32c_kernel, 64, 2);
        ESP_LAUNCH(potential_f32c_kernel, 64, 4);
        ESP_LAUNCH(potential_f32c_kernel, 128, 1);
        ESP_LAUNCH(potential_f32c_kernel, 128, 2);
        ESP_LAUNCH(potential_f32c_kernel, 128, 4);
        ESP_LAUNCH(potential_f32c_kernel, 256, 1);
        ESP_LAUNCH(potential_f32c_kernel, 256, 2);
    }
#undef ESP_LAUNCH
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
    dim3 block(threads);
#define ESP_BLAUNCH(NT, PPT, PR)                                                                              \
    if (threads == NT && ppt == PPT && precision == PR) {                                                   \
        auto k = batch_potential_kernel<NT, PPT, PR>;                                                       \
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) \
            return e;                                                                                       \
        int per_sm = 0;                                                                                     \
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess)        \
            return e;                                                                                       \
        int grid = std::max(1, std::min(per_sm * num_sms, max_items));                                      \
        k<<<grid, block, smem, s>>>(hdr, sys, counter, boys32, boys64, tile_cap);                           \
        launched = true;                                                                                    \
    }
    bool launched = false;
    ESP_BLAUNCH(128, 4, 1)
    ESP_BLAUNCH(128, 2, 1)
    ESP_BLAUNCH(256, 2, 1)
    ESP_BLAUNCH(64, 4, 1)
    ESP_BLAUNCH(128, 2, 0)
    ESP_BLAUNCH(128, 1, 0)
    ESP_BLAUNCH(256, 1, 0)
#undef ESP_BLAUNCH
    if (!launched)
        return cudaErrorInvalidConfiguration;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    batch_reduce_kernel<<<sgrid, 256, 0, s>>>(hdr, sys);
    return cudaGetLastError();
}

bool batch_shape_supported(int precision, int threads, int ppt)
{
    if (precision == 1)
        return (threads == 128 && (ppt == 4 || ppt == 2)) || (threads == 256 && ppt == 2) || (threads == 64 && ppt == 4);
    return (threads == 128 && (ppt == 2 || ppt == 1)) || (threads == 256 && ppt == 1);
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
