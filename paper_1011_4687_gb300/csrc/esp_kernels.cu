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
#include "esp_kernels.h"

namespace esp {

namespace {

// ---------------------------------------------------------------------------
// staging: recentre in FP64, split into FP32 hi + lo
// ---------------------------------------------------------------------------
__global__ void stage_kernel(const double *__restrict__ pos, int n, double cx, double cy, double cz, Staged st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double x = pos[3 * i] - cx, y = pos[3 * i + 1] - cy, z = pos[3 * i + 2] - cz;
    st.x64[i] = x;
    st.y64[i] = y;
    st.z64[i] = z;
    float xh = (float)x, yh = (float)y, zh = (float)z;
    st.xh[i] = xh;
    st.yh[i] = yh;
    st.zh[i] = zh;
    st.xl[i] = (float)(x - (double)xh);
    st.yl[i] = (float)(y - (double)yh);
    st.zl[i] = (float)(z - (double)zh);
}

// error-free a + b = s + e (Knuth TwoSum)
__device__ __forceinline__ void two_sum_acc(float &S, float &C, float x)
{
    float s = S + x;
    float bp = s - S;
    float e = (S - (s - bp)) + (x - bp);
    S = s;
    C += e;
}

__device__ __forceinline__ void two_sum_acc(double &S, double &C, double x)
{
    double s = S + x;
    double bp = s - S;
    double e = (S - (s - bp)) + (x - bp);
    S = s;
    C += e;
}

// one distribution at one position, FP64
template <int L>
__device__ __forceinline__ double dist_f64(const double *__restrict__ r, double cx, double cy, double cz,
                                           const double *__restrict__ boys64)
{
    double dx = r[0] - cx, dy = r[1] - cy, dz = r[2] - cz;
    double sp = r[3];
    double F[L + 1];
    if constexpr (L == 0) {
        double T = (sp * sp) * (dx * dx + dy * dy + dz * dz);
        boys_eval<L, double>(T, boys64, F);
        return r[4] * F[0];
    } else {
        double x = sp * dx, y = sp * dy, z = sp * dz;
        double T = x * x + y * y + z * z;
        boys_eval<L, double>(T, boys64, F);
        return hermite_contract<L, double>(F, x, y, z, r + 4);
    }
}

// whole tile at one position, FP64, records read from global memory
template <int L>
__device__ __noinline__ double tile_f64_global(const double *__restrict__ rec, int n, double cx, double cy,
                                               double cz, const double *__restrict__ boys64)
{
    constexpr int st = rec64_stride(L);
    double acc = 0.0;
    for (int j = 0; j < n; ++j)
        acc += dist_f64<L>(rec + j * st, cx, cy, cz, boys64);
    return acc;
}

__device__ double tile_f64_global_any(int L, const double *rec, int n, double cx, double cy, double cz,
                                      const double *boys64)
{
    switch (L) {
    case 0: return tile_f64_global<0>(rec, n, cx, cy, cz, boys64);
    case 1: return tile_f64_global<1>(rec, n, cx, cy, cz, boys64);
    case 2: return tile_f64_global<2>(rec, n, cx, cy, cz, boys64);
    case 3: return tile_f64_global<3>(rec, n, cx, cy, cz, boys64);
    default: return tile_f64_global<4>(rec, n, cx, cy, cz, boys64);
    }
}

// ---------------------------------------------------------------------------
// FP32-compensated tile: 16-term FP32 blocks, TwoSum of each block into a
// running (S, C) pair per position; near positions skip FP32 and are
// re-evaluated in FP64 afterwards.
// ---------------------------------------------------------------------------
template <int L, int PPT>
__device__ __forceinline__ void tile_f32c(const float *__restrict__ s_rec, int n, const float (&ch)[PPT][3],
                                          const float (&cl)[PPT][3], const bool (&nearq)[PPT],
                                          float (&S)[PPT], float (&Cc)[PPT], const float *__restrict__ s_boys)
{
    constexpr int st = rec32_stride(L);
    constexpr int nh = num_hermite(L);
    for (int j0 = 0; j0 < n; j0 += 16) {
        float blk[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            blk[q] = 0.0f;
        const int j1 = min(j0 + 16, n);
        for (int j = j0; j < j1; ++j) {
            const float *r = s_rec + j * st;
            const float4 r0 = *reinterpret_cast<const float4 *>(r);
            float G[nh];
#pragma unroll
            for (int h = 0; h < nh; ++h)
                G[h] = r[4 + h];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                float dx = (r0.x - ch[q][0]) - cl[q][0];
                float dy = (r0.y - ch[q][1]) - cl[q][1];
                float dz = (r0.z - ch[q][2]) - cl[q][2];
                float v;
                float F[L + 1];
                if constexpr (L == 0) {
                    float T = r0.w * (dx * dx + dy * dy + dz * dz);
                    boys_eval<L, float>(T, s_boys, F);
                    v = G[0] * F[0];
                } else {
                    float x = r0.w * dx, y = r0.w * dy, z = r0.w * dz;
                    float T = x * x + y * y + z * z;
                    boys_eval<L, float>(T, s_boys, F);
                    v = hermite_contract<L, float>(F, x, y, z, G);
                }
                blk[q] += nearq[q] ? 0.0f : v;
            }
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            two_sum_acc(S[q], Cc[q], blk[q]);
    }
}

template <int PPT>
__device__ __forceinline__ void tile_points_f64(const double *__restrict__ s_pts, int n, const double (&c64)[PPT][3],
                                                double (&acc)[PPT])
{
    for (int j = 0; j < n; ++j) {
        const double2 a = *reinterpret_cast<const double2 *>(s_pts + 4 * j);
        const double2 b = *reinterpret_cast<const double2 *>(s_pts + 4 * j + 2);
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            double dx = a.x - c64[q][0], dy = a.y - c64[q][1], dz = b.x - c64[q][2];
            acc[q] += b.y * rsqrt(dx * dx + dy * dy + dz * dz);
        }
    }
}

__device__ __forceinline__ void copy_tile(float4 *__restrict__ dst, const float4 *__restrict__ src, int nvec)
{
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
        dst[i] = __ldg(src + i);
}

// ---------------------------------------------------------------------------
// FP32C kernel
// ---------------------------------------------------------------------------
template <int NT, int PPT>
__global__ void __launch_bounds__(NT) potential_f32c_kernel(EvalArgs a)
{
    extern __shared__ float4 smem4[];
    float4 *s_tile4 = smem4;
    float *s_boys = reinterpret_cast<float *>(smem4 + (a.tile_size * 40) / 4);
    for (int i = threadIdx.x; i < kBoys32Rows * kBoys32Row; i += NT)
        s_boys[i] = a.boys32[i];

    const int split = blockIdx.y;
    const int base = blockIdx.x * NT * PPT + threadIdx.x;
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
    const float near2 = a.near_r;
    for (int t = split; t < a.n_tiles; t += a.n_splits) {
        const TileMeta m = a.tiles[t];
        __syncthreads(); // previous tile fully consumed
        const bool pts = m.cls == kClassPoint;
        const float4 *src = pts ? reinterpret_cast<const float4 *>(a.rec64 + m.off64)
                                : reinterpret_cast<const float4 *>(a.rec32 + m.off32);
        const int nvec = pts ? m.n * 2 : (m.n * rec32_stride(m.cls)) / 4;
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
        bool any_near = false;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            float ex = ch[q][0] - m.cx, ey = ch[q][1] - m.cy, ez = ch[q][2] - m.cz;
            float d = sqrtf(ex * ex + ey * ey + ez * ez) - m.rad;
            nearq[q] = d < near2;
            any_near |= nearq[q];
        }
        const float *s_rec = reinterpret_cast<const float *>(s_tile4);
        switch (m.cls) {
        case 0: tile_f32c<0, PPT>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys); break;
        case 1: tile_f32c<1, PPT>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys); break;
        case 2: tile_f32c<2, PPT>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys); break;
        case 3: tile_f32c<3, PPT>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys); break;
        default: tile_f32c<4, PPT>(s_rec, m.n, ch, cl, nearq, S, Cc, s_boys); break;
        }
        if (any_near) {
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (nearq[q]) {
                    int ic = min(idx[q], a.n_pos - 1);
                    acc64[q] += tile_f64_global_any(m.cls, a.rec64 + m.off64, m.n, a.pos.x64[ic], a.pos.y64[ic],
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

// ---------------------------------------------------------------------------
// FP64 kernel
// ---------------------------------------------------------------------------
template <int L, int PPT>
__device__ __forceinline__ void tile_f64(const double *__restrict__ s_rec, int n, const double (&c)[PPT][3],
                                         double (&tacc)[PPT], const double *__restrict__ boys64)
{
    constexpr int st = rec64_stride(L);
    for (int j = 0; j < n; ++j) {
        const double *r = s_rec + j * st;
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            tacc[q] += dist_f64<L>(r, c[q][0], c[q][1], c[q][2], boys64);
    }
}

template <int NT, int PPT>
__global__ void __launch_bounds__(NT) potential_f64_kernel(EvalArgs a)
{
    extern __shared__ float4 smem4[];
    const double *s_rec = reinterpret_cast<const double *>(smem4);
    const int split = blockIdx.y;
    const int base = blockIdx.x * NT * PPT + threadIdx.x;
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
        const int nvec = pts ? m.n * 2 : (m.n * rec64_stride(m.cls)) / 2;
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
            case 0: tile_f64<0, PPT>(s_rec, m.n, c, tacc, a.boys64); break;
            case 1: tile_f64<1, PPT>(s_rec, m.n, c, tacc, a.boys64); break;
            case 2: tile_f64<2, PPT>(s_rec, m.n, c, tacc, a.boys64); break;
            case 3: tile_f64<3, PPT>(s_rec, m.n, c, tacc, a.boys64); break;
            default: tile_f64<4, PPT>(s_rec, m.n, c, tacc, a.boys64); break;
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

size_t potential_smem_bytes(int precision, int tile_size)
{
    if (precision == 0)
        return (size_t)tile_size * 40 * sizeof(double);
    return (size_t)tile_size * 40 * sizeof(float) + (size_t)kBoys32Rows * kBoys32Row * sizeof(float);
}

cudaError_t launch_stage(const double *pos_in, int n, const double center[3], const Staged &st, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    stage_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos_in, n, center[0], center[1], center[2], st);
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
        ESP_LAUNCH(potential_f64_kernel, 128, 1);
        ESP_LAUNCH(potential_f64_kernel, 128, 2);
        ESP_LAUNCH(potential_f64_kernel, 256, 1);
        ESP_LAUNCH(potential_f64_kernel, 64, 2);
    } else {
        ESP_LAUNCH(potential_f32c_kernel, 128, 1);
        ESP_LAUNCH(potential_f32c_kernel, 128, 2);
        ESP_LAUNCH(potential_f32c_kernel, 128, 4);
        ESP_LAUNCH(potential_f32c_kernel, 256, 2);
        ESP_LAUNCH(potential_f32c_kernel, 64, 4);
    }
#undef ESP_LAUNCH
    return cudaErrorInvalidConfiguration;
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
