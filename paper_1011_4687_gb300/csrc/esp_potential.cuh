// Potential kernel templates (FP32C, FP64, batched persistent) for sm_103a.
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
//
// Only esp_shape.cu instantiates these templates, once per launch shape and
// object file (the shape lists are in esp_shapes.h), so that the shapes
// compile in parallel.
#pragma once

#include "esp_eval_core.h"
#include "esp_kernels.h"

namespace esp {

namespace {

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
    // the same positions as lane pairs (used when PPT is even)
    constexpr int NP = PPT / 2 > 0 ? PPT / 2 : 1;
    f2 ch2[NP][3], cl2[NP][3], S2[NP], C2[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int q0 = 2 * q < PPT ? 2 * q : 0, q1 = 2 * q + 1 < PPT ? 2 * q + 1 : 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ch2[q][d] = f2(ch[q0][d], ch[q1][d]);
            cl2[q][d] = f2(cl[q0][d], cl[q1][d]);
        }
        S2[q] = f2(0.0f);
        C2[q] = f2(0.0f);
    }
    const float near_r = a.near_r;
    // this split's group and its place among the group's splits
    int g = 0;
    while (g + 1 < a.n_groups && split >= a.grp_split[g + 1])
        ++g;
    const int g_stride = a.grp_split[g + 1] - a.grp_split[g];
    const int g_end = a.grp_tile[g + 1];
    for (int t = a.grp_tile[g] + (split - a.grp_split[g]); t < g_end; t += g_stride) {
        const TileMeta m = a.tiles[t];
        __syncthreads(); // previous tile fully consumed
        const bool pts = m.cls == kClassPoint;
        const float4 *src = pts ? reinterpret_cast<const float4 *>(a.rec64 + m.off64)
                                : reinterpret_cast<const float4 *>(a.rec32 + m.off32);
        const int nvec = pts ? m.n * 2 : (m.n * rec32_stride_cls(m.cls)) / 4;
        copy_tile(s_tile4, src, nvec);
        __syncthreads();
        if (m.cls == kClassPoint32) {
            // small point charges: the far form of an L = 0 record, no near path
            const float *s_rec = reinterpret_cast<const float *>(s_tile4);
            // (absolute hi words: th = 0 - C_hi, the exact offset form)
            if constexpr (PPT % 2 == 0) {
                f2 wq[NP], th2[NP][3];
#pragma unroll
                for (int q = 0; q < NP; ++q)
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        th2[q][d] = f2(0.0f) - ch2[q][d];
                tile_f32c2<0, NP, true, false, false>(s_rec, m.n, th2, cl2, cl2, wq, S2, C2, s_boys);
            } else {
                bool none[PPT];
                float th[PPT][3];
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    none[q] = false;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        th[q][d] = 0.0f - ch[q][d];
                }
                tile_f32c<0, PPT, true, false, false>(s_rec, m.n, th, cl, cl, none, S, Cc, s_boys);
            }
            continue;
        }
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
        bool any_near = false, lane_far = true, lane_rel = true;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            bool f, r;
            classify_tile(m, ch[q][0], ch[q][1], ch[q][2], near_r, nearq[q], f, r);
            any_near |= nearq[q];
            lane_far &= f;
            lane_rel &= r;
        }
        const bool far = __all_sync(0xffffffffu, lane_far);
        const bool rel = __all_sync(0xffffffffu, lane_rel); // implies far
        const bool sel = __any_sync(0xffffffffu, any_near); // warp-uniform: any term to select away
        const float *s_rec = reinterpret_cast<const float *>(s_tile4);
        const float ct[3] = {m.cx, m.cy, m.cz}; // the records' reference point T
        if constexpr (PPT % 2 == 0) {
            // two positions per packed FP32 instruction
            f2 wq[NP], th2[NP][3], dq2[NP][3];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                wq[q] = f2(nearq[2 * q] ? 0.0f : 1.0f, nearq[2 * q + 1] ? 0.0f : 1.0f);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    th2[q][d] = f2(ct[d]) - ch2[q][d];
                    dq2[q][d] = th2[q][d] - cl2[q][d];
                }
            }
#define ESP_TILE(CLS, LL, SH)                                                                         \
    case CLS:                                                                                         \
        if (rel && !sel)                                                                              \
            tile_f32c2<LL, NP, true, SH, false, true>(s_rec, m.n, th2, cl2, dq2, wq, S2, C2, s_boys); \
        else if (far && !sel)                                                                         \
            tile_f32c2<LL, NP, true, SH, false>(s_rec, m.n, th2, cl2, dq2, wq, S2, C2, s_boys);       \
        else if (far)                                                                                 \
            tile_f32c2<LL, NP, true, SH, true>(s_rec, m.n, th2, cl2, dq2, wq, S2, C2, s_boys);        \
        else                                                                                          \
            tile_f32c2<LL, NP, false, SH, true>(s_rec, m.n, th2, cl2, dq2, wq, S2, C2, s_boys);       \
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
        } else {
            float th[PPT][3], dq[PPT][3];
#pragma unroll
            for (int q = 0; q < PPT; ++q)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    th[q][d] = ct[d] - ch[q][d];
                    dq[q][d] = th[q][d] - cl[q][d];
                }
#define ESP_TILE(CLS, LL, SH)                                                                         \
    case CLS:                                                                                         \
        if (rel && !sel)                                                                              \
            tile_f32c<LL, PPT, true, SH, false, true>(s_rec, m.n, th, cl, dq, nearq, S, Cc, s_boys);  \
        else if (far && !sel)                                                                         \
            tile_f32c<LL, PPT, true, SH, false>(s_rec, m.n, th, cl, dq, nearq, S, Cc, s_boys);        \
        else if (far)                                                                                 \
            tile_f32c<LL, PPT, true, SH, true>(s_rec, m.n, th, cl, dq, nearq, S, Cc, s_boys);         \
        else                                                                                          \
            tile_f32c<LL, PPT, false, SH, true>(s_rec, m.n, th, cl, dq, nearq, S, Cc, s_boys);        \
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
        }
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
    if constexpr (PPT % 2 == 0) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            S[2 * q] = S2[q].x;
            S[2 * q + 1] = S2[q].y;
            Cc[2 * q] = C2[q].x;
            Cc[2 * q + 1] = C2[q].y;
        }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q)
        if (idx[q] < a.n_pos)
            a.partial[(size_t)split * a.n_pos + idx[q]] = ((double)S[q] + (double)Cc[q]) + acc64[q];
}

template <int NT, int PPT>
__global__ void __launch_bounds__(NT, 512 / NT) potential_f32c_kernel(EvalArgs a)
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
        const bool pts = is_point_class(m.cls);
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
    single_group(a);
    return a;
}

template <int NT, int PPT, int PREC>
__global__ void __launch_bounds__(NT, PREC == 1 ? 512 / NT : 1) batch_potential_kernel(const BatchHeader *__restrict__ hdr,
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

} // namespace

} // namespace esp
