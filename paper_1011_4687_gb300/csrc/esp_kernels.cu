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
// slot_of (optional): the staged slot of position i (spatial order, below)
__global__ void stage_kernel(const double *__restrict__ pos, int n, double cx, double cy, double cz, double q,
                             Staged st, const int *__restrict__ slot_of)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double x = pos[3 * i] - cx, y = pos[3 * i + 1] - cy, z = pos[3 * i + 2] - cz;
    const int j = slot_of ? slot_of[i] : i;
    st.x64[j] = x;
    st.y64[j] = y;
    st.z64[j] = z;
    // hi words on the environment's coordinate grid q (see the pair builder)
    double xh = nearbyint(x / q) * q, yh = nearbyint(y / q) * q, zh = nearbyint(z / q) * q;
    st.xh[j] = (float)xh;
    st.yh[j] = (float)yh;
    st.zh[j] = (float)zh;
    st.xl[j] = (float)(x - xh);
    st.yl[j] = (float)(y - yh);
    st.zl[j] = (float)(z - zh);
}

// ---------------------------------------------------------------------------
// spatial order of the positions: a stable counting sort by the Morton code
// of their cell in a 16^3 grid over [-8, 8]^3 bohr about the QM centre
// (positions outside share the edge cells).  A warp's positions then sit
// close together, so the warp-uniform far/near votes of the FP32C kernel
// follow the tiles' distance to that small region rather than to the whole
// QM sphere.  Deterministic: ties keep the input order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sort_cell(const double *__restrict__ pos, int i, double cx, double cy, double cz)
{
    const double r[3] = {pos[3 * i] - cx, pos[3 * i + 1] - cy, pos[3 * i + 2] - cz};
    int key = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int c = (int)floor((r[d] + kSortHalf) * (double(kSortSide) / (2.0 * kSortHalf)));
        c = min(max(c, 0), kSortSide - 1);
#pragma unroll
        for (int b = 0; b < 4; ++b)
            key |= ((c >> b) & 1) << (3 * b + d);
    }
    return key;
}

// per-block histogram of the cells of positions [b chunk, (b + 1) chunk)
__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(const double *__restrict__ pos, int n, double cx,
                                                                  double cy, double cz, int chunk,
                                                                  int *__restrict__ counts)
{
    __shared__ int h[kSortCells];
    for (int k = threadIdx.x; k < kSortCells; k += kSortThreads)
        h[k] = 0;
    __syncthreads();
    const int beg = blockIdx.x * chunk, end = min(n, beg + chunk);
    for (int i = beg + threadIdx.x; i < end; i += kSortThreads)
        atomicAdd(&h[sort_cell(pos, i, cx, cy, cz)], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < kSortCells; k += kSortThreads)
        counts[(size_t)k * gridDim.x + blockIdx.x] = h[k];
}

// exclusive scan of counts[cell][block] (cell-major) in place, one CTA
__global__ void __launch_bounds__(1024) sort_scan_kernel(int *__restrict__ counts, int m)
{
    __shared__ int part[1024];
    const int t = threadIdx.x, per = (m + 1023) / 1024;
    const int beg = min(m, t * per), end = min(m, beg + per);
    int s = 0;
    for (int i = beg; i < end; ++i)
        s += counts[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = beg; i < end; ++i) {
        const int c = counts[i];
        counts[i] = run;
        run += c;
    }
}

// stable scatter: slot_of[i] and perm[slot] = i
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const double *__restrict__ pos, int n, double cx,
                                                                    double cy, double cz, int chunk,
                                                                    const int *__restrict__ offs,
                                                                    int *__restrict__ slot_of, int *__restrict__ perm)
{
    __shared__ int run[kSortCells];
    for (int k = threadIdx.x; k < kSortCells; k += kSortThreads)
        run[k] = offs[(size_t)k * gridDim.x + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int beg = blockIdx.x * chunk, end = min(n, beg + chunk);
    for (int base = beg; base < end; base += kSortThreads) {
        const int i = base + threadIdx.x;
        const bool valid = i < end;
        const int key = valid ? sort_cell(pos, i, cx, cy, cz) : -1 - lane; // unique dummy keys
        const unsigned mask = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(mask & lt);
        for (int w = 0; w < kSortThreads / 32; ++w) { // warps in order: ties keep the input order
            if (warp == w) {
                const bool leader = valid && rank == 0;
                int b0 = leader ? run[key] : 0;
                b0 = __shfl_sync(0xffffffffu, b0, __ffs(mask) - 1);
                if (leader)
                    run[key] = b0 + __popc(mask);
                if (valid) {
                    slot_of[i] = b0 + rank;
                    perm[b0 + rank] = i;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void batch_stage_kernel(const BatchHeader *__restrict__ hdr, const SysDesc *__restrict__ sys)
{
    const int total = hdr->n_pos_total, n_sys = hdr->n_sys;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
        const SysDesc &d = sys[find_sys(sys, n_sys, g, false)];
        const int i = g - d.pos_begin;
        double x = d.pos_in[3 * i] - d.qm[0], y = d.pos_in[3 * i + 1] - d.qm[1], z = d.pos_in[3 * i + 2] - d.qm[2];
        const int j = d.sorted ? d.slot_of[i] : i;
        d.st.x64[j] = x;
        d.st.y64[j] = y;
        d.st.z64[j] = z;
        const double q = d.quantum;
        double xh = nearbyint(x / q) * q, yh = nearbyint(y / q) * q, zh = nearbyint(z / q) * q;
        d.st.xh[j] = (float)xh;
        d.st.yh[j] = (float)yh;
        d.st.zh[j] = (float)zh;
        d.st.xl[j] = (float)(x - xh);
        d.st.yl[j] = (float)(y - yh);
        d.st.zl[j] = (float)(z - zh);
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
        d.V_out[d.sorted ? d.perm[i] : i] = s + c;
    }
}

// The spatial order of every sorted system of a batch, one CTA per system
// (histogram, scan and stable scatter as above, all in shared memory).
constexpr int kBatchSortThreads = 1024;

__global__ void __launch_bounds__(kBatchSortThreads) batch_sort_kernel(const BatchHeader *__restrict__ hdr,
                                                                       const SysDesc *__restrict__ sys)
{
    __shared__ int h[kSortCells];
    __shared__ int part[kBatchSortThreads];
    if ((int)blockIdx.x >= hdr->n_sys)
        return;
    const SysDesc &d = sys[blockIdx.x];
    if (!d.sorted)
        return;
    const int n = d.n_pos, t = threadIdx.x;
    for (int k = t; k < kSortCells; k += kBatchSortThreads)
        h[k] = 0;
    __syncthreads();
    for (int i = t; i < n; i += kBatchSortThreads)
        atomicAdd(&h[sort_cell(d.pos_in, i, d.qm[0], d.qm[1], d.qm[2])], 1);
    __syncthreads();
    // exclusive scan: each thread four consecutive cells, then the threads in order
    constexpr int per = kSortCells / kBatchSortThreads;
    int v[per], sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = h[per * t + k];
        sum += v[k];
    }
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < kBatchSortThreads; o <<= 1) {
        const int x = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    int run = part[t] - sum;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        h[per * t + k] = run;
        run += v[k];
    }
    __syncthreads();
    const int lane = t & 31, warp = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < n; base += kBatchSortThreads) {
        const int i = base + t;
        const bool valid = i < n;
        const int key = valid ? sort_cell(d.pos_in, i, d.qm[0], d.qm[1], d.qm[2]) : -1 - lane;
        const unsigned mask = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(mask & lt);
        for (int w = 0; w < kBatchSortThreads / 32; ++w) {
            if (warp == w) {
                const bool leader = valid && rank == 0;
                int b0 = leader ? h[key] : 0;
                b0 = __shfl_sync(0xffffffffu, b0, __ffs(mask) - 1);
                if (leader)
                    h[key] = b0 + __popc(mask);
                if (valid) {
                    d.slot_of[i] = b0 + rank;
                    d.perm[b0 + rank] = i;
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// few positions per call (the paper's call pattern: one r_new per Metropolis
// move).  The roles of the main kernels turn back to the paper's: threads
// take environment entries (cells, point charges, distributions) and evaluate
// them at the positions of their CTA's chunk (up to kSmallChunk of the n <=
// kSmallN positions; grid.y = chunk), the CTA reduces per position in a fixed
// order, and CTA (b, chunk) writes partial[b][q] for its chunk's q.  FP32
// point charges are read in one flat coalesced pass over their contiguous
// records (each once per chunk); the other tiles are dealt round-robin to the
// CTAs of a chunk and read from the FP64 records.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 128;

// (s, c) += (s2, c2) with the rounding error of s + s2 kept in c (TwoSum)
__device__ __forceinline__ void two_sum_pair(float &s, float &c, float s2, float c2)
{
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + e;
}

__global__ void __launch_bounds__(kSmallThreads, 4) small_n_kernel(SmallArgs a)
{
    // grid: x = slice of the environment's entries, y = chunk of kSmallChunk
    // positions; each (slice, position) partial sum is written by one CTA
    __shared__ double s_pos[kSmallChunk][3];
    __shared__ float s_ph[kSmallChunk][3], s_pl[kSmallChunk][3]; // FP32 hi (on the records' grid) and lo words
    __shared__ float s_red32[kSmallThreads / 32][kSmallChunk][2];
    __shared__ double s_red64[kSmallThreads / 32][kSmallChunk];
    const int n = a.n_pos;
    const int q0 = blockIdx.y * kSmallChunk;
    const int nq = min(kSmallChunk, n - q0);
    for (int i = threadIdx.x; i < nq * 3; i += kSmallThreads) {
        const int c = i % 3;
        const double x = a.pos_in[3 * q0 + i] - (c == 0 ? a.cx : c == 1 ? a.cy : a.cz);
        const double h = nearbyint(x / a.quantum) * a.quantum;
        s_pos[i / 3][c] = x;
        s_ph[i / 3][c] = float(h);
        s_pl[i / 3][c] = float(x - h);
    }
    // does this CTA evaluate any entry in FP64?  (then its FP64 sums need a
    // FP64 reduction; FP64 instructions run at 1/64 of the FP32 rate here)
    bool has64 = false;
    for (int t = blockIdx.x; t < a.n_tiles && !has64; t += gridDim.x)
        has64 = !(a.tiles[t].cls == kClassPoint32 && a.fp32);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gtid = blockIdx.x * kSmallThreads + threadIdx.x, gthreads = gridDim.x * kSmallThreads;
    float acc32[kSmallChunk];
    double acc[kSmallChunk];
#pragma unroll
    for (int q = 0; q < kSmallChunk; ++q) {
        acc32[q] = 0.0f;
        acc[q] = 0.0;
    }
    // FP32 point charges: one flat, coalesced pass over their contiguous
    // records (thread g takes entries g, g + G, ...: the paper's coalesced
    // mapping); a thread's few terms sum in FP32
    if (a.fp32 && a.n_p32 > 0) {
        for (int e = gtid; e < a.n_p32; e += gthreads) {
            const float *r = a.rec32 + a.p32_off + (size_t)e * rec32_stride(0);
            const float4 r0 = reinterpret_cast<const float4 *>(r)[0];
            const float4 r1 = reinterpret_cast<const float4 *>(r)[1];
            const float qh = r[rec32_m(0)], ql = r1.w;
#pragma unroll
            for (int q = 0; q < kSmallChunk; ++q) {
                if (q >= nq)
                    break;
                const float dx = (r0.x - s_ph[q][0]) + (r1.x - s_pl[q][0]);
                const float dy = (r0.y - s_ph[q][1]) + (r1.y - s_pl[q][1]);
                const float dz = (r0.z - s_ph[q][2]) + (r1.z - s_pl[q][2]);
                const float rs = esp_rsqrt(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                acc32[q] += fmaf(qh, rs, ql * rs);
            }
        }
    }
    // every other tile (FP64 points, distributions; FP32 points under FP64),
    // dealt round-robin to the CTAs, one entry per thread
    if (has64) {
        for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
            const TileMeta m = a.tiles[t];
            if (m.cls == kClassPoint32 && a.fp32)
                continue;
            const bool pts = is_point_class(m.cls);
            const int st = pts ? kPointStride64 : rec64_stride(m.cls & 7);
            for (int j = threadIdx.x; j < m.n; j += kSmallThreads) {
                const double *r = a.rec64 + m.off64 + (size_t)j * st;
#pragma unroll
                for (int q = 0; q < kSmallChunk; ++q) {
                    if (q >= nq)
                        break;
                        if (pts) {
                        const double dx = r[0] - s_pos[q][0], dy = r[1] - s_pos[q][1], dz = r[2] - s_pos[q][2];
                        acc[q] += r[3] * esp_rsqrt(dx * dx + dy * dy + dz * dz);
                    } else {
                        acc[q] += tile_f64_one_any(m.cls, r, 1, s_pos[q][0], s_pos[q][1], s_pos[q][2],
                                                   a.boys64);
                    }
                }
            }
        }
    }
    // fixed-order reduction per position: the FP32 sums as (sum,
    // compensation) pairs by warp shuffles, the FP64 sums (only where this
    // CTA has any) likewise in FP64, then the warps in order in FP64
#pragma unroll
    for (int q = 0; q < kSmallChunk; ++q) {
        if (q >= nq)
            break;
        float sv = acc32[q], cv = 0.0f;
        for (int o = 16; o; o >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, sv, o), co = __shfl_xor_sync(0xffffffffu, cv, o);
            two_sum_pair(sv, cv, so, co);
        }
        double v = 0.0;
        if (has64) {
            v = acc[q];
            for (int o = 16; o; o >>= 1)
                v += __shfl_xor_sync(0xffffffffu, v, o);
        }
        if (lane == 0) {
            s_red32[warp][q][0] = sv;
            s_red32[warp][q][1] = cv;
            s_red64[warp][q] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        double v = 0.0;
        for (int w = 0; w < kSmallThreads / 32; ++w)
            v += (double(s_red32[w][threadIdx.x][0]) + double(s_red32[w][threadIdx.x][1])) +
                 s_red64[w][threadIdx.x];
        a.partial[(size_t)blockIdx.x * n + q0 + threadIdx.x] = v;
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

// perm (optional): the input index of staged slot i
__global__ void reduce_kernel(const double *__restrict__ partial, int n_splits, int n, double *__restrict__ V,
                              const int *__restrict__ perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double s = 0.0, c = 0.0;
    for (int k = 0; k < n_splits; ++k)
        two_sum_acc(s, c, partial[(size_t)k * n + i]);
    V[perm ? perm[i] : i] = s + c;
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
                         cudaStream_t s, const int *slot_of)
{
    if (n <= 0)
        return cudaSuccess;
    stage_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos_in, n, center[0], center[1], center[2], quantum, st, slot_of);
    return cudaGetLastError();
}

int sort_blocks(int n) { return std::max(1, std::min(256, (n + 2047) / 2048)); }

size_t sort_scratch_ints(int n) { return (size_t)kSortCells * sort_blocks(n) + 2 * (size_t)n; }

cudaError_t launch_sort(const double *pos_in, int n, const double center[3], int *scratch, int **slot_of, int **perm,
                        cudaStream_t s)
{
    const int B = sort_blocks(n), chunk = (n + B - 1) / B;
    int *counts = scratch;
    *slot_of = scratch + (size_t)kSortCells * B;
    *perm = *slot_of + n;
    sort_count_kernel<<<B, kSortThreads, 0, s>>>(pos_in, n, center[0], center[1], center[2], chunk, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    sort_scan_kernel<<<1, 1024, 0, s>>>(counts, kSortCells * B);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    sort_scatter_kernel<<<B, kSortThreads, 0, s>>>(pos_in, n, center[0], center[1], center[2], chunk, counts, *slot_of,
                                                   *perm);
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

cudaError_t launch_batch(int precision, const BatchHeader *hdr, const SysDesc *sys, int max_sys, int *counter,
                         int max_items, const float *boys32, const double *boys64, int tile_cap, int threads, int ppt,
                         int num_sms, int max_pos_total, cudaStream_t s)
{
    const int sgrid = std::max(1, std::min(4 * num_sms, (max_pos_total + 255) / 256));
    batch_sort_kernel<<<std::max(1, max_sys), kBatchSortThreads, 0, s>>>(hdr, sys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    batch_stage_kernel<<<sgrid, 256, 0, s>>>(hdr, sys);
    e = cudaGetLastError();
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

// Slices of the environment's entries: about 8 CTAs per SM over all chunks of
// positions, so that with more positions each thread takes more entries and
// the per-position reduction is amortised over more terms.
int small_n_splits(int n_tiles, int num_sms, int n)
{
    const int chunks = std::max(1, (n + kSmallChunk - 1) / kSmallChunk);
    return std::max(1, std::min(n_tiles, 8 * num_sms / chunks));
}

cudaError_t launch_small_n(const SmallArgs &a, int n_splits, double *V, cudaStream_t s)
{
    if (a.n_pos <= 0 || a.n_pos > kSmallN)
        return cudaErrorInvalidValue;
    const dim3 grid(n_splits, (a.n_pos + kSmallChunk - 1) / kSmallChunk);
    small_n_kernel<<<grid, kSmallThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    reduce_wide_kernel<<<a.n_pos, kWideThreads, 0, s>>>(a.partial, n_splits, a.n_pos, V);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partial, int n_splits, int n, double *V, cudaStream_t s, const int *perm)
{
    if (n <= 0)
        return cudaSuccess;
    reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, n_splits, n, V, perm);
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
