// The paper's coalescing study on this GPU.
//
// The paper's kernel (Sec. III, Eq. blockSum) sums the cell potentials
// rho(r_m)/|r_new - r_m| of one position over N_B blocks of N_th threads,
// each thread running N_loop iterations.  Its Results (Eq. coalease vs Eq.
// incoalease, Table Single Core performances) compare two mappings of
// (block b, thread j, iteration l) to a cell index m:
//   coalesced:   m = l N_B N_th + b N_th + j   (neighbouring threads read
//                neighbouring cells in every iteration);
//   incoalesced: m = (b N_th + j) N_loop + l   (each thread walks its own
//                contiguous chunk of cells);
// and find the coalesced one 6.0x faster in the kernel.  This file runs both
// mappings over the context's point charges, either as the library stores
// them (records [x, y, z, Z] of 32 bytes, one sector per cell) or as separate
// coordinate and charge arrays (SoA: one 8-byte FP64 or 4-byte FP32 word per
// cell and array, the layout in which neighbouring threads share sectors), in
// FP64 or FP32 arithmetic with FP64 per-thread sums, with the paper's block
// reduction in shared memory and a fixed-order final sum, and times them with
// CUDA events.  It is a study of the memory mapping, not an evaluation path.
#include <cuda_runtime.h>

#include "../../include/esp.h"
#include "esp_ctx.h"

using namespace esp;

namespace {

constexpr int kStudyThreads = 256; // the paper's N_th

// SoA arrays of the study: x, y, z, q as FP64 (soa64) and FP32 (soa32) copies
struct Soa {
    const double *x64, *y64, *z64, *q64;
    const float *x32, *y32, *z32, *q32;
};

template <bool CONTIG, bool FP64, bool SOA>
__global__ void __launch_bounds__(kStudyThreads) cell_sum_kernel(const double4 *__restrict__ pts, Soa soa,
                                                                 int m_total, int n_loop, double cx, double cy,
                                                                 double cz, double *__restrict__ partial)
{
    __shared__ double s_red[kStudyThreads];
    const int j = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    double acc = 0.0;
    for (int l = 0; l < n_loop; ++l) {
        const long long m = CONTIG ? (long long)(b * kStudyThreads + j) * n_loop + l
                                   : (long long)l * nb * kStudyThreads + b * kStudyThreads + j;
        if (m >= m_total)
            continue;
        if constexpr (FP64) {
            double x, y, z, q;
            if constexpr (SOA) {
                x = soa.x64[m], y = soa.y64[m], z = soa.z64[m], q = soa.q64[m];
            } else {
                const double4 r = pts[m];
                x = r.x, y = r.y, z = r.z, q = r.w;
            }
            const double dx = x - cx, dy = y - cy, dz = z - cz;
            acc += q * rsqrt(dx * dx + dy * dy + dz * dz);
        } else {
            float dx, dy, dz, q;
            if constexpr (SOA) {
                dx = soa.x32[m] - float(cx), dy = soa.y32[m] - float(cy), dz = soa.z32[m] - float(cz), q = soa.q32[m];
            } else {
                const double4 r = pts[m];
                dx = float(r.x - cx), dy = float(r.y - cy), dz = float(r.z - cz), q = float(r.w);
            }
            acc += double(q * rsqrtf(dx * dx + dy * dy + dz * dz));
        }
    }
    // the paper's per-block reduction in shared memory (fixed order)
    s_red[j] = acc;
    __syncthreads();
    for (int o = kStudyThreads / 2; o > 0; o >>= 1) {
        if (j < o)
            s_red[j] += s_red[j + o];
        __syncthreads();
    }
    if (j == 0)
        partial[b] = s_red[0];
}

__global__ void study_final_kernel(const double *__restrict__ partial, int nb, double *__restrict__ V)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b)
            s += partial[b];
        *V = s;
    }
}

__global__ void soa_split_kernel(const double4 *__restrict__ pts, int m, double *x64, double *y64, double *z64,
                                 double *q64, float *x32, float *y32, float *z32, float *q32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m)
        return;
    const double4 r = pts[i];
    x64[i] = r.x, y64[i] = r.y, z64[i] = r.z, q64[i] = r.w;
    x32[i] = float(r.x), y32[i] = float(r.y), z32[i] = float(r.z), q32[i] = float(r.w);
}

template <bool CONTIG, bool FP64, bool SOA>
cudaError_t launch_study(const double4 *pts, const Soa &soa, int m, int n_loop, const double c[3], double *partial,
                         double *V, cudaStream_t s)
{
    const int nb = (m + kStudyThreads * n_loop - 1) / (kStudyThreads * n_loop);
    cell_sum_kernel<CONTIG, FP64, SOA><<<nb, kStudyThreads, 0, s>>>(pts, soa, m, n_loop, c[0], c[1], c[2], partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    study_final_kernel<<<1, 32, 0, s>>>(partial, nb, V);
    return cudaGetLastError();
}

} // namespace

extern "C" esp_status esp_study_cell_sum(esp_ctx *ctx, const double *position, int32_t incoalesced, int32_t fp64,
                                         int32_t soa_layout, int32_t n_loop, int32_t reps, double *V_out,
                                         double *ms_out)
{
    last_error().clear();
    if (!valid_ctx(ctx) || ctx->device < 0)
        return fail(ESP_ERR_STATE, "invalid or host-only context");
    if (!position || !V_out || n_loop < 1 || n_loop > 4096 || reps < 1 || reps > 100000)
        return fail(ESP_ERR_INVALID, "bad study arguments");
    // the point records lead rec64 (point tiles precede distribution tiles)
    int64_t m = 0;
    for (const TileMeta &t : ctx->env.tiles)
        if (is_point_class(t.cls))
            m += t.n;
    if (m == 0)
        return fail(ESP_ERR_UNSUPPORTED, "the environment has no point charges");
    BusyGuard busy(ctx->busy);
    if (!busy.acquired)
        return fail(ESP_ERR_STATE, "context is in use by another thread");
    DeviceGuard dg(ctx->device);
    const double c[3] = {position[0] - ctx->opt.qm_center[0], position[1] - ctx->opt.qm_center[1],
                         position[2] - ctx->opt.qm_center[2]};
    const int nb = int((m + int64_t(kStudyThreads) * n_loop - 1) / (int64_t(kStudyThreads) * n_loop));
    DevBuf part, dv, soa_buf;
    cudaError_t e = part.ensure(size_t(nb) * sizeof(double));
    if (e == cudaSuccess)
        e = dv.ensure(sizeof(double));
    if (e == cudaSuccess && soa_layout)
        e = soa_buf.ensure(size_t(m) * (4 * sizeof(double) + 4 * sizeof(float)));
    if (e != cudaSuccess)
        return cuda_fail(e, "allocating study buffers");
    const double4 *pts = static_cast<const double4 *>(ctx->rec64.p);
    double *P = static_cast<double *>(part.p), *Vd = static_cast<double *>(dv.p);
    cudaStream_t s = ctx->stream;
    Soa soa{};
    if (soa_layout) {
        double *d64 = static_cast<double *>(soa_buf.p);
        float *f32 = reinterpret_cast<float *>(d64 + 4 * m);
        soa = Soa{d64, d64 + m, d64 + 2 * m, d64 + 3 * m, f32, f32 + m, f32 + 2 * m, f32 + 3 * m};
        soa_split_kernel<<<int((m + 255) / 256), 256, 0, s>>>(pts, int(m), d64, d64 + m, d64 + 2 * m, d64 + 3 * m, f32,
                                                               f32 + m, f32 + 2 * m, f32 + 3 * m);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return cuda_fail(e, "building the SoA copy");
    }
    auto run = [&]() {
#define ESP_STUDY(C, F, S) launch_study<C, F, S>(pts, soa, int(m), n_loop, c, P, Vd, s)
        if (soa_layout) {
            if (incoalesced)
                return fp64 ? ESP_STUDY(true, true, true) : ESP_STUDY(true, false, true);
            return fp64 ? ESP_STUDY(false, true, true) : ESP_STUDY(false, false, true);
        }
        if (incoalesced)
            return fp64 ? ESP_STUDY(true, true, false) : ESP_STUDY(true, false, false);
        return fp64 ? ESP_STUDY(false, true, false) : ESP_STUDY(false, false, false);
#undef ESP_STUDY
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return cuda_fail(e, "creating study events");
    e = run(); // warm-up
    if (e == cudaSuccess)
        e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = run();
    if (e == cudaSuccess)
        e = cudaEventRecord(e1, s);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    double v = 0.0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&v, Vd, sizeof(double), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return cuda_fail(e, "running the coalescing study");
    *V_out = v;
    if (ms_out)
        *ms_out = double(ms) / reps;
    return ESP_OK;
}
