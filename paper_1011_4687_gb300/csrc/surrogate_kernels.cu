// Kernels of the learned surrogate of V(r) over the QM region.
//
// Network: Fourier features gamma(u) = [sin(2 pi B u), cos(2 pi B u)] of the
// position u = (r - centre) / R (32 frequencies, 64 features), four hidden
// layers of 256 with SiLU, one linear output.  BF16 weights and activations,
// FP32 accumulation on the tcgen05 tensor cores (training GEMMs in
// surrogate_gemm.cu, fused inference in surrogate_tc.cu), FP32 master weights
// updated by Adam.  The network models the residual of the far
// environment's potential after its FP64 interior solid-harmonic expansion
// (esp_harmonics.h), so that its BF16 output only carries a small correction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "esp_harmonics.h"
#include "surrogate_kernels.h"

namespace esp {
namespace sur {

namespace {

__device__ __forceinline__ float silu_grad(float z)
{
    float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__global__ void features_kernel(const double *__restrict__ pos, int n, const float *__restrict__ freq, double cx,
                                double cy, double cz, double inv_r, __nv_bfloat16 *__restrict__ X)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float ux = float((pos[3 * i] - cx) * inv_r), uy = float((pos[3 * i + 1] - cy) * inv_r),
                uz = float((pos[3 * i + 2] - cz) * inv_r);
#pragma unroll 4
    for (int f = 0; f < kFreq; ++f) {
        float ph = 6.283185307179586f * (freq[3 * f] * ux + freq[3 * f + 1] * uy + freq[3 * f + 2] * uz);
        float s, c;
        __sincosf(ph, &s, &c);
        X[(size_t)i * kFeat + f] = __float2bfloat16(s);
        X[(size_t)i * kFeat + kFreq + f] = __float2bfloat16(c);
    }
}

// y[i] = sum_k H[i][k] w[k] + b; with targets: dy = 2 (y - t) / n, loss partial.
__global__ void output_kernel(const __nv_bfloat16 *__restrict__ H, int n, const float *__restrict__ w,
                              const float *__restrict__ bptr,
                              float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                              float *__restrict__ loss_part)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    float l = 0.0f;
    if (warp < n) {
        float s = 0.0f;
        for (int k = lane; k < kHidden; k += 32)
            s += __bfloat162float(H[(size_t)warp * kHidden + k]) * w[k];
        for (int o = 16; o; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        s += *bptr;
        if (lane == 0) {
            y[warp] = s;
            if (t) {
                float r = s - t[warp];
                dy[warp] = 2.0f * r / float(n);
                l = r * r;
            }
        }
    }
    if (loss_part && lane == 0 && warp < n)
        loss_part[warp] = l;
}

// dZ4[i][k] = dy[i] w[k] SiLU'(Z4[i][k]) (bf16); gradient of the output layer
// parameters is accumulated by out_grad_kernel.
__global__ void out_back_kernel(const float *__restrict__ dy, int n, const float *__restrict__ w,
                                const float *__restrict__ Z, __nv_bfloat16 *__restrict__ dZ)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * kHidden)
        return;
    const int i = int(e / kHidden), k = int(e % kHidden);
    dZ[e] = __float2bfloat16(dy[i] * w[k] * silu_grad(Z[e]));
}

// per-block partials of dw[k] = sum_i dy[i] H[i][k] and db = sum_i dy[i]
__global__ void out_grad_kernel(const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ H, int n, int rows,
                                float *__restrict__ part)
{
    const int k = threadIdx.x; // blockDim = 256 = kHidden
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    float s = 0.0f, sb = 0.0f;
    for (int i = r0; i < r1; ++i) {
        s += dy[i] * __bfloat162float(H[(size_t)i * kHidden + k]);
        sb += dy[i];
    }
    part[(size_t)blockIdx.x * (kHidden + 1) + k] = s;
    if (k == 0)
        part[(size_t)blockIdx.x * (kHidden + 1) + kHidden] = sb;
}

// per-block partial column sums of a BF16 [n x 256] matrix
__global__ void colsum_kernel(const __nv_bfloat16 *__restrict__ M, int n, int rows, float *__restrict__ part)
{
    const int k = threadIdx.x;
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    float s = 0.0f;
    for (int i = r0; i < r1; ++i)
        s += __bfloat162float(M[(size_t)i * kHidden + k]);
    part[(size_t)blockIdx.x * kHidden + k] = s;
}

// out[j] = sum_z part[z][j] in a fixed order
__global__ void sum_parts_kernel(const float *__restrict__ part, int nparts, int len, float *__restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len)
        return;
    float s = 0.0f;
    for (int z = 0; z < nparts; ++z)
        s += part[(size_t)z * len + j];
    out[j] = s;
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, int n, float lr, float b1,
                            float b2, float c1, float c2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    if (wb)
        wb[i] = __float2bfloat16(wi);
}

// Recursion constants of the solid harmonics (uniform across a warp: every
// thread walks the same (l, m) sequence), set by set_harmonic_consts.
__constant__ HarmonicConsts c_harm;

// V[i] = (accumulate ? V[i] : 0) + sum_k coef[k] S_k(u_i) + scale * y[i]
// (y may be null), u_i = (pos_i - centre) / R: the far field's FP64 interior
// expansion plus the network's correction.
__global__ void expansion_kernel(const double *__restrict__ pos, int n, double cx, double cy, double cz,
                                 double inv_r, const double *__restrict__ coef, int L,
                                 const float *__restrict__ y, double scale, int accumulate, double *__restrict__ V)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double ux = (pos[3 * i] - cx) * inv_r, uy = (pos[3 * i + 1] - cy) * inv_r, uz = (pos[3 * i + 2] - cz) * inv_r;
    double s = 0.0;
    solid_harmonics(ux, uy, uz, L, c_harm.a, c_harm.b, c_harm.sec, c_harm.sub,
                    [&](int k, double v) { s = fma(__ldg(coef + k), v, s); });
    if (y)
        s += scale * (double)y[i];
    V[i] = accumulate ? V[i] + s : s;
}

// Fallback flags: untrusted voxel, outside the map, or probe position.
__global__ void flag_kernel(const double *__restrict__ pos, int n, double cx, double cy, double cz, double vox,
                            int dim, const unsigned char *__restrict__ trust, int probe_stride, int probe_offset,
                            int *__restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double h = 0.5 * dim * vox;
    int ix = int(floor((pos[3 * i] - cx + h) / vox)), iy = int(floor((pos[3 * i + 1] - cy + h) / vox)),
        iz = int(floor((pos[3 * i + 2] - cz + h) / vox));
    bool inside = ix >= 0 && iy >= 0 && iz >= 0 && ix < dim && iy < dim && iz < dim;
    bool ok = inside && trust[((size_t)ix * dim + iy) * dim + iz];
    bool probe = probe_stride > 0 && (i % probe_stride) == probe_offset;
    flag[i] = (!ok || probe) ? 1 : 0;
}

// Exclusive scan of flags within blocks of 1024; block totals to `tot`.
__global__ void scan_block_kernel(const int *__restrict__ flag, int n, int *__restrict__ pre, int *__restrict__ tot)
{
    __shared__ int s[1024];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? flag[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n)
        pre[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023)
        tot[blockIdx.x] = s[1023];
}

// Exclusive scan of block totals (one thread; the number of blocks is small).
__global__ void scan_tot_kernel(int *__restrict__ tot, int nb, int *__restrict__ count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    int run = 0;
    for (int b = 0; b < nb; ++b) {
        int t = tot[b];
        tot[b] = run;
        run += t;
    }
    *count = run;
}

__global__ void compact_kernel(const double *__restrict__ pos, const int *__restrict__ flag,
                               const int *__restrict__ pre, const int *__restrict__ tot, int n,
                               double *__restrict__ cpos, int *__restrict__ cidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i])
        return;
    const int j = pre[i] + tot[i / 1024];
    cpos[3 * j] = pos[3 * i];
    cpos[3 * j + 1] = pos[3 * i + 1];
    cpos[3 * j + 2] = pos[3 * i + 2];
    cidx[j] = i;
}

// Scatter exact values back; probe positions whose surrogate value missed by
// more than tol mark their voxel untrusted for later calls.
__global__ void scatter_kernel(const double *__restrict__ cV, const int *__restrict__ cidx, const int *__restrict__ count,
                               double *__restrict__ V, const double *__restrict__ pos, double cx, double cy,
                               double cz, double vox, int dim, unsigned char *__restrict__ trust, int probe_stride,
                               int probe_offset, double tol, int *__restrict__ n_fail)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *count)
        return;
    const int i = cidx[j];
    const double exact = cV[j];
    if (probe_stride > 0 && (i % probe_stride) == probe_offset && fabs(V[i] - exact) > tol) {
        const double h = 0.5 * dim * vox;
        int ix = int(floor((pos[3 * i] - cx + h) / vox)), iy = int(floor((pos[3 * i + 1] - cy + h) / vox)),
            iz = int(floor((pos[3 * i + 2] - cz + h) / vox));
        if (ix >= 0 && iy >= 0 && iz >= 0 && ix < dim && iy < dim && iz < dim)
            trust[((size_t)ix * dim + iy) * dim + iz] = 0;
        atomicAdd(n_fail, 1);
    }
    V[i] = exact;
}

} // namespace

cudaError_t features(const double *pos, int n, const float *freq, const double c[3], double inv_r,
                     __nv_bfloat16 *X, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    features_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos, n, freq, c[0], c[1], c[2], inv_r, X);
    return cudaGetLastError();
}

cudaError_t output(const __nv_bfloat16 *H, int n, const float *w, const float *b, float *y, const float *t, float *dy,
                   float *loss_part, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    output_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(H, n, w, b, y, t, dy, loss_part);
    return cudaGetLastError();
}

cudaError_t out_back(const float *dy, int n, const float *w, const float *Z, __nv_bfloat16 *dZ, cudaStream_t s)
{
    size_t tot = (size_t)n * kHidden;
    out_back_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(dy, n, w, Z, dZ);
    return cudaGetLastError();
}

cudaError_t out_grad(const float *dy, const __nv_bfloat16 *H, int n, float *part, int nparts, float *out,
                     cudaStream_t s)
{
    const int rows = (n + nparts - 1) / nparts;
    out_grad_kernel<<<nparts, kHidden, 0, s>>>(dy, H, n, rows, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return sum_parts(part, nparts, kHidden + 1, out, s);
}

cudaError_t colsum(const __nv_bfloat16 *M, int n, float *part, int nparts, float *out, cudaStream_t s)
{
    const int rows = (n + nparts - 1) / nparts;
    colsum_kernel<<<nparts, kHidden, 0, s>>>(M, n, rows, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return sum_parts(part, nparts, kHidden, out, s);
}

cudaError_t sum_parts(const float *part, int nparts, int len, float *out, cudaStream_t s)
{
    sum_parts_kernel<<<(len + 255) / 256, 256, 0, s>>>(part, nparts, len, out);
    return cudaGetLastError();
}

cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, int n, float lr, float b1,
                 float b2, int step, float eps, cudaStream_t s)
{
    const float c1 = 1.0f / (1.0f - powf(b1, float(step))), c2 = 1.0f / (1.0f - powf(b2, float(step)));
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, wb, n, lr, b1, b2, c1, c2, eps);
    return cudaGetLastError();
}

cudaError_t set_harmonic_consts()
{
    static HarmonicConsts h;
    static bool ready = false;
    if (!ready) {
        harmonic_consts(h);
        ready = true;
    }
    return cudaMemcpyToSymbol(c_harm, &h, sizeof(h));
}

cudaError_t expansion(const double *pos, int n, const double c[3], double inv_r, const double *coef, int L,
                      const float *y, double scale, bool accumulate, double *V, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    if (L < 0 || L > kMaxExpDegree)
        return cudaErrorInvalidValue;
    expansion_kernel<<<(n + 127) / 128, 128, 0, s>>>(pos, n, c[0], c[1], c[2], inv_r, coef, L, y, scale,
                                                     accumulate ? 1 : 0, V);
    return cudaGetLastError();
}

cudaError_t fallback_select(const double *pos, int n, const double c[3], double vox, int dim,
                            const unsigned char *trust, int probe_stride, int probe_offset, int *flag, int *pre,
                            int *tot, int *count, double *cpos, int *cidx, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    flag_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos, n, c[0], c[1], c[2], vox, dim, trust, probe_stride,
                                                probe_offset, flag);
    const int nb = (n + 1023) / 1024;
    scan_block_kernel<<<nb, 1024, 0, s>>>(flag, n, pre, tot);
    scan_tot_kernel<<<1, 1, 0, s>>>(tot, nb, count);
    compact_kernel<<<(n + 255) / 256, 256, 0, s>>>(pos, flag, pre, tot, n, cpos, cidx);
    return cudaGetLastError();
}

cudaError_t fallback_scatter(const double *cV, const int *cidx, const int *count, int n_max, double *V,
                             const double *pos, const double c[3], double vox, int dim, unsigned char *trust,
                             int probe_stride, int probe_offset, double tol, int *n_fail, cudaStream_t s)
{
    if (n_max <= 0)
        return cudaSuccess;
    scatter_kernel<<<(n_max + 255) / 256, 256, 0, s>>>(cV, cidx, count, V, pos, c[0], c[1], c[2], vox, dim, trust,
                                                       probe_stride, probe_offset, tol, n_fail);
    return cudaGetLastError();
}

} // namespace sur
} // namespace esp
