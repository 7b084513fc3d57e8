// Fused inference of the surrogate network on the 5th-generation tensor cores.
//
// One persistent CTA per SM takes tiles of 128 positions (the MMA's M), one
// after the other, through the whole network:
// Fourier features -> 4 x (Linear 256 + SiLU) -> Linear 1, with the
// activations kept in shared memory as BF16 and every layer's accumulator
// (128 x 256 FP32) in tensor memory.  Per layer, one elected thread issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, K = 16 per instruction) from
// shared-memory descriptors, and commits to an mbarrier; the weights of the
// next layer stream in with cp.async.bulk while all 16 warps read the
// accumulator back with tcgen05.ld (warp w: lanes 32 (w % 4).., columns
// 64 (w / 4)..), add the bias (staged in shared memory), apply SiLU and write
// the next layer's BF16 operand.  The output layer is a dot product in the
// last epilogue.  The epilogue is latency-bound, so it runs on 16 warps.
//
// Operands use the no-swizzle K-major canonical layout of tc_ptx.h.
// Weights are packed into this layout once
// per parameter update (pack_weights_kernel), in chunks of 64 K-columns
// (32 KB), so each chunk is one contiguous bulk copy.
//
// The rounding points are those of the unfused path: features and hidden
// activations in BF16, FP32 accumulation, FP32 bias and output weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "surrogate_kernels.h"
#include "tc_ptx.h"

namespace esp {
namespace sur {

namespace {

constexpr int kRows = 128;                       // positions per CTA (MMA M)
constexpr int kThreads = 512;                    // 16 warps: 4 lane quarters x 4 column groups
constexpr int kColGroups = kThreads / 128;       // column groups of the epilogue
constexpr int kGroupCols = kHidden / kColGroups; // 64 accumulator columns per warp
constexpr int kChunkK = 64;                      // K columns per weight chunk
constexpr int kChunkBytes = kHidden * kChunkK * 2; // 32 KB
constexpr int kABytes = kRows * kHidden * 2;     // 64 KB activation operand
constexpr int kWBytes = kHidden * kHidden * 2;   // 128 KB: one whole layer of weights
constexpr int kTmemCols = 256;                   // FP32 accumulator columns (N)
// Bounded waits.  The main waits take their limit from the caller
// (tc_default_wait_limit(): ~1 s at a few hundred ns per suspended try_wait);
// after a wait has given up, the clean-up waits for this CTA's own copies and
// MMAs in flight always use the default, so no asynchronous write into shared
// or tensor memory outlives the CTA's allocations.
constexpr int kWaitLimit = 1 << 22;

constexpr uint32_t kIdesc = tc::idesc_bf16(kRows, kHidden);

using tc::bulk_load;
using tc::fence_async_smem;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::operand_off;
using tc::pack_bf16x2;
using tc::smem_desc;
using tc::smem_u32;
using tc::tmem_ld32;
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    tc::mma_bf16(tmem_d, adesc, bdesc, kIdesc, accumulate);
}

// SiLU with the fast division (the result is rounded to BF16 or multiplied
// into an FP32 dot product; a few ulp of FP32 do not reach it)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__global__ void __launch_bounds__(kThreads, 1)
    mlp_tc_kernel(const double *__restrict__ pos, int n, const float *__restrict__ freq, double cx, double cy,
                  double cz, double inv_r, const __nv_bfloat16 *__restrict__ wpk, const float *__restrict__ params,
                  TcLayout lay, float *__restrict__ y, int *__restrict__ err, int n_tiles, int wait_limit)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;
    unsigned char *sW = smem + kABytes;
    __shared__ __align__(8) uint64_t bar_w[kHidden / kChunkK];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ float s_part[kColGroups][kRows];
    __shared__ __align__(16) float s_bias[kLayers][kHidden];
    __shared__ __align__(16) float s_w5[kHidden];
    __shared__ float s_freq[3 * kFreq];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t aA = smem_u32(sA), aW = smem_u32(sW);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int c = 0; c < kHidden / kChunkK; ++c)
            mbar_init(smem_u32(&bar_w[c]), 1);
        mbar_init(smem_u32(&bar_mma), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // biases and output weights to shared memory
    for (int i = tid; i < kLayers * kHidden; i += kThreads)
        s_bias[i / kHidden][i % kHidden] = params[lay.b[i / kHidden] + i % kHidden];
    for (int i = tid; i < kHidden; i += kThreads)
        s_w5[i] = params[lay.w5 + i];
    for (int i = tid; i < 3 * kFreq; i += kThreads)
        s_freq[i] = freq[i];
    __syncthreads();

    // layer-1 weights of the first tile: K = 64, one chunk
    if (tid == 0 && blockIdx.x < n_tiles)
        bulk_load(aW, wpk + lay.wpk[0], kChunkBytes, smem_u32(&bar_w[0]));

    uint32_t wpar[kHidden / kChunkK] = {0, 0, 0, 0};
    uint32_t mpar = 0;
    bool mma_pending = false;   // a commit whose completion nobody has seen (after a failed wait)
    uint32_t mma_pending_par = 0;
    const int q = warp & 3, hcol = (warp >> 2) * kGroupCols;
    const int row = q * 32 + lane;
    bool ok = true;
    // this thread's feature row (tid % 128) of the first tile; later tiles'
    // rows are loaded during the previous tile's last layer
    double px, py, pz;
    {
        const int i = min(int(blockIdx.x) * kRows + tid % kRows, n - 1);
        px = pos[3 * i];
        py = pos[3 * i + 1];
        pz = pos[3 * i + 2];
    }
    // persistent: this CTA takes row tiles blockIdx.x, + gridDim.x, ...; the
    // tensor memory, barriers, biases and the weight stream carry over
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int row0 = tile * kRows;
        const bool has_next = tile + int(gridDim.x) < n_tiles;
        // Fourier features of this CTA's rows: row tid % 128, frequencies
        // 8 (tid / 128) .. + 7 (sin and cos), one 16-byte store each
        {
            const int r = tid % kRows, f0 = 8 * (tid / kRows);
            const float ux = float((px - cx) * inv_r), uy = float((py - cy) * inv_r), uz = float((pz - cz) * inv_r);
            float sn[8], cs[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int f = f0 + e;
                float ph = 6.283185307179586f * (s_freq[3 * f] * ux + s_freq[3 * f + 1] * uy + s_freq[3 * f + 2] * uz);
                __sincosf(ph, &sn[e], &cs[e]);
            }
            const uint4 vs = make_uint4(pack_bf16x2(sn[0], sn[1]), pack_bf16x2(sn[2], sn[3]), pack_bf16x2(sn[4], sn[5]),
                                        pack_bf16x2(sn[6], sn[7]));
            const uint4 vc = make_uint4(pack_bf16x2(cs[0], cs[1]), pack_bf16x2(cs[2], cs[3]), pack_bf16x2(cs[4], cs[5]),
                                        pack_bf16x2(cs[6], cs[7]));
            *reinterpret_cast<uint4 *>(sA + operand_off(r, f0, kRows)) = vs;
            *reinterpret_cast<uint4 *>(sA + operand_off(r, kFreq + f0, kRows)) = vc;
        }
        fence_async_smem();
        __syncthreads();

        float part = 0.0f;
        for (int l = 0; l < kLayers; ++l) {
            const int nchunk = (l == 0 ? kFeat : kHidden) / kChunkK;
            bool wok = true;
            if (tid == 0) {
                tc_fence_after();
                for (int c = 0; c < nchunk; ++c) {
                    if (!(wok = mbar_wait(smem_u32(&bar_w[c]), wpar[c], wait_limit)))
                        break;
#pragma unroll
                    for (int ks = 0; ks < kChunkK; ks += 16) {
                        const int k0 = c * kChunkK + ks;
                        const uint64_t ad = smem_desc(aA + (k0 >> 3) * (kRows / 8) * 128, (kRows / 8) * 128, 128);
                        const uint64_t bd =
                            smem_desc(aW + c * kChunkBytes + (ks >> 3) * (kHidden / 8) * 128, (kHidden / 8) * 128, 128);
                        mma_bf16(tmem, ad, bd, k0 > 0 ? 1u : 0u);
                    }
                }
                mma_commit(smem_u32(&bar_mma)); // always: tracks whatever was issued
            }
            for (int c = 0; c < nchunk; ++c)
                wpar[c] ^= 1u;
            const bool mok = mbar_wait(smem_u32(&bar_mma), mpar, wait_limit);
            if (!mok) {
                mma_pending = true;
                mma_pending_par = mpar;
            }
            mpar ^= 1u;
            tc_fence_after();
            if (__syncthreads_or((wok && mok) ? 0 : 1)) {
                ok = false;
                break;
            }
            // the weight buffer is free: stream in the next layer (or the next
            // tile's first layer) during the epilogue
            if (tid == 0 && l + 1 < kLayers)
                for (int c = 0; c < kHidden / kChunkK; ++c)
                    bulk_load(aW + c * kChunkBytes, wpk + lay.wpk[l + 1] + size_t(c) * (kChunkBytes / 2), kChunkBytes,
                              smem_u32(&bar_w[c]));
            else if (tid == 0 && has_next)
                bulk_load(aW, wpk + lay.wpk[0], kChunkBytes, smem_u32(&bar_w[0]));
            if (l + 1 == kLayers && has_next) { // the next tile's feature row, ahead of its use
                const int i = min((tile + int(gridDim.x)) * kRows + tid % kRows, n - 1);
                px = pos[3 * i];
                py = pos[3 * i + 1];
                pz = pos[3 * i + 2];
            }

            const float *bias = s_bias[l];
#pragma unroll 1
            for (int cc = 0; cc < kGroupCols; cc += 32) {
                const int col0 = hcol + cc;
                float v[32];
                tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(col0), v);
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    v[e] = silu(v[e] + bias[col0 + e]);
                if (l + 1 < kLayers) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        uint4 pk = make_uint4(pack_bf16x2(v[8 * m], v[8 * m + 1]), pack_bf16x2(v[8 * m + 2], v[8 * m + 3]),
                                              pack_bf16x2(v[8 * m + 4], v[8 * m + 5]),
                                              pack_bf16x2(v[8 * m + 6], v[8 * m + 7]));
                        *reinterpret_cast<uint4 *>(sA + operand_off(row, col0 + 8 * m, kRows)) = pk;
                    }
                } else {
                    const float *w5 = s_w5;
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        part = fmaf(__bfloat162float(__float2bfloat16(v[e])), w5[col0 + e], part);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
        }
        if (ok) {
            s_part[warp >> 2][row] = part;
            __syncthreads();
            if (tid < kRows && row0 + tid < n)
                y[row0 + tid] = ((s_part[0][tid] + s_part[1][tid]) + (s_part[2][tid] + s_part[3][tid])) + params[lay.b5];
        }
    } // row tiles
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        // let weight copies still in flight land before the CTA's shared
        // memory is released (a completed or unused chunk returns at once),
        // and the MMAs of a commit nobody waited for finish before the tensor
        // memory is freed
        for (int c = 0; c < kHidden / kChunkK; ++c)
            mbar_wait(smem_u32(&bar_w[c]), wpar[c] ^ 1u, kWaitLimit);
        if (mma_pending)
            mbar_wait(smem_u32(&bar_mma), mma_pending_par, kWaitLimit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// Weights W_l [256][K] (row-major BF16, as trained) -> the K-major no-swizzle
// layout above, in chunks of 64 K-columns.
__global__ void pack_weights_kernel(const __nv_bfloat16 *__restrict__ wb, TcLayout lay, __nv_bfloat16 *__restrict__ wpk)
{
    const int l = blockIdx.y;
    const int K = l == 0 ? kFeat : kHidden;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kHidden * K)
        return;
    const int nrow = e / K, k = e % K;
    const int c = k / kChunkK, kk = k % kChunkK;
    const size_t dst = size_t(c) * (kChunkBytes / 2) +
                       size_t(((kk >> 3) * (kHidden >> 3) + (nrow >> 3)) * 64 + (nrow & 7) * 8 + (k & 7));
    wpk[lay.wpk[l] + dst] = wb[lay.w[l] + size_t(nrow) * K + k];
}

} // namespace

size_t tc_packed_elems() { return size_t(kHidden) * kFeat + size_t(kLayers - 1) * kHidden * kHidden; }

cudaError_t tc_pack(const __nv_bfloat16 *wb, const TcLayout &lay, __nv_bfloat16 *wpk, cudaStream_t s)
{
    dim3 grid((kHidden * kHidden + 255) / 256, kLayers);
    pack_weights_kernel<<<grid, 256, 0, s>>>(wb, lay, wpk);
    return cudaGetLastError();
}

int tc_default_wait_limit() { return kWaitLimit; }

cudaError_t tc_forward(const double *pos, int n, const float *freq, const double c[3], double inv_r,
                       const __nv_bfloat16 *wpk, const float *params, const TcLayout &lay, float *y, int *err,
                       int wait_limit, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    const int smem = kABytes + kWBytes;
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int n_tiles = (n + kRows - 1) / kRows;
    const int grid = n_tiles < sms ? n_tiles : sms; // one persistent CTA per SM
    mlp_tc_kernel<<<grid, kThreads, smem, s>>>(pos, n, freq, c[0], c[1], c[2], inv_r, wpk, params, lay, y, err,
                                               n_tiles, wait_limit < 0 ? 0 : wait_limit);
    return cudaGetLastError();
}

} // namespace sur
} // namespace esp
