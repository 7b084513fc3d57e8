// The training GEMMs of the surrogate network on the 5th-generation tensor
// cores: C = op(A) op(B) (+ the epilogues of GemmArgs), BF16 x BF16 -> FP32.
//
// One CTA of 128 threads computes a 128 x BN tile of C (BN = 64, or 256 when
// that still gives every SM two CTAs) with its accumulator in tensor memory
// (BN columns).  K runs in chunks of 64
// through two shared-memory stages: every thread stages one 8 x 8 core matrix
// of the A chunk (128 rows) and BN / 16 of the B chunk (BN rows) per chunk,
// loading 8 rows of 16 bytes from global memory and, where the source runs
// along the operand's rows instead of K (op = transpose), transposing the
// 8 x 8 block in registers; the block lands as the 128 contiguous bytes of
// its core matrix in the no-swizzle K-major layout (tc_ptx.h).  One thread
// issues the four K = 16 MMAs of a chunk and commits them to the stage's
// mbarrier; the stage is refilled once that commit has completed, so the
// loads of chunk c + 1 overlap the MMAs of chunk c.  The epilogue reads the
// accumulator back with tcgen05.ld (thread t: row t, 32 columns at a time).
// grid.z splits K into slices of kchunk (partials to C + z M ldc).
//
// Every mbarrier wait is bounded; a CTA whose wait gives up sets *err, waits
// (bounded) for the MMAs it has committed, frees its tensor memory and
// returns without writing C.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "surrogate_kernels.h"
#include "tc_ptx.h"

namespace esp {
namespace sur {

namespace {

constexpr int kTileM = 128;     // MMA M: rows of C per CTA
constexpr int kChunk = 64;      // K columns per stage
constexpr int kGemmThreads = 128;
constexpr int kGemmWait = 1 << 22; // ~1 s of suspended try_waits

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z)
{
    float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// op(X)[r][k] for operand row r (M for A, N for B) and K index k:
// ROWC (rows contiguous in memory): X[k ld + r], else X[r ld + k].
// Stages the 8 x 8 block (rows r0.., k k0..) as one core matrix at dst:
// row i of the block (operand row r0 + i, k0..k0+7) at dst + 16 i.
// Elements outside rows < R or k < kend are zero.
template <bool ROWC>
__device__ __forceinline__ void stage_block(unsigned char *dst, const __nv_bfloat16 *__restrict__ X, int ld, int r0,
                                            int R, int k0, int kend, bool vec)
{
    uint4 out[8];
    if (!ROWC) {
        // 8 rows, each 8 consecutive k: one 16-byte load per row
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = r0 + i;
            if (vec && r < R && k0 + 8 <= kend) {
                out[i] = __ldg(reinterpret_cast<const uint4 *>(X + (size_t)r * ld + k0));
            } else {
                __align__(16) __nv_bfloat16 t[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    t[j] = (r < R && k0 + j < kend) ? X[(size_t)r * ld + k0 + j] : __float2bfloat16(0.0f);
                out[i] = *reinterpret_cast<const uint4 *>(t);
            }
        }
    } else {
        // 8 k-lines, each 8 consecutive rows; transpose the block in registers
        __align__(16) unsigned short w[8][8]; // w[j][i] = element (row r0 + i, k0 + j)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j;
            if (vec && k < kend && r0 + 8 <= R) {
                *reinterpret_cast<uint4 *>(w[j]) = __ldg(reinterpret_cast<const uint4 *>(X + (size_t)k * ld + r0));
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    w[j][i] = (k < kend && r0 + i < R) ? __bfloat16_as_ushort(X[(size_t)k * ld + r0 + i])
                                                       : (unsigned short)0;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            out[i] = make_uint4(uint32_t(w[0][i]) | (uint32_t(w[1][i]) << 16), uint32_t(w[2][i]) | (uint32_t(w[3][i]) << 16),
                                uint32_t(w[4][i]) | (uint32_t(w[5][i]) << 16), uint32_t(w[6][i]) | (uint32_t(w[7][i]) << 16));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
        reinterpret_cast<uint4 *>(dst)[i] = out[i];
}

template <bool A_T, bool B_T, int BN>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_tc_kernel(GemmArgs g, int *__restrict__ err, int vec_a, int vec_b, int wait_limit)
{
    constexpr int kABytes = kTileM * kChunk * 2;  // 16 KB
    constexpr int kBBytes = BN * kChunk * 2;      // 8 or 32 KB
    constexpr int kStage = kABytes + kBBytes;
    constexpr uint32_t kIdesc = tc::idesc_bf16(kTileM, BN);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * kTileM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * g.kchunk;
    const int kend = min(g.K, kbeg + g.kchunk);
    const int nc = kend > kbeg ? (kend - kbeg + kChunk - 1) / kChunk : 0;

    if (warp == 0)
        tc::tmem_alloc(tc::smem_u32(&s_tmem), BN);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&bar[0]), 1);
        tc::mbar_init(tc::smem_u32(&bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;

    int issued[2] = {0, 0}; // commits made on each stage's barrier
    bool ok = true;
    for (int c = 0; c < nc; ++c) {
        const int st = c & 1;
        unsigned char *sA = smem + st * kStage, *sB = sA + kABytes;
        // the stage's previous MMAs (chunk c - 2) must have read it
        bool wok = true;
        if (issued[st] > 0)
            wok = tc::mbar_wait(tc::smem_u32(&bar[st]), uint32_t(issued[st] - 1) & 1u, wait_limit);
        if (!__syncthreads_and(wok)) {
            ok = false;
            break;
        }
        const int k0 = kbeg + c * kChunk;
        // A: 16 row blocks x 8 k blocks = 128 core matrices, one per thread
        {
            const int rb = tid & 15, kb = tid >> 4;
            stage_block<A_T>(sA + tc::operand_off(8 * rb, 8 * kb, kTileM), g.A, g.lda, m0 + 8 * rb, g.M, k0 + 8 * kb,
                             kend, vec_a != 0);
        }
        // B: BN / 8 row blocks x 8 k blocks
#pragma unroll
        for (int b = tid; b < (BN / 8) * 8; b += kGemmThreads) {
            const int rb = b % (BN / 8), kb = b / (BN / 8);
            stage_block<!B_T>(sB + tc::operand_off(8 * rb, 8 * kb, BN), g.B, g.ldb, n0 + 8 * rb, g.N, k0 + 8 * kb,
                              kend, vec_b != 0);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t aA = tc::smem_u32(sA), aB = tc::smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < kChunk; ks += 16)
                tc::mma_bf16(tmem, tc::operand_desc(aA, ks, kTileM), tc::operand_desc(aB, ks, BN), kIdesc,
                             (c > 0 || ks > 0) ? 1u : 0u);
            tc::mma_commit(tc::smem_u32(&bar[st]));
        }
        ++issued[st];
    }
    // all MMAs done: the last commit tracks every earlier one
    if (ok && nc > 0) {
        const int st = (nc - 1) & 1;
        ok = __syncthreads_and(tc::mbar_wait(tc::smem_u32(&bar[st]), uint32_t(issued[st] - 1) & 1u, wait_limit));
    }
    tc::fence_after();
    if (ok) {
        const int row = tid; // TMEM lane = row of the tile
        const int m = m0 + row;
        const uint32_t lane_addr = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            if (nc > 0) {
                tc::tmem_ld32(lane_addr + uint32_t(c0), v);
            } else {
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    v[e] = 0.0f;
            }
            if (m >= g.M)
                continue;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int n = n0 + c0 + e;
                if (n >= g.N)
                    continue;
                const size_t o = (size_t)m * g.ldc + n;
                switch (g.epi) {
                case kEpiSiluFwd: {
                    const float z = v[e] + g.bias[n];
                    if (g.Cf)
                        g.Cf[o] = z;
                    g.Cb[o] = __float2bfloat16(silu_f(z));
                    break;
                }
                case kEpiGradSilu:
                    g.Cb[o] = __float2bfloat16(v[e] * silu_grad_f(g.aux[o]));
                    break;
                default:
                    g.Cf[(size_t)blockIdx.z * g.M * g.ldc + o] = v[e];
                }
            }
        }
    }
    if (tid == 0) {
        if (!ok)
            atomicExch(err, 1);
        // each stage's last commit has completed before the CTA's memory goes
        // away (at once where it was seen above; bounded otherwise)
        for (int st = 0; st < 2; ++st)
            if (issued[st] > 0)
                tc::mbar_wait(tc::smem_u32(&bar[st]), uint32_t(issued[st] - 1) & 1u, kGemmWait);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, BN);
    }
}

template <bool A_T, bool B_T, int BN>
cudaError_t launch_tc(const GemmArgs &g, int ksplit, int *err, int wait_limit, cudaStream_t s)
{
    constexpr int smem = 2 * (kTileM * kChunk * 2 + BN * kChunk * 2);
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<A_T, B_T, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    // 16-byte vector loads need 16-byte aligned rows and K slices starting on
    // multiples of 8
    const bool kal = ksplit == 1 || g.kchunk % 8 == 0;
    const int vec_a = (kal && g.lda % 8 == 0 && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0) ? 1 : 0;
    const int vec_b = (kal && g.ldb % 8 == 0 && (reinterpret_cast<uintptr_t>(g.B) & 15) == 0) ? 1 : 0;
    dim3 grid((g.N + BN - 1) / BN, (g.M + kTileM - 1) / kTileM, ksplit);
    gemm_tc_kernel<A_T, B_T, BN><<<grid, kGemmThreads, smem, s>>>(g, err, vec_a, vec_b, wait_limit);
    return cudaGetLastError();
}

} // namespace

cudaError_t gemm_tc(bool a_t, bool b_t, const GemmArgs &g, int ksplit, int *err, int wait_limit, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0)
        return cudaSuccess;
    if (g.N > 256 || ksplit < 1 || g.kchunk < 1 || !err || wait_limit < 0)
        return cudaErrorInvalidValue;
    // 256-column tiles only when they alone give every SM two CTAs; the
    // training shapes (8,192-row batches, 256 x 256 weight gradients) take
    // 64-column tiles and four times the CTAs
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const long long tiles256 = (long long)((g.N + 255) / 256) * ((g.M + kTileM - 1) / kTileM) * ksplit;
    const bool wide = g.N > 64 && tiles256 >= 2LL * sms;
#define ESP_TC(AT, BT)                                                                                              \
    return wide ? launch_tc<AT, BT, 256>(g, ksplit, err, wait_limit, s)                                             \
                : launch_tc<AT, BT, 64>(g, ksplit, err, wait_limit, s)
    if (a_t) {
        if (b_t)
            ESP_TC(true, true);
        ESP_TC(true, false);
    }
    if (b_t)
        ESP_TC(false, true);
    ESP_TC(false, false);
#undef ESP_TC
}

} // namespace sur
} // namespace esp
