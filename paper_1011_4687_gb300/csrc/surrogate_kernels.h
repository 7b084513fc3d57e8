// Launch interface of the surrogate kernels (see surrogate_kernels.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace esp {
namespace sur {

constexpr int kFreq = 32;       // Fourier frequencies
constexpr int kFeat = 64;       // features: sin and cos of each frequency
constexpr int kHidden = 256;    // width of each hidden layer
constexpr int kLayers = 4;      // hidden layers

enum { kEpiSiluFwd = 0, kEpiGradSilu = 1, kEpiRaw = 2 };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A;
    int lda;
    const __nv_bfloat16 *B;
    int ldb;
    float *Cf;            // FP32 output (Z for kEpiSiluFwd, partials for kEpiRaw)
    __nv_bfloat16 *Cb;    // BF16 output
    int ldc;
    const float *bias;    // [N] (kEpiSiluFwd)
    const float *aux;     // [M][ldc] pre-activation of the previous layer (kEpiGradSilu)
    int epi;
    int kchunk;           // K range of one grid.z slice
};

// C = op(A) op(B) with the epilogue g.epi on the tcgen05 tensor cores
// (surrogate_gemm.cu); N <= 256, grid.z = ksplit slices of g.kchunk.  *err is
// set to 1 if a bounded wait (wait_limit tries) gave up; C is then not written.
cudaError_t gemm_tc(bool a_t, bool b_t, const GemmArgs &g, int ksplit, int *err, int wait_limit, cudaStream_t s);

// Fused tcgen05 inference (surrogate_tc.cu).  Offsets (elements) of each
// layer's weights and biases in the flat parameter vectors, and of each
// layer's packed weights.
struct TcLayout {
    size_t w[kLayers], b[kLayers], w5, b5, wpk[kLayers];
};
size_t tc_packed_elems();
// Pack the BF16 weights (flat layout) into the tensor-core operand layout.
cudaError_t tc_pack(const __nv_bfloat16 *wb, const TcLayout &lay, __nv_bfloat16 *wpk, cudaStream_t s);
// y[i] = network output at position i (features, 4 hidden layers, output
// layer); *err is set to 1 if a bounded wait of the kernel gave up.
// wait_limit: iterations of each of the kernel's mbarrier waits before it
// gives up (sets *err, drains its own copies, frees its tensor memory and
// returns); tc_default_wait_limit() is about one second.
int tc_default_wait_limit();
cudaError_t tc_forward(const double *pos, int n, const float *freq, const double c[3], double inv_r,
                       const __nv_bfloat16 *wpk, const float *params, const TcLayout &lay, float *y, int *err,
                       int wait_limit, cudaStream_t s);
cudaError_t features(const double *pos, int n, const float *freq, const double c[3], double inv_r,
                     __nv_bfloat16 *X, cudaStream_t s);
// y[i] = H[i] . w + *b; with targets t: dy = 2 (y - t) / n and squared errors
cudaError_t output(const __nv_bfloat16 *H, int n, const float *w, const float *b, float *y, const float *t, float *dy,
                   float *loss_part, cudaStream_t s);
cudaError_t out_back(const float *dy, int n, const float *w, const float *Z, __nv_bfloat16 *dZ, cudaStream_t s);
cudaError_t out_grad(const float *dy, const __nv_bfloat16 *H, int n, float *part, int nparts, float *out,
                     cudaStream_t s);
// out[k] = sum_i M[i][k] for a BF16 [n x 256] matrix (fixed-order partials)
cudaError_t colsum(const __nv_bfloat16 *M, int n, float *part, int nparts, float *out, cudaStream_t s);
cudaError_t sum_parts(const float *part, int nparts, int len, float *out, cudaStream_t s);
cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, int n, float lr, float b1,
                 float b2, int step, float eps, cudaStream_t s);
// Recursion constants of the solid harmonics into the current device's
// constant memory (once per device before the first expansion launch).
cudaError_t set_harmonic_consts();
// V[i] = (accumulate ? V[i] : 0) + sum_k coef[k] S_k(u_i) + scale * y[i]
// (y may be null): the far field's interior expansion of degree L
// (esp_harmonics.h) plus the network's correction, u_i = (pos_i - c) inv_r.
cudaError_t expansion(const double *pos, int n, const double c[3], double inv_r, const double *coef, int L,
                      const float *y, double scale, bool accumulate, double *V, cudaStream_t s);
cudaError_t fallback_select(const double *pos, int n, const double c[3], double vox, int dim,
                            const unsigned char *trust, int probe_stride, int probe_offset, int *flag, int *pre,
                            int *tot, int *count, double *cpos, int *cidx, cudaStream_t s);
cudaError_t fallback_scatter(const double *cV, const int *cidx, const int *count, int n_max, double *V,
                             const double *pos, const double c[3], double vox, int dim, unsigned char *trust,
                             int probe_stride, int probe_offset, double tol, int *n_fail, cudaStream_t s);

} // namespace sur
} // namespace esp
