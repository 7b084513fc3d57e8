// Launch shapes of the potential kernels compiled into the library.
//
// Each entry is one object file: the build compiles esp_shape.cu once per
// entry (threads per CTA, positions per thread[, precision]), so the shapes
// compile in parallel, and the dispatchers in esp_kernels.cu call the
// launchers declared here.  The build reads these three lists.
#pragma once

#include "esp_kernels.h"

#define ESP_F32C_SHAPES(X) X(64, 2) X(64, 4) X(128, 1) X(128, 2) X(128, 4) X(256, 1) X(256, 2)
#define ESP_F64_SHAPES(X) X(64, 1) X(64, 2) X(128, 1) X(128, 2) X(256, 1) X(256, 2)
// precision 1 = FP32C, 0 = FP64
#define ESP_BATCH_SHAPES(X) X(128, 4, 1) X(128, 2, 1) X(256, 2, 1) X(64, 4, 1) X(128, 2, 0) X(128, 1, 0) X(256, 1, 0)

namespace esp {

// One launch of potential_f32c_kernel<NT, PPT> / potential_f64_kernel<NT, PPT>
// on grid (position blocks, splits) with `smem` bytes of dynamic shared memory.
template <int NT, int PPT>
cudaError_t launch_f32c_shape(const EvalArgs &a, dim3 grid, size_t smem, cudaStream_t s);
template <int NT, int PPT>
cudaError_t launch_f64_shape(const EvalArgs &a, dim3 grid, size_t smem, cudaStream_t s);

// The persistent batched kernel with as many CTAs as fit on the GPU (capped
// at max_items work items).
template <int NT, int PPT, int PREC>
cudaError_t launch_batch_shape(const BatchHeader *hdr, const SysDesc *sys, int *counter, int max_items,
                               const float *boys32, const double *boys64, int tile_cap, int num_sms, size_t smem,
                               cudaStream_t s);

} // namespace esp
