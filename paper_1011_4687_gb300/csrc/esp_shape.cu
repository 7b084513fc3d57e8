// One launch shape of the potential kernels.  The build compiles this file
// once per entry of the lists in esp_shapes.h, defining ESP_NT, ESP_PPT and
// one of ESP_SHAPE_F32C, ESP_SHAPE_F64 or ESP_SHAPE_BATCH (with ESP_PREC).
#include "esp_potential.cuh"
#include "esp_shapes.h"

#include <algorithm>

#if !defined(ESP_NT) || !defined(ESP_PPT)
#error "esp_shape.cu is compiled once per launch shape: define ESP_NT and ESP_PPT"
#endif

namespace esp {

#if defined(ESP_SHAPE_F32C)
template <int NT, int PPT>
cudaError_t launch_f32c_shape(const EvalArgs &a, dim3 grid, size_t smem, cudaStream_t s)
{
    auto k = potential_f32c_kernel<NT, PPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_f32c_shape<ESP_NT, ESP_PPT>(const EvalArgs &, dim3, size_t, cudaStream_t);

#elif defined(ESP_SHAPE_F64)
template <int NT, int PPT>
cudaError_t launch_f64_shape(const EvalArgs &a, dim3 grid, size_t smem, cudaStream_t s)
{
    auto k = potential_f64_kernel<NT, PPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_f64_shape<ESP_NT, ESP_PPT>(const EvalArgs &, dim3, size_t, cudaStream_t);

#elif defined(ESP_SHAPE_BATCH)
template <int NT, int PPT, int PREC>
cudaError_t launch_batch_shape(const BatchHeader *hdr, const SysDesc *sys, int *counter, int max_items,
                               const float *boys32, const double *boys64, int tile_cap, int num_sms, size_t smem,
                               cudaStream_t s)
{
    auto k = batch_potential_kernel<NT, PPT, PREC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(per_sm * num_sms, max_items));
    k<<<grid, NT, smem, s>>>(hdr, sys, counter, boys32, boys64, tile_cap);
    return cudaGetLastError();
}
template cudaError_t launch_batch_shape<ESP_NT, ESP_PPT, ESP_PREC>(const BatchHeader *, const SysDesc *, int *, int,
                                                                   const float *, const double *, int, int, size_t,
                                                                   cudaStream_t);
#else
#error "define ESP_SHAPE_F32C, ESP_SHAPE_F64 or ESP_SHAPE_BATCH"
#endif

} // namespace esp
