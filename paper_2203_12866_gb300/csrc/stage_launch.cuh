// Host-side launcher of the fused RK4 stage kernels; each (scheme, precision)
// pair is instantiated in its own translation unit so the four compile in
// parallel.
#pragma once

#include "stage_kernel.cuh"

namespace cosenu {

template <int SCHEME, int PREC>
cudaError_t launch_rk4_stage(int stage, const StageArgs& a, int grid, int block, size_t smem,
                             cudaStream_t stream);

template <int SCHEME, int PREC>
int stage_max_blocks_per_sm(int stage, int block, size_t smem);

#define COSENU_INSTANTIATE_STAGE(SCHEME, PREC)                                                   \
  template <int STAGE>                                                                           \
  static cudaError_t launch_one_##SCHEME##_##PREC(const StageArgs& a, int grid, int block,      \
                                                  size_t smem, cudaStream_t stream) {            \
    static bool attr_set = false;                                                                \
    auto fn = rk4_stage_kernel<SCHEME, PREC, STAGE>;                                             \
    if (!attr_set) {                                                                             \
      cudaError_t e =                                                                            \
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);         \
      if (e != cudaSuccess) return e;                                                            \
      attr_set = true;                                                                           \
    }                                                                                            \
    fn<<<grid, block, smem, stream>>>(a);                                                        \
    return cudaGetLastError();                                                                   \
  }                                                                                              \
  template <>                                                                                    \
  cudaError_t launch_rk4_stage<SCHEME, PREC>(int stage, const StageArgs& a, int grid, int block, \
                                             size_t smem, cudaStream_t stream) {                 \
    switch (stage) {                                                                             \
      case 1: return launch_one_##SCHEME##_##PREC<1>(a, grid, block, smem, stream);              \
      case 2: return launch_one_##SCHEME##_##PREC<2>(a, grid, block, smem, stream);              \
      case 3: return launch_one_##SCHEME##_##PREC<3>(a, grid, block, smem, stream);              \
      case 4: return launch_one_##SCHEME##_##PREC<4>(a, grid, block, smem, stream);              \
      default: return cudaErrorInvalidValue;                                                     \
    }                                                                                            \
  }                                                                                              \
  template <>                                                                                    \
  int stage_max_blocks_per_sm<SCHEME, PREC>(int stage, int block, size_t smem) {                 \
    int n = 0;                                                                                   \
    cudaError_t e = cudaErrorInvalidValue;                                                       \
    switch (stage) {                                                                             \
      case 1: e = cudaFuncSetAttribute(rk4_stage_kernel<SCHEME, PREC, 1>,                        \
                  cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);                          \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
                  &n, rk4_stage_kernel<SCHEME, PREC, 1>, block, smem); break;                    \
      case 2: e = cudaFuncSetAttribute(rk4_stage_kernel<SCHEME, PREC, 2>,                        \
                  cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);                          \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
                  &n, rk4_stage_kernel<SCHEME, PREC, 2>, block, smem); break;                    \
      case 3: e = cudaFuncSetAttribute(rk4_stage_kernel<SCHEME, PREC, 3>,                        \
                  cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);                          \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
                  &n, rk4_stage_kernel<SCHEME, PREC, 3>, block, smem); break;                    \
      case 4: e = cudaFuncSetAttribute(rk4_stage_kernel<SCHEME, PREC, 4>,                        \
                  cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);                          \
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
                  &n, rk4_stage_kernel<SCHEME, PREC, 4>, block, smem); break;                    \
      default: break;                                                                            \
    }                                                                                            \
    return e == cudaSuccess ? n : -1;                                                            \
  }

}  // namespace cosenu
