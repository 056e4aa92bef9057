// Declarations of the reduction kernels (diag_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cosenu {

constexpr int kDiagBlock = 256;
constexpr int kDiagMaxBlocks = 1024;

__global__ void ymoments_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out, int stride);
__global__ void y32_from_y_kernel(const double* __restrict__ y, float* __restrict__ y32,
                                  int64_t n);
__global__ void apply_increment_kernel(double* __restrict__ y, float* __restrict__ y32,
                                       const float* __restrict__ dy, int64_t n, uint32_t* err);
__global__ void zavg_kernel(const double* __restrict__ y, int64_t nz, int nv,
                            double* __restrict__ out);
__global__ void conserved_partial_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                         double* __restrict__ partial);
__global__ void conserved_final_kernel(const double* __restrict__ partial, int nblocks,
                                       double* __restrict__ out);

}  // namespace cosenu
