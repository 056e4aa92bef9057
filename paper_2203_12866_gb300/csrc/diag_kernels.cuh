// Declarations of the reduction kernels (diag_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cosenu_device.cuh"

namespace cosenu {

constexpr int kDiagBlock = 256;
constexpr int kDiagMaxBlocks = 1024;
constexpr int64_t kApplyChunk4 = 1024;  // float4 groups per chunk of the batched increment

// One state of the batched increment kernel: n4 = 2 nz nv float4 groups.
struct ApplySeg {
  double* y;
  float* y32;
  const float* d[4];  // the four stage increments
  int64_t n4;
  uint32_t* err;
};

__global__ void ymoments_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out, int stride, int vgrid);
__global__ void y32_from_y_kernel(const double* __restrict__ y, float* __restrict__ y32,
                                  int64_t n);
__global__ void apply_increment_kernel(double* __restrict__ y, float* __restrict__ y32,
                                       const float* __restrict__ d1, const float* __restrict__ d2,
                                       const float* __restrict__ d3, const float* __restrict__ d4,
                                       int64_t n, uint32_t* err);
__global__ void apply_increment_batch_kernel(const ApplySeg* __restrict__ segs,
                                             const int64_t* __restrict__ chunk_first, int nseg,
                                             int64_t nchunks);
__global__ void collective_fill_kernel(double* __restrict__ y, int64_t nz, int nv,
                                       const double* __restrict__ g,
                                       const double* __restrict__ ph);
__global__ void gather_flags_kernel(uint32_t* const* __restrict__ flags, int n,
                                    uint32_t* __restrict__ out, int clear);
__global__ void dp_field_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out);
__global__ void dft_beam_kernel(const double* __restrict__ y, int64_t nz, int nv, int s, int j,
                                int64_t m0, double* __restrict__ out);
__global__ void zavg_kernel(const double* __restrict__ y, int64_t nz, int nv,
                            double* __restrict__ out);
__global__ void conserved_partial_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                         double* __restrict__ partial, int vgrid);
__global__ void conserved_final_kernel(const double* __restrict__ partial, int nblocks,
                                       double* __restrict__ out);

}  // namespace cosenu
