// Declarations of the reduction kernels (diag_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cosenu_device.cuh"

namespace cosenu {

constexpr int kDiagBlock = 256;
constexpr int kDiagMaxBlocks = 1024;
constexpr int kApplyGroups = 1024;  // float4 groups per chunk of the increment kernels
constexpr int kApplyThreads = 256;
constexpr int kFoldRows = 1024;     // z rows per block of the batched moment fold

// One mixed-precision state for the increment kernels.  The flat arrays are
// [species][component][z][v]; a plane-row is one (species, component, z) run of
// nv values, and a chunk is rows_per_chunk whole plane-rows (nv / 4 float4
// groups each, at most kApplyGroups in all).
struct ApplySeg {
  double* y;
  float* y32;
  const float* d[4];    // the four stage increments
  float4* pmom;         // [8 nz] per plane-row: sum_j w_j dy_j, sum_j w_j v_j dy_j as
                        // float pairs (hi, lo, hi, lo)
  const float* wtab;    // [4][nv]: the double weights w_j, w_j v_j of the quadrature as
                        // float pairs: high parts [0], [1], low parts [2], [3]
  double* my;           // [nz][8] running FP64 v-moments of y
  int64_t nz;
  int32_t nv;
  int32_t rows_per_chunk;
  int64_t nchunks;      // ceil(8 nz / rows_per_chunk)
  uint32_t* err;
  float w3, w6;         // dy = (delta_1 + 2 delta_2 + delta_3) w3 + delta_4 w6: 1/3 and 1/6
                        // divided by the scale the stages store their increments in
};

// One FP64 state for the FP64 increment kernel: n2 = 4 nz nv double2 groups.
struct ApplySeg64 {
  const double* y_in;
  double* y_out;
  const double* d[4];  // the four stage increments
  int64_t n2;
  uint32_t* err;
};

// Plane-rows per chunk of a grid with nv beams.
inline int apply_rows_per_chunk(int nv) { return kApplyGroups / (nv / 4); }

__global__ void ymoments_kernel(const double* __restrict__ y, int64_t nz, int nv,
                                double* __restrict__ out, int stride, int vgrid);
__global__ void y32_moments_kernel(const double* __restrict__ y, float* __restrict__ y32,
                                   int64_t nz, int nv, const double* __restrict__ vtab,
                                   double* __restrict__ my);
__global__ void apply_increment_kernel(ApplySeg sg);
__global__ void apply_increment_batch_kernel(const ApplySeg* __restrict__ segs,
                                             const int64_t* __restrict__ chunk_first, int nseg,
                                             int64_t nchunks);
__global__ void apply_increment_fp64_kernel(const double* __restrict__ y_in,
                                            double* __restrict__ y_out,
                                            const double* __restrict__ d1,
                                            const double* __restrict__ d2,
                                            const double* __restrict__ d3,
                                            const double* __restrict__ d4, int64_t n2,
                                            uint32_t* err);
__global__ void apply_increment_fp64_batch_kernel(const ApplySeg64* __restrict__ segs,
                                                  const int64_t* __restrict__ chunk_first,
                                                  int nseg, int64_t nchunks);
__global__ void fold_moments_kernel(double* __restrict__ my, const float4* __restrict__ pmom,
                                    int64_t nz);
__global__ void fold_moments_batch_kernel(const ApplySeg* __restrict__ segs,
                                          const int64_t* __restrict__ block_first, int nseg,
                                          int64_t nblocks);
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
