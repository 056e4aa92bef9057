// Host-side launcher of the fused RK4 stage kernels; each (scheme, precision)
// pair is instantiated in its own translation unit so the four compile in
// parallel.  `bt` == nullptr launches the single-grid kernel (CTA b owns a
// contiguous z range of the grid in `a`); otherwise the batched kernel walks
// the work items of `*bt`.
#pragma once

#include "stage_kernel.cuh"

namespace cosenu {

constexpr int kStageSmemLimit = 232448;  // opt-in dynamic shared memory per CTA

template <int SCHEME, int PREC>
cudaError_t launch_rk4_stage(int stage, const StageArgs& a, const BatchTable* bt, int grid,
                             int block, size_t smem, cudaStream_t stream);

// Resident CTAs per SM of one stage kernel, or -1 if the query failed.
template <int SCHEME, int PREC>
int stage_max_blocks_per_sm(int stage, bool batched, int block, size_t smem);

namespace detail {

template <int SCHEME, int PREC, int STAGE, bool BATCHED>
cudaError_t set_smem_attr() {
  static bool done = false;  // once per kernel and process
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(rk4_stage_kernel<SCHEME, PREC, STAGE, BATCHED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStageSmemLimit);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int SCHEME, int PREC, int STAGE, bool BATCHED>
cudaError_t launch_one(const StageArgs& a, const BatchTable& bt, int grid, int block,
                       size_t smem, cudaStream_t stream) {
  cudaError_t e = set_smem_attr<SCHEME, PREC, STAGE, BATCHED>();
  if (e != cudaSuccess) return e;
  rk4_stage_kernel<SCHEME, PREC, STAGE, BATCHED><<<grid, block, smem, stream>>>(a, bt);
  return cudaGetLastError();
}

template <int SCHEME, int PREC, int STAGE, bool BATCHED>
int occupancy_one(int block, size_t smem) {
  if (set_smem_attr<SCHEME, PREC, STAGE, BATCHED>() != cudaSuccess) return -1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, rk4_stage_kernel<SCHEME, PREC, STAGE, BATCHED>, block, smem) != cudaSuccess)
    return -1;
  return n;
}

template <int SCHEME, int PREC, int STAGE>
cudaError_t launch_stage_n(const StageArgs& a, const BatchTable* bt, int grid, int block,
                           size_t smem, cudaStream_t stream) {
  if (bt) return launch_one<SCHEME, PREC, STAGE, true>(a, *bt, grid, block, smem, stream);
  return launch_one<SCHEME, PREC, STAGE, false>(a, BatchTable{}, grid, block, smem, stream);
}

template <int SCHEME, int PREC, int STAGE>
int occupancy_n(bool batched, int block, size_t smem) {
  return batched ? occupancy_one<SCHEME, PREC, STAGE, true>(block, smem)
                 : occupancy_one<SCHEME, PREC, STAGE, false>(block, smem);
}

}  // namespace detail

#define COSENU_INSTANTIATE_STAGE(SCHEME, PREC)                                                  \
  template <>                                                                                   \
  cudaError_t launch_rk4_stage<SCHEME, PREC>(int stage, const StageArgs& a,                     \
                                             const BatchTable* bt, int grid, int block,         \
                                             size_t smem, cudaStream_t stream) {                \
    switch (stage) {                                                                            \
      case 1: return detail::launch_stage_n<SCHEME, PREC, 1>(a, bt, grid, block, smem, stream); \
      case 2: return detail::launch_stage_n<SCHEME, PREC, 2>(a, bt, grid, block, smem, stream); \
      case 3: return detail::launch_stage_n<SCHEME, PREC, 3>(a, bt, grid, block, smem, stream); \
      case 4: return detail::launch_stage_n<SCHEME, PREC, 4>(a, bt, grid, block, smem, stream); \
      default: return cudaErrorInvalidValue;                                                    \
    }                                                                                           \
  }                                                                                             \
  template <>                                                                                   \
  int stage_max_blocks_per_sm<SCHEME, PREC>(int stage, bool batched, int block, size_t smem) {  \
    switch (stage) {                                                                            \
      case 1: return detail::occupancy_n<SCHEME, PREC, 1>(batched, block, smem);                \
      case 2: return detail::occupancy_n<SCHEME, PREC, 2>(batched, block, smem);                \
      case 3: return detail::occupancy_n<SCHEME, PREC, 3>(batched, block, smem);                \
      case 4: return detail::occupancy_n<SCHEME, PREC, 4>(batched, block, smem);                \
      default: return -1;                                                                       \
    }                                                                                           \
  }

}  // namespace cosenu
