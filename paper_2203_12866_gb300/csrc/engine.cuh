// Internal declarations shared by the host translation units of the C ABI:
// the single-grid solver handle (api.cu) and the batched solver (batch.cu).
#pragma once

#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/cosenu.h"
#include "stage_launch.cuh"

namespace cosenu {

// Launch shape of one stage kernel.
struct StageCfg {
  int grid = 0, block = 0, ring = 0, rows_per_slot = 1, slot_bytes = 0;
  int64_t rows = 0;  // z rows per CTA (single-grid launches)
  size_t smem = 0;
};

// Byte offsets of a handle's buffers inside its workspace.
struct Layout {
  size_t y0, y1, y32a, y32b, d1, d2, d3, d4, my, pmom, wtab, zavg, vtab, partial, result, err, total;
};

// One admissible ring shape of a stage kernel: R rows per slot, D slots.
struct RingChoice {
  int rows_per_slot = 0, ring = 0, slot_bytes = 0, occ = 0;
  size_t smem = 0;
  int64_t score = 0;  // bytes per bulk copy per plane x resident CTAs, capped
};

}  // namespace cosenu

// A single-grid solver (opaque to C callers).
struct cosenu_s {
  int64_t nz = 0;
  int32_t nv = 0;
  double L = 0;
  int scheme = 0, precision = 0;
  int vgrid = 0;  // velocity quadrature (COSENU_MIDPOINT, ...)
  cosenu_params p{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool own_mem = false;
  unsigned char* ws = nullptr;
  cosenu::Layout lay{};
  double* y[2] = {nullptr, nullptr};
  float* y32[2] = {nullptr, nullptr};  // mixed: float copy of y[0]
  int ycur = 0;
  void* d[4] = {nullptr, nullptr, nullptr, nullptr};  // delta_1..3 (mixed: and delta_4)
  double* my = nullptr;
  float4* pmom = nullptr;  // mixed: weighted v-sums of the step's increment per plane-row (float pairs)
  float* wtab = nullptr;   // mixed: w_j and w_j v_j as float pairs (hi [2][nv], lo [2][nv])
  double* vtab = nullptr;  // beam velocities [nv] and quadrature weights [nv]
  uint32_t* err = nullptr;
  cosenu::StageCfg cfg[5];
  int nsm = 0;
  cudaGraphExec_t graph = nullptr;  // two RK4 steps starting from y[0]
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;                         // reusable events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[6];  // per kernel: (start, stop)
  int64_t steps = 0;
  bool in_batch = false;  // created by a batch: stepped, streamed and destroyed by it
  uint64_t version = 0;   // bumped by every parameter change
  std::string error;
};

namespace cosenu {

void set_thread_error(const std::string& msg);  // message for cosenu_last_error(NULL)
void count_launches(int n);                     // cosenu_kernel_launches counter

// Threads of a stage kernel for nv velocity bins: consumer warps for 2 nv
// columns (2 columns per thread for FD4+KO, 1 for WENO7), a producer and a reducer warp.
int stage_block(int scheme, int precision, int nv, int stage);

// Halo rows a CTA's march reads besides its own z range (below and above).
int stage_halo_rows(int scheme);

// Admissible ring shapes of one stage kernel, best first: the largest copy
// size per plane times resident CTAs (capped at 4 KB), then the most resident
// CTAs, then the deepest ring.  Empty if none fits; *query_failed is set if an
// occupancy query failed.
std::vector<RingChoice> ring_choices(int scheme, int precision, int nv, int stage, bool batched,
                                     bool* query_failed);

// Every pointer a stage kernel dereferences is set (a launch with a missing
// buffer is refused instead of faulting on the device).
bool stage_args_complete(int precision, int stage, const StageArgs& a);

// Launch one stage kernel of the given (scheme, precision); bt == nullptr is a
// single-grid launch.  Refuses arguments with a missing buffer.
cudaError_t launch_stage_kernel(int scheme, int precision, int stage, const StageArgs& a,
                                const BatchTable* bt, int grid, int block, size_t smem,
                                cudaStream_t stream);

// A handle on `stream` (owned by the caller), for batches.  NULL on failure
// (reason in the thread's error message).
cosenu_t create_member(int64_t nz, int32_t nv, double L, int scheme, int precision,
                       cudaStream_t stream);
// Release a handle and the device memory it allocated (waits for its stream).
void destroy_member(cosenu_t h);

// Arguments of stage `stage` of a handle whose current state buffer is `ycur`
// (launch-shape fields from h->cfg).
StageArgs stage_args(const cosenu_s* h, int stage, int ycur);

// The handle's state and buffers as one segment of the increment kernels (mixed).
struct ApplySeg;
ApplySeg apply_seg(const cosenu_s* h);

// Wait for the batch's stream; (*flags)[i] = error bits of member i (then
// cleared on the device).
int batch_member_flags(cosenu_batch_t b, std::vector<uint32_t>* flags);

// The state buffer that follows a step from `ycur` (the mixed path updates in place).
inline int next_y(const cosenu_s* h, int ycur) {
  return h->precision == COSENU_FP64 ? ycur ^ 1 : ycur;
}

}  // namespace cosenu
