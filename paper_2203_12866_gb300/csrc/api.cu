// C ABI of the COSEnu GB300 engine (declared in include/cosenu.h).
//
// A handle owns one solver: the state (FP64 path: two ping-pong buffers, the
// increment kernel writing the new state into the other; mixed path: one buffer
// plus its float copy, updated in place by the increment kernel), the four RK4
// stage increments, the per-z running moments of the mixed path, and a small
// reduction scratch area.  cosenu_step() enqueues the four fused stage kernels
// of each RK4 step and the increment kernel (mixed: and the moment fold) on the
// handle's stream; pairs of steps are replayed from a CUDA graph when the
// stream allows capture.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cosenu.h"
#include "diag_kernels.cuh"
#include "engine.cuh"

using namespace cosenu;

namespace {

std::atomic<uint64_t> g_launches{0};
thread_local std::string tl_error;

constexpr size_t kAlign = 256;
// Fewest z rows per CTA of a single-grid launch.  A CTA's march is latency-bound
// per row (and an FP64 CTA of few columns waits on one scheduler's share of the
// FP64 pipe), so a small grid is spread over as many SMs and schedulers as it
// can use.  Measured on the 512 x 32 steps (us per step for 4 / 2 / 1 rows):
// FD4+KO FP64 109 / 66 / 55, FD4+KO mixed 63 / 49 / 54, WENO7 FP64 306 / 222 / 249,
// WENO7 mixed 69 / 78 / 84 (its march takes two rows per iteration); 16 rows gave
// 320 us for FD4+KO FP64.  Grids of more than SMs x resident CTAs x this many rows
// are unaffected.
int64_t min_rows_per_cta(int scheme, int precision) {
  if (scheme == COSENU_WENO7) return precision == COSENU_FP64 ? 2 : 4;
  return precision == COSENU_FP64 ? 1 : 2;  // FD4+KO, r = 2 and 3
}

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool valid_sizes(int64_t nz, int32_t nv, int scheme, int precision) {
  return nz >= 1 && nv >= 4 && nv <= 256 && nv % 4 == 0 &&
         (scheme == COSENU_FDKO || scheme == COSENU_WENO7 || scheme == COSENU_FDKO3) &&
         (precision == COSENU_FP64 || precision == COSENU_MIXED) &&
         nz <= ((int64_t)1 << 40) / ((int64_t)8 * nv);
}

Layout make_layout(int64_t nz, int32_t nv, int precision) {
  Layout L;
  const size_t n = (size_t)8 * nz * nv;
  const size_t dsz = precision == COSENU_FP64 ? sizeof(double) : sizeof(float);
  size_t off = 0;
  L.y0 = off; off = align_up(off + n * sizeof(double));
  const size_t n1 = precision == COSENU_FP64 ? n : 0;    // second state buffer (fp64)
  L.y1 = off; off = align_up(off + n1 * sizeof(double));
  const size_t n32 = precision == COSENU_MIXED ? n : 0;  // float copy of y (mixed)
  L.y32a = off; off = align_up(off + n32 * sizeof(float));
  L.y32b = off;
  L.d1 = off; off = align_up(off + n * dsz);
  L.d2 = off; off = align_up(off + n * dsz);
  L.d3 = off; off = align_up(off + n * dsz);
  L.d4 = off; off = align_up(off + n * dsz);
  L.my = off; off = align_up(off + (size_t)nz * 8 * sizeof(double));
  const size_t npm = precision == COSENU_MIXED ? (size_t)8 * nz : 0;
  L.pmom = off; off = align_up(off + npm * sizeof(float4));
  const size_t nwt = precision == COSENU_MIXED ? (size_t)4 * nv : 0;
  L.wtab = off; off = align_up(off + nwt * sizeof(float));
  L.zavg = off; off = align_up(off + (size_t)8 * nv * sizeof(double));
  L.vtab = off; off = align_up(off + (size_t)2 * nv * sizeof(double));
  L.partial = off; off = align_up(off + (size_t)kDiagMaxBlocks * 8 * sizeof(double));
  L.result = off; off = align_up(off + 8 * sizeof(double));
  L.err = off; off = align_up(off + 64);
  L.total = off;
  return L;
}

}  // namespace

namespace cosenu {
void set_thread_error(const std::string& msg) { tl_error = msg; }
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace cosenu

namespace {

int fail(cosenu_t h, int code, const std::string& msg) {
  if (h)
    h->error = msg;
  else
    tl_error = msg;
  return code;
}

int cuda_fail(cosenu_t h, cudaError_t e, const char* what) {
  return fail(h, COSENU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                  \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

cudaError_t launch_stage(cosenu_t h, int stage, const StageArgs& a) {
  const StageCfg& c = h->cfg[stage];
  cudaError_t e = launch_stage_kernel(h->scheme, h->precision, stage, a, nullptr, c.grid, c.block,
                                      c.smem, h->stream);
  if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// Launch shape of each stage: the best ring shape of ring_choices() and a
// persistent grid of at most SMs x resident CTAs, contiguous z ranges of at
// least min_rows_per_cta() rows.  A shape whose slot holds more than half of the
// rows a CTA marches (its z range and halo) is passed over while a smaller one
// fits: on short grids the march would otherwise wait for one large first copy
// (512 x 32 mixed WENO7 steps: 8-row slots 102 us, 4-row slots 72 us).
int configure(cosenu_t h) {
  int dev = 0, nsm = 0;
  CK(h, cudaGetDevice(&dev));
  CK(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  h->nsm = nsm;
  for (int s = 1; s <= 4; ++s) {
    bool qfail = false;
    const std::vector<RingChoice> rc =
        ring_choices(h->scheme, h->precision, h->nv, s, false, &qfail);
    if (qfail) return fail(h, COSENU_ECUDA, "occupancy query failed");
    if (rc.empty()) return fail(h, COSENU_EINVAL, "grid row does not fit in shared memory");
    const int halo = stage_halo_rows(h->scheme);
    auto shape_for = [&](const RingChoice& ch) {
      StageCfg c;
      c.block = stage_block(h->scheme, h->precision, h->nv, s);
      c.ring = ch.ring;
      c.rows_per_slot = ch.rows_per_slot;
      c.slot_bytes = ch.slot_bytes;
      c.smem = ch.smem;
      const int64_t max_grid = (int64_t)nsm * ch.occ;
      const int64_t min_rows = min_rows_per_cta(h->scheme, h->precision);
      int64_t grid = (h->nz + min_rows - 1) / min_rows;
      if (grid > max_grid) grid = max_grid;
      if (grid < 1) grid = 1;
      c.rows = (h->nz + grid - 1) / grid;
      c.grid = (int)((h->nz + c.rows - 1) / c.rows);
      return c;
    };
    StageCfg c = shape_for(rc.front());
    for (const RingChoice& ch : rc) {
      const StageCfg t = shape_for(ch);
      if (2 * (int64_t)t.rows_per_slot <= t.rows + halo) {
        c = t;
        break;
      }
    }
    h->cfg[s] = c;
  }
  return COSENU_OK;
}

}  // namespace

namespace cosenu {

namespace {

// Per-stage launch traits of a (scheme, precision) pair.
struct StageTraits {
  int cols, header, max_ring_rows;
  int (*reducers)(int ncw);  // reducer warps for ncw consumer warps
};

template <int SCHEME, int PREC, int STAGE>
StageTraits traits_of() {
  return {stage_cols<SCHEME, PREC, STAGE>(), stage_smem_header_bytes<SCHEME, PREC, STAGE>(),
          stage_max_ring_rows<SCHEME, PREC>(), &stage_reducer_warps<SCHEME, PREC>};
}

template <int SCHEME, int PREC>
StageTraits traits_for_stage(int stage) {
  switch (stage) {
    case 1: return traits_of<SCHEME, PREC, 1>();
    case 2: return traits_of<SCHEME, PREC, 2>();
    case 3: return traits_of<SCHEME, PREC, 3>();
    default: return traits_of<SCHEME, PREC, 4>();
  }
}

StageTraits stage_traits(int scheme, int precision, int stage) {
  if (scheme == COSENU_FDKO)
    return precision == COSENU_FP64 ? traits_for_stage<kFDKO, kFP64>(stage)
                                    : traits_for_stage<kFDKO, kMIXED>(stage);
  if (scheme == COSENU_FDKO3)
    return precision == COSENU_FP64 ? traits_for_stage<kFDKO3, kFP64>(stage)
                                    : traits_for_stage<kFDKO3, kMIXED>(stage);
  return precision == COSENU_FP64 ? traits_for_stage<kWENO7, kFP64>(stage)
                                  : traits_for_stage<kWENO7, kMIXED>(stage);
}

int max_blocks(int scheme, int precision, int stage, bool batched, int block, size_t smem) {
  if (scheme == COSENU_FDKO && precision == COSENU_FP64)
    return stage_max_blocks_per_sm<kFDKO, kFP64>(stage, batched, block, smem);
  if (scheme == COSENU_FDKO)
    return stage_max_blocks_per_sm<kFDKO, kMIXED>(stage, batched, block, smem);
  if (scheme == COSENU_FDKO3)
    return precision == COSENU_FP64
               ? stage_max_blocks_per_sm<kFDKO3, kFP64>(stage, batched, block, smem)
               : stage_max_blocks_per_sm<kFDKO3, kMIXED>(stage, batched, block, smem);
  if (precision == COSENU_FP64)
    return stage_max_blocks_per_sm<kWENO7, kFP64>(stage, batched, block, smem);
  return stage_max_blocks_per_sm<kWENO7, kMIXED>(stage, batched, block, smem);
}

int slot_bytes_of(int precision, int nv, int stage, int rows) {
  return precision == COSENU_FP64 ? slot_layout<kFP64>(nv, stage, rows).bytes
                                  : slot_layout<kMIXED>(nv, stage, rows).bytes;
}

}  // namespace

// Every pointer a stage kernel dereferences must be set (a launch with a
// missing buffer is refused instead of faulting on the device).
bool stage_args_complete(int precision, int stage, const StageArgs& a) {
  const bool mixed = precision == COSENU_MIXED;
  if (!a.err || !a.vtab || (mixed ? !a.y32_in || !a.my : !a.y_in)) return false;
  if (stage > 1 && !a.d_in) return false;
  if (!a.d_out) return false;
  return true;
}

int stage_halo_rows(int scheme) {
  if (scheme == COSENU_FDKO) return Scheme<kFDKO>::kLo + Scheme<kFDKO>::kHi;
  if (scheme == COSENU_FDKO3) return Scheme<kFDKO3>::kLo + Scheme<kFDKO3>::kHi;
  return Scheme<kWENO7>::kLo + Scheme<kWENO7>::kHi;
}

int stage_block(int scheme, int precision, int nv, int stage) {
  const StageTraits t = stage_traits(scheme, precision, stage);
  const int ncw = (2 * nv + 32 * t.cols - 1) / (32 * t.cols);
  return (ncw + 1 + t.reducers(ncw)) * 32;
}

// Ring shapes: R z rows per slot (one bulk copy per component plane moves R
// rows) and D >= 2 slots.  Bandwidth depends mostly on the contiguous bytes
// each bulk copy moves per component plane (R rows of nv values) times the
// resident CTAs: ~1 KB per copy reaches about 40% of HBM peak, 2 KB with two
// CTAs or 4 KB with one about 95% (measured on GB300).
std::vector<RingChoice> ring_choices(int scheme, int precision, int nv, int stage, bool batched,
                                     bool* query_failed) {
  std::vector<RingChoice> out;
  *query_failed = false;
  const StageTraits t = stage_traits(scheme, precision, stage);
  const int header = t.header;
  const int block = stage_block(scheme, precision, nv, stage);
  for (int R = 1; R <= 32; R *= 2) {
    const int slot = slot_bytes_of(precision, nv, stage, R);
    for (int D = 2; D <= kMaxRing; ++D) {
      // The warps of a CTA drift apart by at most D * R rows, which the moment
      // slots bound (stage_max_ring_rows).
      if (D * R > t.max_ring_rows) break;
      const size_t smem = (size_t)header + (size_t)D * slot;
      if (smem > (size_t)kStageSmemLimit) break;
      const int occ = max_blocks(scheme, precision, stage, batched, block, smem);
      if (occ < 0) {
        *query_failed = true;
        return {};
      }
      if (occ == 0) continue;
      RingChoice c;
      c.rows_per_slot = R;
      c.ring = D;
      c.slot_bytes = slot;
      c.occ = occ;
      c.smem = smem;
      c.score = std::min<int64_t>((int64_t)R * nv * 4 * occ, 4096);
      out.push_back(c);
    }
  }
  std::stable_sort(out.begin(), out.end(), [](const RingChoice& x, const RingChoice& y) {
    if (x.score != y.score) return x.score > y.score;
    if (x.occ != y.occ) return x.occ > y.occ;
    return x.ring > y.ring;
  });
  return out;
}

cudaError_t launch_stage_kernel(int scheme, int precision, int stage, const StageArgs& a,
                                const BatchTable* bt, int grid, int block, size_t smem,
                                cudaStream_t stream) {
  if (!bt && !stage_args_complete(precision, stage, a)) return cudaErrorInvalidValue;
  if (scheme == COSENU_FDKO && precision == COSENU_FP64)
    return launch_rk4_stage<kFDKO, kFP64>(stage, a, bt, grid, block, smem, stream);
  if (scheme == COSENU_FDKO)
    return launch_rk4_stage<kFDKO, kMIXED>(stage, a, bt, grid, block, smem, stream);
  if (scheme == COSENU_FDKO3)
    return precision == COSENU_FP64
               ? launch_rk4_stage<kFDKO3, kFP64>(stage, a, bt, grid, block, smem, stream)
               : launch_rk4_stage<kFDKO3, kMIXED>(stage, a, bt, grid, block, smem, stream);
  if (precision == COSENU_FP64)
    return launch_rk4_stage<kWENO7, kFP64>(stage, a, bt, grid, block, smem, stream);
  return launch_rk4_stage<kWENO7, kMIXED>(stage, a, bt, grid, block, smem, stream);
}

StageArgs stage_args(const cosenu_s* h, int stage, int ycur) {
  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nz = h->nz;
  a.nv = h->nv;
  a.ncols = 2 * h->nv;
  a.rows_per_cta = h->cfg[stage].rows;
  a.ring = h->cfg[stage].ring;
  a.rows_per_slot = h->cfg[stage].rows_per_slot;
  a.slot_bytes = h->cfg[stage].slot_bytes;
  a.vtab = h->vtab;
  a.inv_dz = (double)h->nz / h->L;
  a.dt = h->p.dt;
  a.mu = h->p.mu;
  a.hvac_d = -h->p.omega * std::cos(2.0 * h->p.theta);
  a.hvac_r = 0.5 * h->p.omega * std::sin(2.0 * h->p.theta);
  a.lambda = h->p.lambda;
  a.ko_eps = h->p.ko_eps;
  a.weno_eps = h->p.weno_eps;
  a.y_in = h->y[ycur];
  a.y32_in = h->y32[0];
  a.my = h->my;
  a.err = h->err;
  switch (stage) {
    case 1: a.d_out = h->d[0]; break;
    case 2: a.d_in = h->d[0]; a.d_out = h->d[1]; break;
    case 3: a.d_in = h->d[1]; a.d_out = h->d[2]; break;
    default:
      a.d_in = h->d[2]; a.d_out = h->d[3]; break;
  }
  return a;
}

// The mixed path's increment kernels of one handle.
ApplySeg apply_seg(const cosenu_s* h) {
  ApplySeg sg;
  sg.y = h->y[0];
  sg.y32 = h->y32[0];
  for (int k = 0; k < 4; ++k) sg.d[k] = static_cast<const float*>(h->d[k]);
  sg.pmom = h->pmom;
  sg.wtab = h->wtab;
  sg.my = h->my;
  sg.nz = h->nz;
  sg.nv = h->nv;
  sg.rows_per_chunk = apply_rows_per_chunk(h->nv);
  sg.nchunks = (8 * h->nz + sg.rows_per_chunk - 1) / sg.rows_per_chunk;
  sg.err = h->err;
  // the mixed WENO7 stages store their increments times kWenoScale
  const double inv = h->scheme == COSENU_WENO7 ? kWenoInvScale : 1.0;
  sg.w3 = (float)(inv / 3.0);
  sg.w6 = (float)(inv / 6.0);
  return sg;
}

}  // namespace cosenu

namespace {

cudaError_t take_event(cosenu_t h, cudaEvent_t* out) {
  if (!h->ev_free.empty()) {
    *out = h->ev_free.back();
    h->ev_free.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(out);
}


// End of an RK4 step.  FP64 (kernel 5): y[ycur ^ 1] = y[ycur] + the step's
// increment.  Mixed: y <- y + dy in place with the plane-row v-sums of dy
// (kernel 5), then the running FP64 moments of y advanced by them (kernel 6).
cudaError_t launch_apply(cosenu_t h, int k, int ycur) {
  if (h->precision == COSENU_FP64) {
    const int64_t n2 = 4 * h->nz * (int64_t)h->nv;  // double2 groups
    const int64_t blocks = std::min<int64_t>((n2 + 255) / 256, (int64_t)h->nsm * 8);
    apply_increment_fp64_kernel<<<(int)blocks, 256, 0, h->stream>>>(
        h->y[ycur], h->y[ycur ^ 1], static_cast<const double*>(h->d[0]),
        static_cast<const double*>(h->d[1]), static_cast<const double*>(h->d[2]),
        static_cast<const double*>(h->d[3]), n2, h->err);
  } else if (k == 5) {
    const ApplySeg sg = apply_seg(h);
    const int64_t blocks = std::min<int64_t>(sg.nchunks, (int64_t)h->nsm * 8);
    apply_increment_kernel<<<(int)blocks, kApplyThreads, 0, h->stream>>>(sg);
  } else {
    const int64_t blocks = std::min<int64_t>((h->nz + 255) / 256, (int64_t)h->nsm * 8);
    fold_moments_kernel<<<(int)blocks, 256, 0, h->stream>>>(h->my, h->pmom, h->nz);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// One RK4 step: stages 1-4, the increment kernel and (mixed) the moment fold.
// Kernels 1..5 of the step (stages, increment) are bracketed by events when
// timing is on; the fold (a few hundredths of a millisecond) is not.
cudaError_t enqueue_step(cosenu_t h, int ycur) {
  const int nk = h->precision == COSENU_MIXED ? 6 : 5;
  for (int s = 1; s <= nk; ++s) {
    if (s == 6) {
      cudaError_t e = launch_apply(h, 6, ycur);
      if (e != cudaSuccess) return e;
      continue;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->timing) {
      cudaError_t e = take_event(h, &e0);
      if (e == cudaSuccess) e = take_event(h, &e1);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = s <= 4 ? launch_stage(h, s, stage_args(h, s, ycur)) : launch_apply(h, 5, ycur);
    if (e != cudaSuccess) return e;
    if (h->timing) {
      e = cudaEventRecord(e1, h->stream);
      if (e != cudaSuccess) return e;
      h->ev[s].push_back({e0, e1});
    }
  }
  return cudaSuccess;
}

void drop_graph(cosenu_t h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
}

// Capture two RK4 steps starting from y[0] (they end in y[0] again).
int build_graph(cosenu_t h) {
  if (h->stream == nullptr) return COSENU_OK;  // the legacy stream cannot be captured
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const uint64_t before = g_launches.load();
  cudaError_t e = enqueue_step(h, 0);
  if (e == cudaSuccess) e = enqueue_step(h, next_y(h, 0));
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
  g_launches.store(before);  // captured launches run later, counted per replay
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e, "stage launch during capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return cuda_fail(h, e, "cudaGraphInstantiate");
  }
  return COSENU_OK;
}

void default_params(cosenu_t h) {
  h->p.mu = 1.0;
  h->p.omega = 0.0;
  h->p.theta = 0.0;
  h->p.lambda = 0.0;
  h->p.ko_eps = 0.1;
  h->p.weno_eps = 1e-6;
  h->p.dt = 0.4 * h->L / (double)h->nz;
}

// The beam velocities and weights of the handle's quadrature into its device
// table (the stage kernels read them once per column).
cudaError_t upload_vtab(cosenu_t h) {
  const size_t nv = (size_t)h->nv;
  std::vector<double> t(2 * nv);
  // mixed: w_j and w_j v_j (double) as float pairs hi + lo, hi = float(x), lo = float(x - hi)
  std::vector<float> w(4 * nv);
  for (size_t j = 0; j < nv; ++j) {
    t[j] = vgrid_v((int)j, h->nv, h->vgrid);
    t[nv + j] = vgrid_w((int)j, h->nv, h->vgrid);
    const double x[2] = {t[nv + j], t[nv + j] * t[j]};
    for (int k = 0; k < 2; ++k) {
      const float hi = (float)x[k];
      w[k * nv + j] = hi;
      w[(2 + k) * nv + j] = (float)(x[k] - (double)hi);
    }
  }
  cudaError_t e = cudaMemcpyAsync(h->vtab, t.data(), t.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->wtab)
    e = cudaMemcpyAsync(h->wtab, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // t, w die here
  return e;
}

cosenu_t create_common(int64_t nz, int32_t nv, double L, int scheme, int precision,
                       void* workspace, size_t ws_bytes, cudaStream_t stream = nullptr) {
  if (!valid_sizes(nz, nv, scheme, precision) || !(L > 0.0) || !std::isfinite(L)) {
    fail(nullptr, COSENU_EINVAL,
         "invalid grid: need nz >= 1, 4 <= nv <= 256, nv % 4 == 0, L > 0, known scheme/precision");
    return nullptr;
  }
  cosenu_t h = new (std::nothrow) cosenu_s;
  if (!h) {
    fail(nullptr, COSENU_ENOMEM, "host allocation failed");
    return nullptr;
  }
  h->nz = nz;
  h->nv = nv;
  h->L = L;
  h->scheme = scheme;
  h->precision = precision;
  default_params(h);
  h->lay = make_layout(nz, nv, precision);
  auto bail = [&](const std::string& why, int code) -> cosenu_t {
    fail(nullptr, code, why + (h->error.empty() ? "" : (": " + h->error)));
    if (h->own_mem && h->ws) cudaFree(h->ws);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return nullptr;
  };
  if (workspace) {
    if (ws_bytes < h->lay.total || ((uintptr_t)workspace % kAlign) != 0)
      return bail("workspace too small or not 256-byte aligned", COSENU_EINVAL);
    h->ws = static_cast<unsigned char*>(workspace);
  } else {
    cudaError_t e = cudaMalloc(&h->ws, h->lay.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->ws = nullptr;
      return bail(std::string("cudaMalloc of the workspace failed: ") + cudaGetErrorString(e),
                  COSENU_ENOMEM);
    }
    h->own_mem = true;
  }
  cudaError_t e = cudaSuccess;
  if (stream) {
    h->stream = stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess)
      return bail(std::string("stream: ") + cudaGetErrorString(e), COSENU_ECUDA);
    h->own_stream = true;
  }
  h->y[0] = reinterpret_cast<double*>(h->ws + h->lay.y0);
  if (precision == COSENU_FP64)
    h->y[1] = reinterpret_cast<double*>(h->ws + h->lay.y1);
  else
    h->y32[0] = reinterpret_cast<float*>(h->ws + h->lay.y32a);
  h->d[0] = h->ws + h->lay.d1;
  h->d[1] = h->ws + h->lay.d2;
  h->d[2] = h->ws + h->lay.d3;
  h->d[3] = h->ws + h->lay.d4;
  if (precision == COSENU_MIXED) {
    h->pmom = reinterpret_cast<float4*>(h->ws + h->lay.pmom);
    h->wtab = reinterpret_cast<float*>(h->ws + h->lay.wtab);
  }
  h->my = reinterpret_cast<double*>(h->ws + h->lay.my);
  h->err = reinterpret_cast<uint32_t*>(h->ws + h->lay.err);
  h->vtab = reinterpret_cast<double*>(h->ws + h->lay.vtab);
  if (configure(h) != COSENU_OK) return bail("launch configuration failed", COSENU_ECUDA);
  e = cudaMemsetAsync(h->ws, 0, h->lay.total, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = upload_vtab(h);
  if (e != cudaSuccess) return bail(std::string("memset: ") + cudaGetErrorString(e), COSENU_ECUDA);
  return h;
}

// After the state was replaced: the mixed path's float copy of y and its
// running FP64 moments.
cudaError_t refresh_moments(cosenu_t h) {
  if (h->precision != COSENU_MIXED) return cudaSuccess;
  y32_moments_kernel<<<(int)std::min<int64_t>((h->nz + 7) / 8, (int64_t)h->nsm * 8), 256, 0,
                       h->stream>>>(h->y[0], h->y32[0], h->nz, h->nv, h->vtab, h->my);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

int check_n(cosenu_t h, size_t n) {
  if ((int64_t)n != 8 * h->nz * (int64_t)h->nv)
    return fail(h, COSENU_EINVAL, "state length must be 8 * nz * nv");
  return COSENU_OK;
}

}  // namespace

extern "C" {

size_t cosenu_workspace_bytes(int64_t nz, int32_t nv, int scheme, int precision) {
  if (!valid_sizes(nz, nv, scheme, precision)) return 0;
  return make_layout(nz, nv, precision).total;
}

cosenu_t cosenu_create(int64_t nz, int32_t nv, double L, int scheme, int precision) {
  return create_common(nz, nv, L, scheme, precision, nullptr, 0);
}

cosenu_t cosenu_create_external(int64_t nz, int32_t nv, double L, int scheme, int precision,
                                void* workspace, size_t workspace_bytes) {
  if (!workspace) {
    fail(nullptr, COSENU_EINVAL, "workspace is NULL");
    return nullptr;
  }
  return create_common(nz, nv, L, scheme, precision, workspace, workspace_bytes);
}

void cosenu_destroy(cosenu_t h) {
  if (!h) return;
  if (h->in_batch) {
    fail(nullptr, COSENU_EINVAL, "cosenu_destroy: the handle belongs to a batch (cosenu_batch_remove)");
    return;
  }
  destroy_member(h);
}

}  // extern "C"

namespace cosenu {

cosenu_t create_member(int64_t nz, int32_t nv, double L, int scheme, int precision,
                       cudaStream_t stream) {
  if (!stream) {
    fail(nullptr, COSENU_EINVAL, "create_member: NULL stream");
    return nullptr;
  }
  cosenu_t h = create_common(nz, nv, L, scheme, precision, nullptr, 0, stream);
  if (h) h->in_batch = true;
  return h;
}

void destroy_member(cosenu_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  for (int s = 1; s <= 5; ++s)
    for (auto& pr : h->ev[s]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
  if (h->own_mem && h->ws) cudaFree(h->ws);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // namespace cosenu

extern "C" {

int cosenu_set_params(cosenu_t h, const cosenu_params* p) {
  if (!h || !p) return fail(h, COSENU_EINVAL, "NULL argument");
  const double vals[7] = {p->mu, p->omega, p->theta, p->lambda, p->ko_eps, p->weno_eps, p->dt};
  for (double x : vals)
    if (!std::isfinite(x)) return fail(h, COSENU_EINVAL, "parameters must be finite");
  if (p->weno_eps <= 0.0) return fail(h, COSENU_EINVAL, "weno_eps must be positive");
  if (p->ko_eps < 0.0) return fail(h, COSENU_EINVAL, "ko_eps must be non-negative");
  h->p = *p;
  if (h->p.dt <= 0.0) h->p.dt = 0.4 * h->L / (double)h->nz;
  ++h->version;
  drop_graph(h);
  return COSENU_OK;
}

int cosenu_set_quadrature(cosenu_t h, int32_t mode) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  if (mode != COSENU_MIDPOINT && mode != COSENU_TRAPEZOID && mode != COSENU_SIMPSON)
    return fail(h, COSENU_EINVAL, "unknown quadrature");
  if (mode == h->vgrid) return COSENU_OK;
  CK(h, cudaStreamSynchronize(h->stream));  // queued steps read the old table
  h->vgrid = mode;
  ++h->version;
  drop_graph(h);
  CK(h, upload_vtab(h));
  CK(h, refresh_moments(h));  // the mixed path's running moments use the weights
  return COSENU_OK;
}

int cosenu_velocities(cosenu_t h, double* v, double* w) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  for (int j = 0; j < h->nv; ++j) {
    if (v) v[j] = vgrid_v(j, h->nv, h->vgrid);
    if (w) w[j] = vgrid_w(j, h->nv, h->vgrid);
  }
  return COSENU_OK;
}

int cosenu_get_params(cosenu_t h, cosenu_params* p) {
  if (!h || !p) return fail(h, COSENU_EINVAL, "NULL argument");
  *p = h->p;
  return COSENU_OK;
}

int cosenu_set_stream(cosenu_t h, void* stream) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  if (h->in_batch) return fail(h, COSENU_EINVAL, "a batch member uses the batch's stream");
  CK(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = static_cast<cudaStream_t>(stream);
  return COSENU_OK;
}

int cosenu_set_state(cosenu_t h, const double* host, size_t n) {
  if (!h || !host) return fail(h, COSENU_EINVAL, "NULL argument");
  if (int rc = check_n(h, n)) return rc;
  h->ycur = 0;
  CK(h, cudaMemcpyAsync(h->y[0], host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(h, refresh_moments(h));
  CK(h, cudaMemsetAsync(h->err, 0, 64, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->steps = 0;
  return COSENU_OK;
}

int cosenu_set_state_device(cosenu_t h, const double* dev, size_t n) {
  if (!h || !dev) return fail(h, COSENU_EINVAL, "NULL argument");
  if (int rc = check_n(h, n)) return rc;
  h->ycur = 0;
  CK(h, cudaMemcpyAsync(h->y[0], dev, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(h, refresh_moments(h));
  CK(h, cudaMemsetAsync(h->err, 0, 64, h->stream));
  h->steps = 0;
  return COSENU_OK;
}

int cosenu_set_state_collective(cosenu_t h, double alpha, double sigma_nu, double sigma_nubar,
                                double eps0, uint64_t seed) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  if (!std::isfinite(alpha) || !std::isfinite(eps0) || !(sigma_nu > 0.0) ||
      !(sigma_nubar > 0.0) || !std::isfinite(sigma_nu) || !std::isfinite(sigma_nubar))
    return fail(h, COSENU_EINVAL, "need finite alpha, eps0 and positive finite sigmas");
  const int64_t nz = h->nz;
  const int nv = h->nv;
  // the two species' angular factors g_nu(v) and alpha g_nubar(v), normalised on the bins
  std::vector<double> hv((size_t)2 * nv + (size_t)2 * nz);
  for (int s = 0; s < 2; ++s) {
    const double sig = s == 0 ? sigma_nu : sigma_nubar;
    double norm = 0.0;  // sum_j w_j g(v_j)
    for (int j = 0; j < nv; ++j) {
      const double v = vgrid_v(j, nv, h->vgrid);
      hv[(size_t)s * nv + j] = std::exp(-((v - 1.0) * (v - 1.0)) / (2.0 * sig * sig));
    }
    if (h->vgrid == kVgridMidpoint) {  // equal weights: sum first, then scale
      double sum = 0.0;
      for (int j = 0; j < nv; ++j) sum += hv[(size_t)s * nv + j];
      norm = sum * (2.0 / nv);
    } else {
      for (int j = 0; j < nv; ++j) norm += vgrid_w(j, nv, h->vgrid) * hv[(size_t)s * nv + j];
    }
    for (int j = 0; j < nv; ++j)
      hv[(size_t)s * nv + j] = (s == 0 ? 1.0 : alpha) * (hv[(size_t)s * nv + j] / norm);
  }
  // off-diagonal seed eps0 exp(i phi(z)), phi = 2 pi u, u = (splitmix64(z ^ seed) >> 11) 2^-53
  double* ph = hv.data() + (size_t)2 * nv;
  for (int64_t z = 0; z < nz; ++z) {
    uint64_t x = ((uint64_t)z ^ seed) + 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    const double phi = 2.0 * M_PI * ((double)(x >> 11) * 0x1.0p-53);
    ph[z] = eps0 * std::cos(phi);
    ph[nz + z] = eps0 * std::sin(phi);
  }
  // the factors go through the delta_1 buffer (free between steps; 32 nz nv >= 16 (nz + nv) bytes)
  double* dev = static_cast<double*>(h->d[0]);
  h->ycur = 0;
  CK(h, cudaMemcpyAsync(dev, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream));
  const int64_t n = 8 * nz * (int64_t)nv;
  collective_fill_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, h->stream>>>(
      h->y[0], nz, nv, dev, dev + 2 * nv);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CK(h, cudaGetLastError());
  CK(h, refresh_moments(h));
  CK(h, cudaMemsetAsync(h->err, 0, 64, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));  // hv dies here
  h->steps = 0;
  return COSENU_OK;
}

int cosenu_get_state(cosenu_t h, double* host, size_t n) {
  if (!h || !host) return fail(h, COSENU_EINVAL, "NULL argument");
  if (int rc = check_n(h, n)) return rc;
  CK(h, cudaMemcpyAsync(host, h->y[h->ycur], n * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

int cosenu_get_rows(cosenu_t h, int64_t z0, int64_t nrows, double* host) {
  if (!h || !host) return fail(h, COSENU_EINVAL, "NULL argument");
  if (z0 < 0 || nrows < 0 || z0 + nrows > h->nz) return fail(h, COSENU_EINVAL, "rows out of range");
  if (nrows == 0) return COSENU_OK;
  const size_t rowb = (size_t)h->nv * sizeof(double);
  // 8 planes of nz rows -> 8 blocks of nrows rows
  CK(h, cudaMemcpy2DAsync(host, nrows * rowb, h->y[h->ycur] + z0 * h->nv, h->nz * rowb,
                          nrows * rowb, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

const double* cosenu_state_device(cosenu_t h) { return h ? h->y[h->ycur] : nullptr; }

int cosenu_step(cosenu_t h, int64_t nsteps) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(h, COSENU_EINVAL, "nsteps must be >= 0");
  int64_t left = nsteps;
  if (left >= 2 && !h->graph && h->stream && !h->timing) {
    if (int rc = build_graph(h)) return rc;
  }
  if (left >= 2 && h->graph && !h->timing) {
    if (h->ycur == 1) {  // the graph starts from y[0]
      CK(h, enqueue_step(h, 1));
      h->ycur = 0;
      --left;
    }
    for (; left >= 2; left -= 2) {
      CK(h, cudaGraphLaunch(h->graph, h->stream));
      // two steps of 6 (mixed: stages, increment, moment fold) or 5 (FP64) kernels
      g_launches.fetch_add(h->precision == COSENU_MIXED ? 12 : 10, std::memory_order_relaxed);
    }
  }
  for (; left > 0; --left) {
    CK(h, enqueue_step(h, h->ycur));
    h->ycur = next_y(h, h->ycur);
  }
  h->steps += nsteps;
  return COSENU_OK;
}

int cosenu_sync(cosenu_t h) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  uint32_t flags = 0;
  CK(h, cudaMemcpyAsync(&flags, h->err, sizeof(flags), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (flags) {
    CK(h, cudaMemsetAsync(h->err, 0, 64, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (flags & kErrTimeout) return fail(h, COSENU_ETIMEOUT, "a device-side wait gave up");
    return fail(h, COSENU_ENONFINITE, "non-finite value in the state");
  }
  return COSENU_OK;
}

int cosenu_moments(cosenu_t h, double* zavg, double* vmom) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  const double* y = h->y[h->ycur];
  if (zavg) {
    double* dz = reinterpret_cast<double*>(h->ws + h->lay.zavg);
    zavg_kernel<<<dim3((h->nv + 31) / 32, 8), 256, 0, h->stream>>>(y, h->nz, h->nv, dz);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(zavg, dz, (size_t)8 * h->nv * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
  }
  if (vmom) {
    // staged in the delta_1 buffer (free between steps), row stride 8
    double* dm = reinterpret_cast<double*>(h->d[0]);
    ymoments_kernel<<<(int)std::min<int64_t>((h->nz + 7) / 8, 65535), 256, 0, h->stream>>>(
        y, h->nz, h->nv, dm, 8, h->vgrid);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpy2DAsync(vmom, 6 * sizeof(double), dm, 8 * sizeof(double), 6 * sizeof(double),
                            (size_t)h->nz, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

int cosenu_running_moments(cosenu_t h, double* vmom) {
  if (!h || !vmom) return fail(h, COSENU_EINVAL, "NULL argument");
  if (h->precision != COSENU_MIXED) return cosenu_moments(h, nullptr, vmom);
  // my is [nz][8] (6 used)
  CK(h, cudaMemcpy2DAsync(vmom, 6 * sizeof(double), h->my, 8 * sizeof(double), 6 * sizeof(double),
                          (size_t)h->nz, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

int cosenu_dp_field(cosenu_t h, double* out) {
  if (!h || !out) return fail(h, COSENU_EINVAL, "NULL argument");
  // staged in the delta_1 buffer (free between steps; 16 nz nv <= its 32 nz nv bytes)
  double* dev = static_cast<double*>(h->d[0]);
  const int64_t n = 2 * h->nz * (int64_t)h->nv;
  dp_field_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, h->stream>>>(
      h->y[h->ycur], h->nz, h->nv, dev);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(out, dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

int cosenu_spectrum(cosenu_t h, int32_t species, int32_t v_index, int64_t m0, int64_t nk,
                    double* out) {
  if (!h || !out) return fail(h, COSENU_EINVAL, "NULL argument");
  if (species < 0 || species > 1 || v_index < 0 || v_index >= h->nv || nk < 0 || nk > h->nz ||
      h->nz > ((int64_t)1 << 31))
    return fail(h, COSENU_EINVAL,
                "need species 0 or 1, 0 <= v_index < nv, 0 <= nk <= nz, nz <= 2^31");
  if (nk == 0) return COSENU_OK;
  double* dev = static_cast<double*>(h->d[0]);  // 16 nk <= 16 nz bytes
  dft_beam_kernel<<<(int)nk, 256, 0, h->stream>>>(h->y[h->ycur], h->nz, h->nv, species,
                                                  v_index, m0, dev);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(out, dev, (size_t)nk * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return COSENU_OK;
}

int cosenu_conserved(cosenu_t h, cosenu_conserved_t* out) {
  if (!h || !out) return fail(h, COSENU_EINVAL, "NULL argument");
  const int64_t ncell = h->nz * h->nv;
  const int nb = (int)std::min<int64_t>(kDiagMaxBlocks, (ncell + kDiagBlock - 1) / kDiagBlock);
  double* part = reinterpret_cast<double*>(h->ws + h->lay.partial);
  double* res = reinterpret_cast<double*>(h->ws + h->lay.result);
  conserved_partial_kernel<<<nb, kDiagBlock, 0, h->stream>>>(h->y[h->ycur], h->nz, h->nv, part,
                                                              h->vgrid);
  CK(h, cudaGetLastError());
  conserved_final_kernel<<<1, 32, 0, h->stream>>>(part, nb, res);
  CK(h, cudaGetLastError());
  g_launches.fetch_add(2, std::memory_order_relaxed);
  double r[8];
  CK(h, cudaMemcpyAsync(r, res, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const double w = (2.0 / h->nv) * (h->L / (double)h->nz);
  out->tr_nu = w * r[0];
  out->tr_nubar = w * r[1];
  out->M[0] = w * r[2];
  out->M[1] = w * r[3];
  out->M[2] = w * r[4];
  out->M_vac = std::sin(2.0 * h->p.theta) * out->M[0] - std::cos(2.0 * h->p.theta) * out->M[2];
  out->dP_max = r[5];
  out->dP_mean = r[7] > 0.0 ? r[6] / r[7] : 0.0;
  out->step = h->steps;
  return COSENU_OK;
}

int cosenu_set_stage_timing(cosenu_t h, int on) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  h->timing = on != 0;
  return COSENU_OK;
}

int cosenu_stage_times(cosenu_t h, double* ms, int64_t* n) {
  if (!h) return fail(h, COSENU_EINVAL, "NULL handle");
  CK(h, cudaStreamSynchronize(h->stream));
  for (int s = 1; s <= 5; ++s) {
    double sum = 0.0;
    for (auto& pr : h->ev[s]) {
      float t = 0.0f;
      CK(h, cudaEventElapsedTime(&t, pr.first, pr.second));
      sum += t;
      h->ev_free.push_back(pr.first);
      h->ev_free.push_back(pr.second);
    }
    if (ms) ms[s - 1] = sum;
    if (n) n[s - 1] = (int64_t)h->ev[s].size();
    h->ev[s].clear();
  }
  return COSENU_OK;
}

int64_t cosenu_steps_taken(cosenu_t h) { return h ? h->steps : -1; }

const char* cosenu_last_error(cosenu_t h) {
  return h ? h->error.c_str() : tl_error.c_str();
}

uint64_t cosenu_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
