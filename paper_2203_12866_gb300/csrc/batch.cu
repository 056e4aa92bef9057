// Batched solver of the C ABI (declared in include/cosenu.h): many independent
// grids advanced together.
//
// Members are ordinary handles created on the batch's stream.  They are grouped
// into classes of equal (scheme, precision, nv).  A class runs the batched form
// of the fused stage kernels: each member's z rows are cut into work items of
// about the same length (a z range of one member), one per CTA, so members of
// any size share one launch per stage.  A CTA runs exactly the code of a
// single-grid CTA on its item, which makes a member's results independent of
// the batch it is in.
//
// The launch tables (per-member stage arguments for both FP64 state parities,
// work items, increment segments, error-flag pointers) live in one device
// buffer, rebuilt when members or parameters change.  Two steps are captured
// in a CUDA graph, the class chains as parallel branches (or in series, as the
// tuner decides).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/cosenu.h"
#include "diag_kernels.cuh"
#include "engine.cuh"

using namespace cosenu;

namespace {

thread_local std::string tl_berror;

constexpr int kGraphSteps = 2;
constexpr int64_t kMinRowsPerCta = 16;
constexpr size_t kTableAlign = 256;

size_t align_t(size_t x) { return (x + kTableAlign - 1) & ~(kTableAlign - 1); }

struct ClassKey {
  int scheme, precision, nv;
  bool operator<(const ClassKey& o) const {
    return std::tie(scheme, precision, nv) < std::tie(o.scheme, o.precision, o.nv);
  }
};

// Launch shape of one stage of a class: index into its ring choices, grid factor.
struct Shape {
  int choice = 0, gridf = 1;
};

struct ClassPlan {
  ClassKey key{};
  std::vector<int> members;  // indices into the batch's member list
  int64_t rows = 0;
  std::vector<RingChoice> choices[5];
  Shape shape[5];
  StageCfg cfg[5];
  int occ[5] = {};
  size_t inst_off[5][2] = {}, item_off[5] = {};
  size_t seg_off = 0, chunk_off = 0, fold_off = 0;
  size_t seg64_off[2] = {};  // FP64: increment segments per state parity
  int nseg = 0;
  int64_t nchunks = 0, nfold = 0;  // increment chunks, fold blocks
  double kernel_ms[6] = {};  // mean device time per launch at the last cosenu_batch_stage_times
};

struct TimedKernel {
  int cls, kernel;  // kernel 1..4 stages, 5 increment
  cudaEvent_t e0, e1;
};

}  // namespace

struct cosenu_batch_s {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> side;  // one per class (parallel branches)
  std::vector<cudaEvent_t> joins;  // one per class
  cudaEvent_t fork = nullptr;
  std::vector<cosenu_t> members;
  std::vector<uint64_t> versions;  // members' parameter versions at the last plan
  std::vector<ClassPlan> classes;
  std::map<ClassKey, std::vector<Shape>> tuned;  // per class key: shapes of stages 1..4
  bool plan_ok = false;
  bool concurrent = true;
  unsigned char* tables = nullptr;
  size_t tables_bytes = 0, tables_cap = 0;
  size_t flagptr_off = 0, flagout_off = 0;
  uint32_t* flags_host = nullptr;  // pinned
  size_t flags_host_cap = 0;
  cudaGraphExec_t graph = nullptr;
  int parity = 0;  // FP64 members' current state buffer
  bool timing = false;
  bool capturing = false;  // launches being captured are counted per replay instead
  std::vector<TimedKernel> timed;
  std::vector<cudaEvent_t> ev_free;
  std::string error;
};

namespace {

int bfail(cosenu_batch_t b, int code, const std::string& msg) {
  if (b)
    b->error = msg;
  else
    tl_berror = msg;
  return code;
}

int bcuda(cosenu_batch_t b, cudaError_t e, const char* what) {
  return bfail(b, COSENU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call)                                        \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);      \
  } while (0)

void drop_graph(cosenu_batch_t b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

bool versions_current(const cosenu_batch_t b) {
  if (b->versions.size() != b->members.size()) return false;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->versions[i] != b->members[i]->version) return false;
  return true;
}

// Work items of one class stage: at most factor x SMs x resident CTAs of them
// (a whole number of waves of resident CTAs, so no last wave runs a few items
// on an otherwise idle GPU), at least kMinRowsPerCta rows each (cfg.rows: the
// rows per item; each member is cut into ceil(nz / rows) near-equal ranges).
void shape_stage(cosenu_batch_t b, ClassPlan& c, int s) {
  const Shape sh = c.shape[s];
  const RingChoice& rc = c.choices[s][sh.choice];
  StageCfg& cf = c.cfg[s];
  cf.block = stage_block(c.key.scheme, c.key.precision, c.key.nv, s);
  cf.ring = rc.ring;
  cf.rows_per_slot = rc.rows_per_slot;
  cf.slot_bytes = rc.slot_bytes;
  cf.smem = rc.smem;
  c.occ[s] = rc.occ;
  const int64_t target = std::max<int64_t>(1, (int64_t)b->nsm * rc.occ * sh.gridf);
  auto items_for = [&](int64_t rows) {
    int64_t n = 0;
    for (int mi : c.members) n += (b->members[mi]->nz + rows - 1) / rows;
    return n;
  };
  int64_t lo = std::max<int64_t>(kMinRowsPerCta, (c.rows + target - 1) / target);
  if (items_for(lo) > target) {
    // the smallest row count whose items fit the waves (items fall as rows grow;
    // with more members than target, one item per member is the floor)
    int64_t hi = lo;
    for (int mi : c.members) hi = std::max<int64_t>(hi, b->members[mi]->nz);
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (items_for(mid) > target) lo = mid + 1; else hi = mid;
    }
  }
  cf.rows = lo;
  cf.grid = (int)items_for(cf.rows);
}

// Host image of the launch tables; offsets are recorded in the class plans.
struct TableImage {
  std::vector<unsigned char> bytes;
  size_t put(const void* p, size_t n) {
    const size_t off = align_t(bytes.size());
    bytes.resize(off + n);
    if (n) std::memcpy(bytes.data() + off, p, n);
    return off;
  }
};

int write_tables(cosenu_batch_t b) {
  TableImage img;
  img.bytes.reserve(1 << 16);
  for (ClassPlan& c : b->classes) {
    for (int s = 1; s <= 4; ++s) {
      const StageCfg& cf = c.cfg[s];
      // per-member arguments, both parities, with the launch shape of this stage
      for (int par = 0; par < 2; ++par) {
        std::vector<StageArgs> inst;
        inst.reserve(c.members.size());
        for (int mi : c.members) {
          const cosenu_t h = b->members[mi];
          StageArgs a = stage_args(h, s, h->precision == COSENU_FP64 ? par : 0);
          a.ring = cf.ring;
          a.rows_per_slot = cf.rows_per_slot;
          a.slot_bytes = cf.slot_bytes;
          a.rows_per_cta = cf.rows;
          if (!stage_args_complete(h->precision, s, a))
            return bfail(b, COSENU_EINVAL, "a member's stage buffers are missing");
          inst.push_back(a);
        }
        c.inst_off[s][par] = img.put(inst.data(), inst.size() * sizeof(StageArgs));
      }
      // work items: member m's rows in ceil(nz / rows) near-equal ranges; longest first
      std::vector<WorkItem> items;
      for (int m = 0; m < (int)c.members.size(); ++m) {
        const int64_t nz = b->members[c.members[m]]->nz;
        const int64_t n = (nz + cf.rows - 1) / cf.rows;
        for (int64_t k = 0; k < n; ++k) {
          WorkItem w;
          w.inst = m;
          w.pad = 0;
          w.z_begin = nz * k / n;
          w.z_end = nz * (k + 1) / n;
          items.push_back(w);
        }
      }
      std::stable_sort(items.begin(), items.end(), [](const WorkItem& x, const WorkItem& y) {
        return x.z_end - x.z_begin > y.z_end - y.z_begin;
      });
      c.item_off[s] = img.put(items.data(), items.size() * sizeof(WorkItem));
    }
    c.nseg = 0;
    c.nchunks = 0;
    c.nfold = 0;
    if (c.key.precision == COSENU_MIXED) {
      std::vector<ApplySeg> segs;
      std::vector<int64_t> chunk_first, fold_first;
      for (int mi : c.members) {
        const ApplySeg sg = apply_seg(b->members[mi]);
        segs.push_back(sg);
        chunk_first.push_back(c.nchunks);
        c.nchunks += sg.nchunks;
        fold_first.push_back(c.nfold);
        c.nfold += (sg.nz + kFoldRows - 1) / kFoldRows;
      }
      chunk_first.push_back(c.nchunks);
      fold_first.push_back(c.nfold);
      c.nseg = (int)segs.size();
      c.seg_off = img.put(segs.data(), segs.size() * sizeof(ApplySeg));
      c.chunk_off = img.put(chunk_first.data(), chunk_first.size() * sizeof(int64_t));
      c.fold_off = img.put(fold_first.data(), fold_first.size() * sizeof(int64_t));
    } else {
      std::vector<int64_t> chunk_first;
      for (int mi : c.members) {
        const cosenu_t h = b->members[mi];
        chunk_first.push_back(c.nchunks);
        c.nchunks += (4 * h->nz * (int64_t)h->nv + kApplyGroups - 1) / kApplyGroups;
      }
      chunk_first.push_back(c.nchunks);
      for (int par = 0; par < 2; ++par) {
        std::vector<ApplySeg64> segs;
        for (int mi : c.members) {
          const cosenu_t h = b->members[mi];
          ApplySeg64 sg;
          sg.y_in = h->y[par];
          sg.y_out = h->y[par ^ 1];
          for (int k = 0; k < 4; ++k) sg.d[k] = static_cast<const double*>(h->d[k]);
          sg.n2 = 4 * h->nz * (int64_t)h->nv;
          sg.err = h->err;
          segs.push_back(sg);
        }
        c.seg64_off[par] = img.put(segs.data(), segs.size() * sizeof(ApplySeg64));
      }
      c.nseg = (int)c.members.size();
      c.chunk_off = img.put(chunk_first.data(), chunk_first.size() * sizeof(int64_t));
    }
  }
  // error flags: every member's word
  std::vector<uint32_t*> fp;
  for (cosenu_t h : b->members) fp.push_back(h->err);
  b->flagptr_off = img.put(fp.data(), fp.size() * sizeof(uint32_t*));
  std::vector<uint32_t> zeros(fp.size(), 0u);
  b->flagout_off = img.put(zeros.data(), zeros.size() * sizeof(uint32_t));

  const size_t need = align_t(img.bytes.size());
  if (need > b->tables_cap) {
    if (b->tables) cudaFree(b->tables);
    b->tables = nullptr;
    b->tables_cap = 0;
    cudaError_t e = cudaMalloc(&b->tables, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, COSENU_ENOMEM, std::string("launch tables: ") + cudaGetErrorString(e));
    }
    b->tables_cap = need;
  }
  b->tables_bytes = img.bytes.size();
  BCK(b, cudaMemcpyAsync(b->tables, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice,
                         b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));  // the host image dies here
  if (b->flags_host_cap < fp.size()) {
    if (b->flags_host) cudaFreeHost(b->flags_host);
    b->flags_host = nullptr;
    b->flags_host_cap = 0;
    BCK(b, cudaMallocHost(&b->flags_host, fp.size() * sizeof(uint32_t)));
    b->flags_host_cap = fp.size();
  }
  return COSENU_OK;
}

// (Re)build classes, launch shapes and tables if members or parameters changed.
int plan(cosenu_batch_t b, bool force = false) {
  if (b->plan_ok && !force && versions_current(b)) return COSENU_OK;
  BCK(b, cudaStreamSynchronize(b->stream));  // queued work may still read the old tables
  drop_graph(b);
  b->plan_ok = false;
  std::map<ClassKey, std::vector<int>> groups;
  for (size_t i = 0; i < b->members.size(); ++i) {
    const cosenu_t h = b->members[i];
    groups[{h->scheme, h->precision, h->nv}].push_back((int)i);
  }
  std::vector<ClassPlan> classes;
  for (auto& kv : groups) {
    ClassPlan c;
    c.key = kv.first;
    c.members = kv.second;
    for (int mi : c.members) c.rows += b->members[mi]->nz;
    auto tuned = b->tuned.find(c.key);
    for (int s = 1; s <= 4; ++s) {
      bool qfail = false;
      c.choices[s] = ring_choices(c.key.scheme, c.key.precision, c.key.nv, s, true, &qfail);
      if (qfail) return bfail(b, COSENU_ECUDA, "occupancy query failed");
      if (c.choices[s].empty()) return bfail(b, COSENU_EINVAL, "grid row does not fit in shared memory");
      if (tuned != b->tuned.end()) c.shape[s] = tuned->second[s];
      if (c.shape[s].choice >= (int)c.choices[s].size()) c.shape[s] = Shape{};
      shape_stage(b, c, s);
    }
    classes.push_back(std::move(c));
  }
  b->classes = std::move(classes);
  while (b->side.size() < b->classes.size()) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BCK(b, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->side.push_back(st);
    BCK(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->joins.push_back(ev);
  }
  if (int rc = write_tables(b)) return rc;
  b->versions.resize(b->members.size());
  for (size_t i = 0; i < b->members.size(); ++i) b->versions[i] = b->members[i]->version;
  b->plan_ok = true;
  return COSENU_OK;
}

cudaError_t take_event(cosenu_batch_t b, cudaEvent_t* out) {
  if (!b->ev_free.empty()) {
    *out = b->ev_free.back();
    b->ev_free.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(out);
}

// Kernel k (1..4 stage, 5 increment, 6 moment fold) of class c for state parity
// `par` on `st`.
cudaError_t launch_kernel(cosenu_batch_t b, int ci, int k, int par, cudaStream_t st) {
  const ClassPlan& c = b->classes[ci];
  if (k == 5 && c.key.precision == COSENU_FP64) {
    const ApplySeg64* segs = reinterpret_cast<const ApplySeg64*>(b->tables + c.seg64_off[par]);
    const int64_t* cf = reinterpret_cast<const int64_t*>(b->tables + c.chunk_off);
    const int64_t blocks = std::min<int64_t>(c.nchunks, (int64_t)b->nsm * 8);
    apply_increment_fp64_batch_kernel<<<(int)blocks, 256, 0, st>>>(segs, cf, c.nseg, c.nchunks);
    return cudaGetLastError();
  }
  if (k == 5) {
    const ApplySeg* segs = reinterpret_cast<const ApplySeg*>(b->tables + c.seg_off);
    const int64_t* cf = reinterpret_cast<const int64_t*>(b->tables + c.chunk_off);
    const int64_t blocks = std::min<int64_t>(c.nchunks, (int64_t)b->nsm * 6);  // two waves of three per SM
    apply_increment_batch_kernel<<<(int)blocks, kApplyThreads, 0, st>>>(segs, cf, c.nseg,
                                                                        c.nchunks);
    return cudaGetLastError();
  }
  if (k == 6) {
    const ApplySeg* segs = reinterpret_cast<const ApplySeg*>(b->tables + c.seg_off);
    const int64_t* ff = reinterpret_cast<const int64_t*>(b->tables + c.fold_off);
    const int64_t blocks = std::min<int64_t>(c.nfold, (int64_t)b->nsm * 8);
    fold_moments_batch_kernel<<<(int)blocks, 256, 0, st>>>(segs, ff, c.nseg, c.nfold);
    return cudaGetLastError();
  }
  const StageCfg& cf = c.cfg[k];
  StageArgs unused;
  std::memset(&unused, 0, sizeof(unused));
  BatchTable bt;
  bt.inst = reinterpret_cast<const StageArgs*>(b->tables + c.inst_off[k][par]);
  bt.items = reinterpret_cast<const WorkItem*>(b->tables + c.item_off[k]);
  return launch_stage_kernel(c.key.scheme, c.key.precision, k, unused, &bt, cf.grid, cf.block,
                             cf.smem, st);
}

// One class's RK4 step on `st`; kernels bracketed by events when timing.
cudaError_t enqueue_chain(cosenu_batch_t b, int ci, int par, cudaStream_t st, bool timed) {
  const int nk = b->classes[ci].key.precision == COSENU_MIXED ? 6 : 5;
  for (int k = 1; k <= nk; ++k) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && k <= 5) {  // the moment fold is not timed
      cudaError_t e = take_event(b, &e0);
      if (e == cudaSuccess) e = take_event(b, &e1);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_kernel(b, ci, k, par, st);
    if (e != cudaSuccess) return e;
    if (!b->capturing) count_launches(1);
    if (timed && k <= 5) {
      e = cudaEventRecord(e1, st);
      if (e != cudaSuccess) return e;
      b->timed.push_back({ci, k, e0, e1});
    }
  }
  return cudaSuccess;
}

// One RK4 step of every member from parity `par`: the class chains in series
// on the batch stream, or forked onto one stream per class and joined.
cudaError_t enqueue_step(cosenu_batch_t b, int par, bool concurrent, bool timed) {
  const int nc = (int)b->classes.size();
  if (!concurrent || nc < 2) {
    for (int ci = 0; ci < nc; ++ci) {
      cudaError_t e = enqueue_chain(b, ci, par, b->stream, timed);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (int ci = 0; ci < nc && e == cudaSuccess; ++ci) {
    e = cudaStreamWaitEvent(b->side[ci], b->fork, 0);
    if (e == cudaSuccess) e = enqueue_chain(b, ci, par, b->side[ci], timed);
    if (e == cudaSuccess) e = cudaEventRecord(b->joins[ci], b->side[ci]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[ci], 0);
  }
  return e;
}

int build_graph(cosenu_batch_t b) {
  cudaGraph_t g = nullptr;
  BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  b->capturing = true;
  for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k)
    e = enqueue_step(b, k & 1, b->concurrent, false);
  b->capturing = false;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bcuda(b, e, "batched step launch during capture");
  }
  if (e2 != cudaSuccess) return bcuda(b, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bcuda(b, e, "cudaGraphInstantiate");
  }
  return COSENU_OK;
}

// Launches one graph replay stands for (captured launches are counted per replay).
int graph_launches(const cosenu_batch_t b) {
  int n = 0;
  for (const ClassPlan& c : b->classes) n += c.key.precision == COSENU_MIXED ? 6 : 5;
  return n * kGraphSteps;
}

// FP64 members must hold their state in buffer `parity`; a member stepped on
// its own since may not: copy its state over (stream-ordered).
int align_parity(cosenu_batch_t b) {
  for (cosenu_t h : b->members) {
    if (h->precision != COSENU_FP64 || h->ycur == b->parity) continue;
    const size_t n = (size_t)8 * h->nz * h->nv;
    BCK(b, cudaMemcpyAsync(h->y[b->parity], h->y[h->ycur], n * sizeof(double),
                           cudaMemcpyDeviceToDevice, b->stream));
    h->ycur = b->parity;
  }
  return COSENU_OK;
}

void advance_members(cosenu_batch_t b, int64_t n) {
  for (cosenu_t h : b->members) {
    h->steps += n;
    h->ycur = h->precision == COSENU_FP64 ? b->parity : 0;
  }
}

// n RK4 steps: pairs from the graph (from parity 0), the rest launched directly.
int run_steps(cosenu_batch_t b, int64_t n, bool allow_graph) {
  if (n == 0 || b->members.empty()) {
    advance_members(b, n);
    return COSENU_OK;
  }
  if (int rc = align_parity(b)) return rc;
  int64_t left = n;
  const bool use_graph = allow_graph && !b->timing && left >= 2;
  if (use_graph) {
    if (b->parity == 1) {
      BCK(b, enqueue_step(b, 1, b->concurrent, false));
      b->parity = 0;
      --left;
    }
    if (!b->graph)
      if (int rc = build_graph(b)) return rc;
    for (; left >= kGraphSteps; left -= kGraphSteps) {
      BCK(b, cudaGraphLaunch(b->graph, b->stream));
      count_launches(graph_launches(b));
    }
  }
  for (; left > 0; --left) {
    // timed steps run the classes in series, so each kernel's time is its own
    BCK(b, enqueue_step(b, b->parity, b->concurrent && !b->timing, b->timing));
    b->parity ^= 1;
  }
  // (the graph's pair of steps leaves the parity unchanged)
  advance_members(b, n);
  return COSENU_OK;
}

// Summed device time per (class, kernel) of the timed launches; clears them.
int collect_times(cosenu_batch_t b, std::vector<double>* per_class_kernel) {
  BCK(b, cudaStreamSynchronize(b->stream));
  for (cudaStream_t st : b->side) BCK(b, cudaStreamSynchronize(st));
  const size_t nc = b->classes.size();
  per_class_kernel->assign(nc * 6, 0.0);
  for (const TimedKernel& t : b->timed) {
    float ms = 0.0f;
    BCK(b, cudaEventElapsedTime(&ms, t.e0, t.e1));
    if ((size_t)t.cls < nc) (*per_class_kernel)[t.cls * 6 + t.kernel] += ms;
    b->ev_free.push_back(t.e0);
    b->ev_free.push_back(t.e1);
  }
  b->timed.clear();
  return COSENU_OK;
}

}  // namespace

extern "C" {

cosenu_batch_t cosenu_batch_create(void) {
  cosenu_batch_t b = new (std::nothrow) cosenu_batch_s;
  if (!b) {
    bfail(nullptr, COSENU_ENOMEM, "host allocation failed");
    return nullptr;
  }
  auto bail = [&](cudaError_t e, const char* what) -> cosenu_batch_t {
    bfail(nullptr, COSENU_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return nullptr;
  };
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
  e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
  e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "cudaEventCreate");
  return b;
}

void cosenu_batch_destroy(cosenu_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (cudaStream_t st : b->side) cudaStreamSynchronize(st);
  drop_graph(b);
  for (cosenu_t h : b->members) destroy_member(h);
  for (const TimedKernel& t : b->timed) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (cudaEvent_t e : b->ev_free) cudaEventDestroy(e);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->tables) cudaFree(b->tables);
  if (b->flags_host) cudaFreeHost(b->flags_host);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int cosenu_batch_add(cosenu_batch_t b, int64_t nz, int32_t nv, double L, int scheme,
                     int precision, cosenu_t* member) {
  if (!b || !member) return bfail(b, COSENU_EINVAL, "NULL argument");
  *member = nullptr;
  int dev = -1;
  BCK(b, cudaGetDevice(&dev));
  if (dev != b->device) return bfail(b, COSENU_EINVAL, "the current device is not the batch's");
  cosenu_t h = create_member(nz, nv, L, scheme, precision, b->stream);
  if (!h) return bfail(b, COSENU_EINVAL, std::string("member: ") + cosenu_last_error(nullptr));
  // zero state: either FP64 buffer will do (mixed members have one state buffer)
  h->ycur = h->precision == COSENU_FP64 ? b->parity : 0;
  b->members.push_back(h);
  b->plan_ok = false;
  *member = h;
  return COSENU_OK;
}

int cosenu_batch_remove(cosenu_batch_t b, cosenu_t member) {
  if (!b || !member) return bfail(b, COSENU_EINVAL, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), member);
  if (it == b->members.end()) return bfail(b, COSENU_EINVAL, "not a member of this batch");
  BCK(b, cudaStreamSynchronize(b->stream));
  for (cudaStream_t st : b->side) BCK(b, cudaStreamSynchronize(st));
  drop_graph(b);
  destroy_member(member);
  b->members.erase(it);
  b->plan_ok = false;
  return COSENU_OK;
}

int32_t cosenu_batch_size(cosenu_batch_t b) { return b ? (int32_t)b->members.size() : -1; }

size_t cosenu_batch_device_bytes(cosenu_batch_t b) {
  if (!b) return 0;
  size_t n = b->tables_cap;
  for (cosenu_t h : b->members) n += h->lay.total;
  return n;
}

cosenu_t cosenu_batch_member(cosenu_batch_t b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->members.size()) return nullptr;
  return b->members[i];
}

int cosenu_batch_step(cosenu_batch_t b, int64_t nsteps) {
  if (!b) return bfail(b, COSENU_EINVAL, "NULL batch");
  if (nsteps < 0) return bfail(b, COSENU_EINVAL, "nsteps must be >= 0");
  if (int rc = plan(b)) return rc;
  return run_steps(b, nsteps, true);
}

}  // extern "C"

namespace cosenu {

int batch_member_flags(cosenu_batch_t b, std::vector<uint32_t>* flags) {
  flags->clear();
  if (int rc = plan(b)) return rc;
  const int n = (int)b->members.size();
  if (n == 0) return COSENU_OK;
  uint32_t* const* ptrs = reinterpret_cast<uint32_t* const*>(b->tables + b->flagptr_off);
  uint32_t* out = reinterpret_cast<uint32_t*>(b->tables + b->flagout_off);
  gather_flags_kernel<<<(n + 255) / 256, 256, 0, b->stream>>>(ptrs, n, out, 1);
  BCK(b, cudaGetLastError());
  count_launches(1);
  BCK(b, cudaMemcpyAsync(b->flags_host, out, n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                         b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  flags->assign(b->flags_host, b->flags_host + n);
  return COSENU_OK;
}

}  // namespace cosenu

extern "C" {

int cosenu_batch_sync(cosenu_batch_t b, int32_t* first_bad) {
  if (!b) return bfail(b, COSENU_EINVAL, "NULL batch");
  if (first_bad) *first_bad = -1;
  std::vector<uint32_t> flags;
  if (int rc = batch_member_flags(b, &flags)) return rc;
  uint32_t any = 0;
  for (size_t i = 0; i < flags.size(); ++i) {
    if (flags[i] && first_bad && *first_bad < 0) *first_bad = (int32_t)i;
    any |= flags[i];
  }
  if (any & kErrTimeout) return bfail(b, COSENU_ETIMEOUT, "a device-side wait gave up");
  if (any) return bfail(b, COSENU_ENONFINITE, "non-finite value in a member's state");
  return COSENU_OK;
}

}  // extern "C"

namespace {

int tune(cosenu_batch_t b, int32_t reps, int64_t& taken) {
  const int nc = (int)b->classes.size();
  // candidate shapes per (class, stage)
  std::vector<std::vector<Shape>> cand(nc * 5);
  size_t ncand = 1;
  for (int ci = 0; ci < nc; ++ci)
    for (int s = 1; s <= 4; ++s) {
      auto& v = cand[ci * 5 + s];
      const auto& ch = b->classes[ci].choices[s];
      for (int k = 0; k < (int)ch.size() && k < 3; ++k) {
        if (k > 0 && ch[k].score < ch[0].score / 2) break;
        v.push_back({k, 1});
      }
      v.push_back({0, 2});
      v.push_back({0, 4});
      ncand = std::max(ncand, v.size());
    }
  std::vector<double> best(nc * 5, 1e300);
  std::vector<Shape> pick(nc * 5);
  std::vector<double> t;
  for (size_t k = 0; k < ncand; ++k) {
    for (int ci = 0; ci < nc; ++ci)
      for (int s = 1; s <= 4; ++s) {
        const auto& v = cand[ci * 5 + s];
        b->classes[ci].shape[s] = v[k % v.size()];
        shape_stage(b, b->classes[ci], s);
      }
    if (int rc = write_tables(b)) return rc;
    for (int r = 0; r < reps; ++r) {
      if (int rc = align_parity(b)) return rc;
      BCK(b, enqueue_step(b, b->parity, false, true));
      b->parity ^= 1;
      advance_members(b, 1);
      ++taken;
      if (int rc = collect_times(b, &t)) return rc;
      for (int ci = 0; ci < nc; ++ci)
        for (int s = 1; s <= 4; ++s) {
          const double ms = t[ci * 6 + s];
          if (ms < best[ci * 5 + s]) {
            best[ci * 5 + s] = ms;
            pick[ci * 5 + s] = b->classes[ci].shape[s];
          }
        }
    }
  }
  for (int ci = 0; ci < nc; ++ci) {
    std::vector<Shape> keep(5);
    for (int s = 1; s <= 4; ++s) {
      b->classes[ci].shape[s] = pick[ci * 5 + s];
      shape_stage(b, b->classes[ci], s);
      keep[s] = pick[ci * 5 + s];
    }
    b->tuned[b->classes[ci].key] = keep;
  }
  if (int rc = write_tables(b)) return rc;
  // classes in series or as parallel branches: time two graph replays of each
  if (nc > 1) {
    double mode_ms[2] = {0.0, 0.0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    for (int mode = 0; mode < 2; ++mode) {
      drop_graph(b);
      b->concurrent = mode == 1;
      if (b->parity == 1) {
        BCK(b, enqueue_step(b, 1, b->concurrent, false));
        b->parity = 0;
        advance_members(b, 1);
        ++taken;
      }
      if (int rc = build_graph(b)) return rc;
      BCK(b, cudaGraphLaunch(b->graph, b->stream));  // warm-up replay
      BCK(b, cudaEventRecord(e0, b->stream));
      BCK(b, cudaGraphLaunch(b->graph, b->stream));
      BCK(b, cudaEventRecord(e1, b->stream));
      BCK(b, cudaEventSynchronize(e1));
      count_launches(2 * graph_launches(b));
      float ms = 0.0f;
      BCK(b, cudaEventElapsedTime(&ms, e0, e1));
      mode_ms[mode] = ms;
      advance_members(b, 2 * kGraphSteps);
      taken += 2 * kGraphSteps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool conc = mode_ms[1] < mode_ms[0];
    if (conc != b->concurrent) drop_graph(b);
    b->concurrent = conc;
  }
  return COSENU_OK;
}

}  // namespace

extern "C" {

int cosenu_batch_tune(cosenu_batch_t b, int32_t reps, int64_t* steps_taken) {
  if (!b) return bfail(b, COSENU_EINVAL, "NULL batch");
  if (steps_taken) *steps_taken = 0;
  if (reps < 1) return bfail(b, COSENU_EINVAL, "reps must be >= 1");
  if (int rc = plan(b)) return rc;
  if (b->members.empty()) return COSENU_OK;
  int64_t taken = 0;
  const int rc = tune(b, reps, taken);
  if (steps_taken) *steps_taken = taken;
  return rc;
}

int32_t cosenu_batch_classes(cosenu_batch_t b) {
  if (!b) return -1;
  if (plan(b) != COSENU_OK) return -1;
  return (int32_t)b->classes.size();
}

int cosenu_batch_class_info(cosenu_batch_t b, int32_t ci, cosenu_batch_class* out) {
  if (!b || !out) return bfail(b, COSENU_EINVAL, "NULL argument");
  if (int rc = plan(b)) return rc;
  if (ci < 0 || ci >= (int32_t)b->classes.size()) return bfail(b, COSENU_EINVAL, "no such class");
  const ClassPlan& c = b->classes[ci];
  std::memset(out, 0, sizeof(*out));
  out->scheme = c.key.scheme;
  out->precision = c.key.precision;
  out->nv = c.key.nv;
  out->members = (int32_t)c.members.size();
  out->rows = c.rows;
  for (int s = 1; s <= 4; ++s) {
    out->rows_per_slot[s - 1] = c.cfg[s].rows_per_slot;
    out->ring[s - 1] = c.cfg[s].ring;
    out->grid[s - 1] = c.cfg[s].grid;
    out->smem[s - 1] = (int32_t)c.cfg[s].smem;
    out->occupancy[s - 1] = c.occ[s];
  }
  for (int k = 1; k <= 5; ++k) out->kernel_ms[k - 1] = c.kernel_ms[k];
  out->concurrent = b->concurrent ? 1 : 0;
  return COSENU_OK;
}

int cosenu_batch_set_stage_timing(cosenu_batch_t b, int on) {
  if (!b) return bfail(b, COSENU_EINVAL, "NULL batch");
  b->timing = on != 0;
  return COSENU_OK;
}

int cosenu_batch_stage_times(cosenu_batch_t b, double* ms, int64_t* n) {
  if (!b) return bfail(b, COSENU_EINVAL, "NULL batch");
  const size_t nc = b->classes.size();
  std::vector<int64_t> cnt(nc * 6, 0), tot(6, 0);
  for (const TimedKernel& t : b->timed)
    if ((size_t)t.cls < nc) {
      cnt[t.cls * 6 + t.kernel] += 1;
      tot[t.kernel] += 1;
    }
  std::vector<double> t;
  if (int rc = collect_times(b, &t)) return rc;
  for (size_t ci = 0; ci < nc; ++ci)
    for (int k = 1; k <= 5; ++k)
      b->classes[ci].kernel_ms[k] = cnt[ci * 6 + k] ? t[ci * 6 + k] / cnt[ci * 6 + k] : 0.0;
  for (int k = 1; k <= 5; ++k) {
    double sum = 0.0;
    for (size_t ci = 0; ci < nc; ++ci) sum += t[ci * 6 + k];
    if (ms) ms[k - 1] = sum;
    if (n) n[k - 1] = tot[k];
  }
  return COSENU_OK;
}

void* cosenu_batch_stream(cosenu_batch_t b) { return b ? static_cast<void*>(b->stream) : nullptr; }

const char* cosenu_batch_last_error(cosenu_batch_t b) {
  return b ? b->error.c_str() : tl_berror.c_str();
}

}  // extern "C"
