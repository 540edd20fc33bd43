// runtime.cpp -- the C-ABI of diffuse.h: stores, views, partitions, task
// submission, and flush_window() (Section 5.1) with memoised analysis and
// code generation (Section 5.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <stdexcept>

#include "jit.hpp"
#include "runtime.hpp"

namespace dfs {

int64_t StoreRec::nelem() const {
  int64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= shape[d];
  return n;
}

// One launch of a cached window: a compiled kernel and how to fill its
// parameters from a window isomorphic to the one it was generated for.
struct CachedLaunch {
  const Compiled* k = nullptr;
  std::string name;
  int block = 256;
  int grid = 1;
  bool cooperative = false;
  int nbarriers = 0;
  int nptr = 0, nimm = 0;
  std::vector<int> ptr_canon;                 // canonical root id per pointer param
  std::vector<std::pair<int, int>> imm_src;   // (window task, arg) per immediate param
  int64_t red_stride = 1;
  size_t partial_bytes = 0;
  int first_task = 0, last_task = 0;
  std::string source;
};

struct CachedWindow {
  Plan plan;
  std::vector<CachedLaunch> launches;
  std::vector<int> materialise;  // canonical ids that need device memory
  std::vector<int> made_valid;   // canonical ids holding a value afterwards
};

struct Stats {
  int64_t tasks = 0, groups = 0, launches = 0, barriers = 0, flushes = 0;
  int64_t plan_hits = 0, plan_misses = 0, temporaries = 0, window_growths = 0;
  int last_regs = 0, last_occupancy = 0, last_grid = 0, last_block = 0;
  int64_t bytes_allocated = 0, allocations = 0;
  double analysis_s = 0.0;
};

}  // namespace dfs

namespace dfs {
// gather.cu
cudaError_t launch_gather_scalars(const int64_t* desc_dev, int n, double* out_dev, cudaStream_t s);
}  // namespace dfs

struct dfs_ctx {
  dfs_config cfg{};
  bool device = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 0;
  dfs::Driver drv;
  std::unique_ptr<dfs::Jit> jit;
  std::map<int64_t, dfs::StoreRec> stores;
  std::map<int64_t, dfs::PartRec> parts;
  int64_t next_handle = 1;
  std::vector<dfs::Task> window;
  int64_t seq = 0;
  std::string err;
  dfs::Ctl* ctl = nullptr;
  void* partials = nullptr;
  size_t partials_cap = 0;
  std::unordered_map<std::string, std::unique_ptr<dfs::CachedWindow>> wcache;
  dfs::Stats st;
  std::string last_source;
  // per-launch device timing (cfg.time_launches)
  struct Timed {
    cudaEvent_t a, b;
    std::string name;
  };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> event_pool;
  std::map<std::string, std::pair<double, int64_t>> ktime;  // kernel -> (ms, launches)
  // CUDA-graph capture
  bool capturing = false;
  std::set<int64_t> captured_allocs;    // roots allocated inside the capture
  std::vector<void*> capture_deferred;  // pre-capture memory released while capturing
  int64_t capture_launches = 0;
  struct GraphRec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> owned;           // memory freed when the graph is destroyed
    int64_t launches = 0;
  };
  std::map<int64_t, GraphRec> graphs;
  // batched execution
  bool batching = false;
  std::vector<size_t> batch_marks;      // window positions where instances end
  struct BatchEntry {
    dfs::BatchCode code;
    const dfs::Compiled* k = nullptr;
    dfs::Plan plan;
    // canonical index (first-use order within an instance) of the root of
    // each pointer slot: later batches of the same structure use other stores
    std::vector<int> ptr_canon;
  };
  std::unordered_map<std::string, std::unique_ptr<BatchEntry>> bcache;
  struct Table {
    void* dev = nullptr;
    size_t bytes = 0;
  };
  std::unordered_map<std::string, Table> tables;  // descriptor bytes -> device copy
  double* sval = nullptr;
  size_t sval_cap = 0;
  int64_t batches = 0, batched_instances = 0, batch_fallbacks = 0, batch_repeats = 0;
  std::string batch_fallback_reason;
  // the most recent batched launch, kept for dfs_batch_repeat while steady
  struct LastBatch {
    bool ok = false;
    CUfunction fn = nullptr;
    int grid = 0, block = 0, nbarriers = 0, ninst = 0;
    int dyn_smem = 0;
    bool coop = false;
    uint64_t blob[8] = {};
    int64_t groups = 0;
    std::string name;
    const std::string* source = nullptr;  // the kernel's source (batch cache entries live as long as the context)
  };
  LastBatch lastb;
  // dfs_read_scalars: descriptors (pinned) and gathered values (device)
  int64_t* gather_host = nullptr;
  void* gather_dev = nullptr;
  size_t gather_cap = 0;  // scalars
  // completion tickets (dfs_record): an event recorded on the stream each
  std::map<uint64_t, cudaEvent_t> tickets;
  std::vector<cudaEvent_t> ticket_pool;
  uint64_t next_ticket = 1;
  // instance templates (dfs_template_*): a recorded sequence of store
  // creations, views, submissions and releases, replayed with other stores
  struct RecEv {
    int kind = 0;  // 0 create, 1 view, 2 submit, 3 release
    int64_t h = 0, parent = 0;
    int32_t dtype = 0, ndim = 0, op = 0;
    int64_t shape[DFS_MAX_DIM] = {0, 0, 0}, off[DFS_MAX_DIM] = {0, 0, 0}, dom[DFS_MAX_DIM] = {1, 1, 1};
    std::vector<dfs_arg> args;
  };
  struct Template {
    std::vector<RecEv> evs;
    std::vector<int64_t> ext;                    // stores used but not created, in first-use order
    std::vector<std::array<int64_t, 2 + DFS_MAX_DIM>> ext_info;  // dtype, ndim, shape
  };
  bool recording = false;
  std::string rec_fault;                         // why the recording cannot become a template
  Template rec;
  std::set<int64_t> rec_created, rec_live;
  std::map<uint64_t, Template> templates;
  uint64_t next_template = 1;
};

namespace dfs {
namespace {

int fail(dfs_ctx* c, int code, const std::string& m) {
  if (c) c->err = m;
  return code;
}

#define CUDA_OK(expr)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(c, DFS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

StoreRec* find_store(dfs_ctx* c, int64_t h) {
  auto it = c->stores.find(h);
  if (it == c->stores.end() || it->second.released) return nullptr;
  return &it->second;
}
StoreRec& root_of(dfs_ctx* c, const StoreRec& s) { return c->stores.at(s.root); }

void maybe_free(dfs_ctx* c, int64_t root) {
  auto it = c->stores.find(root);
  if (it == c->stores.end()) return;
  StoreRec& r = it->second;
  if (r.app_refs > 0 || r.pending > 0) return;
  if (r.owned && r.ptr && c->device) {
    c->lastb.ok = false;
    if (c->capturing && !c->captured_allocs.count(root)) {
      // allocated before the capture: replays of the graph may still read it
      c->capture_deferred.push_back(r.ptr);
    } else {
      cudaFreeAsync(r.ptr, c->stream);  // recorded as a free node while capturing
    }
  }
  c->captured_allocs.erase(root);
  c->stores.erase(it);
}

int materialise(dfs_ctx* c, StoreRec& r) {
  if (r.ptr) return DFS_OK;
  if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context has no device memory");
  const size_t bytes = std::max<size_t>(r.nbytes, 16);
  cudaError_t e = cudaMallocAsync(&r.ptr, bytes, c->stream);
  if (e != cudaSuccess) {
    r.ptr = nullptr;
    return fail(c, DFS_ERR_OOM, std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  r.owned = true;
  if (c->capturing) c->captured_allocs.insert(r.handle);
  c->st.bytes_allocated += (int64_t)bytes;
  c->st.allocations += 1;
  return DFS_OK;
}

// --------------------------------------------------------- submit validation
bool arity_ok(int op, int nargs) {
  if (op >= DFS_OP_COPY && op <= DFS_OP_NCDF) return nargs == 2;
  if (op >= DFS_OP_ADD && op <= DFS_OP_MIN) return nargs == 3;
  if (op == DFS_OP_DOT) return nargs == 3;
  if (op == DFS_OP_SUM) return nargs == 2;
  if (op == DFS_OP_SPMV) return nargs == 5 || nargs == 6;
  return false;
}
bool elementwise(int op) { return (op >= DFS_OP_COPY && op <= DFS_OP_NCDF) || (op >= DFS_OP_ADD && op <= DFS_OP_MIN); }

// Shape of a non-0-d argument's sub-store as a function of the point.
// Two accesses touch sub-stores of one shape at every point: the same
// partition kind and rank, extents, and (tilings) tile, offset from the view
// origin and projection.
bool same_substores(const Arg& a, const Arg& b) {
  if (a.part.kind != b.part.kind || a.nd != b.nd) return false;
  for (int d = 0; d < a.nd; ++d) {
    if (a.part.vhi[d] - a.part.vlo[d] != b.part.vhi[d] - b.part.vlo[d]) return false;
    if (a.part.kind && (a.part.tile[d] != b.part.tile[d] || a.part.proj[d] != b.part.proj[d] ||
                        a.part.off[d] - a.part.vlo[d] != b.part.off[d] - b.part.vlo[d]))
      return false;
  }
  return true;
}

int validate(dfs_ctx* c, const Task& t) {
  const int op = t.op;
  const auto& A = t.args;
  auto bad = [&](const std::string& m) { return fail(c, DFS_ERR_INVALID, m); };
  const bool scalar_task = t.scalar();
  if (scalar_task && t.npoints() != 1) return bad("a task over 0-d stores only must have a single-point launch domain");
  for (const Arg& a : A) {
    if (a.imm) continue;
    if (a.part.kind == 1) {
      for (int d = 0; d < a.nd; ++d)
        if (a.part.proj[d] < 0 || a.part.proj[d] >= t.dnd) return bad("tiling projection names a missing launch-domain coordinate");
    }
    if (a.nd == 0 && a.part.kind != 0) return bad("0-d stores are accessed through the None partition");
    if (a.is_w()) {
      if (a.part.kind == 0 && t.npoints() != 1 && a.nd != 0) return bad("a write through None needs a single-point launch domain (point tasks would interfere)");
      if (a.part.kind == 0 && a.nd == 0 && t.npoints() != 1) return bad("a 0-d store can only be written by a single-point task");
      if (a.part.kind == 1) {
        for (int cdim = 0; cdim < t.dnd; ++cdim) {
          if (t.dom[cdim] <= 1) continue;
          bool used = false;
          for (int d = 0; d < a.nd; ++d) used |= a.part.proj[d] == cdim;
          if (!used) return bad("a write through a tiling whose projection drops a launch-domain coordinate interferes");
        }
      }
    }
  }
  // aliasing inside one task: accesses to one root must agree when one writes,
  // and a reduced root is not read or written by the same task
  for (size_t i = 0; i < A.size(); ++i)
    for (size_t j = 0; j < A.size(); ++j) {
      if (i == j || A[i].imm || A[j].imm || A[i].root != A[j].root) continue;
      if (A[i].is_w() && A[i].part != A[j].part) return bad("a task writes a store and accesses an aliasing view of it");
      if (A[i].is_rd() && (A[j].is_r() || A[j].is_w())) return bad("a task reads or writes a store it reduces to");
    }
  if (elementwise(op)) {
    const Arg& out = A.back();
    if (out.imm || !out.is_w() || out.is_rd()) return bad("element-wise output must be a store with W or RW");
    if (!dtype_is_float(out.dtype)) return bad("element-wise ops need a floating dtype");
    const Arg* first = nullptr;  // the first operand with a shape
    for (size_t k = 0; k + 1 < A.size(); ++k)
      if (!A[k].imm && A[k].priv != DFS_PRIV_R) return bad("element-wise inputs are read (R) or immediates");
    for (const Arg& a : A) {
      if (a.imm) continue;
      if (a.dtype != out.dtype) return bad("element-wise operands must share one dtype");
      if (a.nd == 0) continue;
      if (!first) first = &a;
      else if (!same_substores(a, *first)) return bad("element-wise operands must have equal sub-store shapes at every point");
    }
    if (out.nd == 0 && !scalar_task) return bad("a 0-d output needs every operand 0-d");
    if (out.nd != 0 && out.part.kind == 0 && t.npoints() != 1) return bad("array operands need a tiling when the domain has several points");
  } else if (op == DFS_OP_DOT || op == DFS_OP_SUM) {
    const Arg& out = A.back();
    if (out.imm || !out.is_rd() || out.redop != DFS_REDOP_SUM || out.nd != 0) return bad("reduction output must be a 0-d store with RD(SUM)");
    for (size_t k = 0; k + 1 < A.size(); ++k) {
      if (A[k].imm || A[k].priv != DFS_PRIV_R || A[k].nd == 0) return bad("reduction inputs are non-0-d stores read (R)");
      if (A[k].dtype != out.dtype || !dtype_is_float(out.dtype)) return bad("reduction operands must share one floating dtype");
    }
    if (op == DFS_OP_DOT && !same_substores(A[0], A[1])) return bad("DOT operands must have equal sub-store shapes");
    if (A[0].part.kind == 0 && t.npoints() != 1) return bad("reduction inputs need a tiling when the domain has several points");
  } else if (op == DFS_OP_SPMV) {
    for (size_t k = 0; k < A.size(); ++k)
      if (A[k].imm) return bad("SPMV takes no immediates");
    const Arg &rp = A[0], &col = A[1], &val = A[2], &x = A[3], &y = A[4];
    if (rp.dtype != DFS_I32 || col.dtype != DFS_I32) return bad("SPMV rowptr and col are int32");
    if (!dtype_is_float(val.dtype) || x.dtype != val.dtype || y.dtype != val.dtype) return bad("SPMV val, x and y share one floating dtype");
    for (int k = 0; k < 4; ++k)
      if (A[k].priv != DFS_PRIV_R || A[k].part.kind != 0 || A[k].nd != 1) return bad("SPMV rowptr, col, val and x are 1-D, read (R) through None");
    if (!y.is_w() || y.nd != 1 || (y.part.kind != 1 && t.npoints() != 1)) return bad("SPMV y is 1-D, written through a tiling");
    const int64_t rows = y.part.vhi[0] - y.part.vlo[0];
    if (rp.part.vhi[0] - rp.part.vlo[0] != rows + 1) return bad("SPMV rowptr must have rows(y) + 1 entries");
    if (col.part.vhi[0] - col.part.vlo[0] != val.part.vhi[0] - val.part.vlo[0]) return bad("SPMV col and val lengths differ");
    if (A.size() == 6) {
      // the x-window hint: one record of 6 int32 per point of y's tiling
      const Arg& w = A[5];
      if (w.dtype != DFS_I32 || w.nd != 1 || w.priv != DFS_PRIV_R) return bad("SPMV windows are a 1-D int32 store read (R)");
      if (y.part.kind != 1 || w.part.kind != 1 || w.part.tile[0] != 6 || w.part.off[0] != w.part.vlo[0] ||
          w.part.proj[0] != y.part.proj[0])
        return bad("SPMV windows are read through a Tiling of 6 elements per point, projected like y");
      const int64_t ypts = (y.part.vhi[0] - y.part.off[0] + y.part.tile[0] - 1) / y.part.tile[0];
      if (w.part.vhi[0] - w.part.vlo[0] < 6 * std::max<int64_t>(ypts, t.dom[y.part.proj[0]]))
        return bad("SPMV windows need one 6-element record per point of the launch domain");
    }
  } else {
    return bad("unknown op");
  }
  return DFS_OK;
}

// -------------------------------------------------------------- flushing
struct WindowInfo {
  std::map<int64_t, RootInfo> roots;
  std::map<int64_t, int> canon;   // root -> canonical id
  std::vector<int64_t> by_canon;  // canonical id -> root
  std::string key;
};

WindowInfo window_info(dfs_ctx* c) {
  WindowInfo wi;
  for (const Task& t : c->window)
    for (const Arg& a : t.args) {
      if (a.imm) continue;
      if (!wi.canon.count(a.root)) {
        wi.canon[a.root] = (int)wi.by_canon.size();
        wi.by_canon.push_back(a.root);
      }
      if (wi.roots.count(a.root)) continue;
      const StoreRec& r = c->stores.at(a.root);
      RootInfo ri;
      ri.root = a.root;
      ri.ndim = r.ndim;
      for (int d = 0; d < MAXD; ++d) ri.shape[d] = d < r.ndim ? r.shape[d] : 0;
      ri.app_live = r.app_refs > 0;
      ri.wrapped = r.wrapped;
      ri.valid = r.valid;
      wi.roots[a.root] = ri;
    }
  // configuration, pointer alignment of every root, then the window's form
  std::string& k = wi.key;
  const int64_t head[] = {c->cfg.fusion, c->cfg.launch_mode, c->cfg.block_threads, c->cfg.unroll,
                          c->cfg.debug_skip_arrival, c->cfg.ctas_per_sm};
  k.append(reinterpret_cast<const char*>(head), sizeof head);
  for (int64_t r : wi.by_canon) {
    const StoreRec& s = c->stores.at(r);
    k.push_back((s.ptr && (uintptr_t)s.ptr % 16 != 0) ? 'u' : 'a');
  }
  k += canonical_key(c->window, wi.roots);
  return wi;
}

std::string plan_json(const Plan& p, const std::vector<Task>& w, const WindowInfo& wi) {
  std::ostringstream o;
  o << "{\"groups\": [";
  for (size_t g = 0; g < p.groups.size(); ++g) {
    o << (g ? ", " : "") << "[";
    for (int i = p.groups[g].begin; i < p.groups[g].end; ++i) o << (i > p.groups[g].begin ? ", " : "") << i;
    o << "]";
  }
  o << "], \"temporaries\": [";
  // roots temporary in every group that references them
  std::map<int64_t, std::pair<int, int>> cnt;  // root -> (groups referencing, groups temp)
  for (size_t g = 0; g < p.groups.size(); ++g) {
    std::set<int64_t> seen;
    for (int i = p.groups[g].begin; i < p.groups[g].end; ++i)
      for (const Arg& a : w[i].args)
        if (!a.imm) seen.insert(a.root);
    for (int64_t r : seen) {
      cnt[r].first++;
      if (p.temps.count({(int)g, r})) cnt[r].second++;
    }
  }
  bool first = true;
  for (int64_t r : wi.by_canon) {
    auto it = cnt.find(r);
    if (it != cnt.end() && it->second.first == it->second.second) {
      o << (first ? "" : ", ") << r;
      first = false;
    }
  }
  o << "], \"launches\": [";
  for (size_t l = 0; l < p.launches.size(); ++l) {
    o << (l ? ", " : "") << "[";
    for (int g = p.launches[l].first; g < p.launches[l].second; ++g) o << (g > p.launches[l].first ? ", " : "") << g;
    o << "]";
  }
  int bars = 0;
  for (const auto& L : p.launches)
    for (int g = L.first + 1; g < L.second; ++g)
      if (!p.groups[g - 1].scalar) ++bars;
  o << "], \"scalar_groups\": [";
  first = true;
  for (size_t g = 0; g < p.groups.size(); ++g)
    if (p.groups[g].scalar) {
      o << (first ? "" : ", ") << g;
      first = false;
    }
  o << "], \"barriers\": " << bars << "}";
  return o.str();
}

// Builds the cached form of a window: plan, generated and compiled kernels.
// The launch of fused groups [g0, g1) of window w: its tasks, groups and the
// role of every root (pointer parameter, temporary, 0-d value loaded before
// or published after the launch).  `valid` is the value state before it.
LaunchSpec make_spec(dfs_ctx* c, const std::vector<Task>& w, const std::map<int64_t, RootInfo>& roots,
                     const Plan& P, int g0, int g1, std::map<int64_t, bool>& valid) {
  const int t0 = P.groups[g0].begin, t1 = P.groups[g1 - 1].end;
  LaunchSpec spec;
  spec.block = c->cfg.block_threads;
  spec.min_blocks = c->cfg.ctas_per_sm;
  spec.unroll = c->cfg.unroll;
  spec.persistent = (g1 - g0) > 1;
  spec.debug_skip = c->cfg.debug_skip_arrival;
  for (int i = t0; i < t1; ++i) spec.tasks.push_back(w[i]);
  for (int g = g0; g < g1; ++g) {
    Group G = P.groups[g];
    G.begin -= t0;
    G.end -= t0;
    spec.groups.push_back(G);
  }
  std::map<int64_t, std::pair<int, int>> tcount;  // groups referencing / temp in
  for (int g = g0; g < g1; ++g) {
    std::set<int64_t> seen;
    for (int i = P.groups[g].begin; i < P.groups[g].end; ++i)
      for (const Arg& a : w[i].args)
        if (!a.imm) seen.insert(a.root);
    for (int64_t r : seen) {
      tcount[r].first++;
      if (P.temps.count({g, r})) tcount[r].second++;
    }
  }
  int nparam = 0;
  for (int i = t0; i < t1; ++i)
    for (const Arg& a : w[i].args) {
      if (a.imm || spec.root_index.count(a.root)) continue;
      const StoreRec& s = c->stores.at(a.root);
      LaunchRoot lr{};
      lr.root = a.root;
      lr.dtype = s.dtype;
      lr.ndim = s.ndim;
      for (int d = 0; d < MAXD; ++d) {
        lr.shape[d] = d < s.ndim ? s.shape[d] : 1;
        lr.stride[d] = d < s.ndim ? s.stride[d] : 1;
      }
      lr.zero_d = s.ndim == 0;
      lr.valid_before = valid[a.root];
      lr.aligned16 = s.ptr ? ((uintptr_t)s.ptr % 16 == 0) : true;
      lr.param = -1;
      spec.root_index[a.root] = (int)spec.roots.size();
      spec.roots.push_back(lr);
    }
  for (LaunchRoot& lr : spec.roots) {
    for (int i = t0; i < t1; ++i)
      for (const Arg& a : w[i].args) {
        if (a.imm || a.root != lr.root) continue;
        lr.written |= a.is_w() || a.is_rd();
        lr.read |= a.is_r();
      }
    const auto& tc = tcount[lr.root];
    const RootInfo& ri = roots.at(lr.root);
    if (lr.zero_d) {
      // 0-d values live in registers; memory is needed to load a prior value
      // or to publish the result beyond this launch
      bool used_later = false;
      for (int i = t1; i < (int)w.size(); ++i)
        for (const Arg& a : w[i].args)
          if (!a.imm && a.root == lr.root && (a.is_r() || a.is_rd())) used_later = true;
      lr.live_out = lr.written && (ri.app_live || ri.wrapped || used_later);
      lr.temp = !lr.live_out;
      bool load = false;
      if (lr.valid_before) {
        // first access in program order decides whether the old value is used
        for (int i = t0; i < t1 && !load; ++i) {
          bool touched = false;
          for (const Arg& a : w[i].args) {
            if (a.imm || a.root != lr.root) continue;
            touched = true;
            if (a.is_r() || a.is_rd()) load = true;
          }
          if (touched) break;
        }
      }
      lr.valid_before = lr.valid_before && load;
      if (load || lr.live_out) lr.param = nparam++;
    } else {
      lr.temp = c->cfg.fusion && tc.first > 0 && tc.first == tc.second;
      if (!lr.temp) lr.param = nparam++;
    }
  }
  return spec;
}

int build_window(dfs_ctx* c, const WindowInfo& wi, std::unique_ptr<CachedWindow>& out) {
  const auto& w = c->window;
  auto cw = std::make_unique<CachedWindow>();
  cw->plan = analyse(w, wi.roots, c->cfg.fusion != 0, c->cfg.launch_mode);
  const Plan& P = cw->plan;
  // value state through the window: valid before each launch
  std::map<int64_t, bool> valid;
  for (const auto& kv : wi.roots) valid[kv.first] = kv.second.valid;
  std::set<int64_t> need_mem;
  for (size_t li = 0; li < P.launches.size(); ++li) {
    const int g0 = P.launches[li].first, g1 = P.launches[li].second;
    const int t0 = P.groups[g0].begin, t1 = P.groups[g1 - 1].end;
    LaunchSpec spec = make_spec(c, w, wi.roots, P, g0, g1, valid);
    for (const LaunchRoot& lr : spec.roots)
      if (lr.param >= 0) need_mem.insert(lr.root);
    KernelCode kc;
    try {
      kc = generate(spec);
    } catch (const std::exception& e) {
      return fail(c, DFS_ERR_INVALID, std::string("code generation: ") + e.what());
    }
    std::string err;
    c->last_source = kc.source;
    if (!c->device) {
      // analysis-only context: check that the kernel compiles for the target
      if (!c->jit->compile_only(kc.source, kc.name, err)) return fail(c, DFS_ERR_COMPILE, err);
      continue;
    }
    const Compiled* comp = c->jit->get(kc.source, kc.name, spec.block, err, kc.dyn_smem);
    if (!comp) return fail(c, DFS_ERR_COMPILE, err);
    CachedLaunch L;
    L.k = comp;
    L.name = kc.name;
    L.block = spec.block;
    L.nbarriers = kc.nbarriers;
    L.cooperative = kc.nbarriers > 0;
    bool all_scalar = true;
    for (const Group& G : spec.groups) all_scalar &= G.scalar;
    // per-point groups want one CTA per point (more CTAs would only wait at
    // the barriers); kernels made only of flat sweeps use every resident CTA
    int64_t want = 1;
    if (!all_scalar) want = kc.has_points ? kc.max_points : (kc.has_flat ? INT64_MAX : 1);
    int per_sm = comp->occupancy > 0 ? comp->occupancy : 1;
    if (c->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, c->cfg.ctas_per_sm);
    const int64_t cap = (int64_t)per_sm * c->sms;
    if (L.cooperative && comp->occupancy <= 0) return fail(c, DFS_ERR_CUDA, "generated kernel cannot be resident for a cooperative launch");
    L.grid = (int)std::max<int64_t>(1, std::min(want, cap));
    L.nptr = kc.nptr;
    L.nimm = kc.nimm;
    for (int64_t r : kc.ptr_roots) L.ptr_canon.push_back(wi.canon.at(r));
    for (const auto& s : kc.imm_src) L.imm_src.push_back({s.first + t0, s.second});
    int64_t stride = 1;
    for (int64_t p : kc.red_points) stride = std::max(stride, p);
    L.red_stride = stride;
    L.partial_bytes = kc.partial_bytes;
    L.first_task = t0;
    L.last_task = t1;
    L.source = kc.source;
    cw->launches.push_back(L);
    for (const LaunchRoot& lr : spec.roots)
      if (lr.written && lr.param >= 0) valid[lr.root] = true;
  }
  for (int64_t r : need_mem) cw->materialise.push_back(wi.canon.at(r));
  for (const auto& kv : valid)
    if (kv.second && need_mem.count(kv.first)) cw->made_valid.push_back(wi.canon.at(kv.first));
  out = std::move(cw);
  return DFS_OK;
}

int run_window(dfs_ctx* c, const CachedWindow& cw, const WindowInfo& wi) {
  c->lastb.ok = false;
  for (int id : cw.materialise) {
    StoreRec& r = c->stores.at(wi.by_canon[id]);
    int rc = materialise(c, r);
    if (rc) return rc;
  }
  for (const CachedLaunch& L : cw.launches) {
    if (L.partial_bytes > c->partials_cap) {
      if (c->capturing)
        return fail(c, DFS_ERR_STATE, "reduction scratch would grow inside a capture: run the window once first");
      if (c->partials) cudaFreeAsync(c->partials, c->stream);
      c->partials = nullptr;
      size_t cap = std::max<size_t>(L.partial_bytes, 4096);
      CUDA_OK(cudaMallocAsync(&c->partials, cap, c->stream));
      c->partials_cap = cap;
    }
    std::vector<uint64_t> blob((size_t)std::max(1, L.nptr) + (size_t)std::max(1, L.nimm) + 4, 0);
    for (int i = 0; i < L.nptr; ++i) {
      const StoreRec& r = c->stores.at(wi.by_canon[L.ptr_canon[i]]);
      void* p = r.ptr;
      std::memcpy(&blob[i], &p, sizeof p);
    }
    const size_t ib = (size_t)std::max(1, L.nptr);
    for (int i = 0; i < L.nimm; ++i) {
      const double v = c->window[L.imm_src[i].first].args[L.imm_src[i].second].immv;
      std::memcpy(&blob[ib + i], &v, sizeof v);
    }
    const size_t tb = ib + (size_t)std::max(1, L.nimm);
    void* pp = c->partials;
    std::memcpy(&blob[tb], &pp, sizeof pp);
    void* cp = c->ctl;
    std::memcpy(&blob[tb + 1], &cp, sizeof cp);
    const uint64_t to = (uint64_t)(c->cfg.barrier_timeout_s * 1e9);
    blob[tb + 2] = to;
    const int64_t rs = L.red_stride;
    std::memcpy(&blob[tb + 3], &rs, sizeof rs);
    void* bp = blob.data();
    void* params[] = {bp};
    // the kernel takes one struct parameter: pass its bytes as the argument
    CUresult cr;
    dfs_ctx::Timed tm{nullptr, nullptr, L.name};
    const bool timing = c->cfg.time_launches && !c->capturing;
    if (timing) {
      for (cudaEvent_t* e : {&tm.a, &tm.b}) {
        if (!c->event_pool.empty()) {
          *e = c->event_pool.back();
          c->event_pool.pop_back();
        } else {
          CUDA_OK(cudaEventCreate(e));
        }
      }
      CUDA_OK(cudaEventRecord(tm.a, c->stream));
    }
    if (L.cooperative)
      cr = c->drv.LaunchCooperativeKernel(L.k->fn, L.grid, 1, 1, L.block, 1, 1, (unsigned)L.k->dyn_smem,
                                          (CUstream)c->stream, params);
    else
      cr = c->drv.LaunchKernel(L.k->fn, L.grid, 1, 1, L.block, 1, 1, (unsigned)L.k->dyn_smem, (CUstream)c->stream,
                               params, nullptr);
    if (cr != CUDA_SUCCESS) {
      const char* s = nullptr;
      c->drv.GetErrorString(cr, &s);
      return fail(c, DFS_ERR_CUDA, std::string("launch of ") + L.name + ": " + (s ? s : "?"));
    }
    if (timing) {
      CUDA_OK(cudaEventRecord(tm.b, c->stream));
      c->timed.push_back(tm);
    }
    if (c->capturing)
      c->capture_launches += 1;
    else
      c->st.launches += 1;
    c->st.last_regs = L.k->regs;
    c->st.last_occupancy = L.k->occupancy;
    c->st.last_grid = L.grid;
    c->st.last_block = L.block;
    c->st.barriers += L.nbarriers;
  }
  for (int id : cw.made_valid) c->stores.at(wi.by_canon[id]).valid = true;
  return DFS_OK;
}

void release_window(dfs_ctx* c) {
  std::vector<int64_t> roots;
  for (const Task& t : c->window)
    for (const Arg& a : t.args)
      if (!a.imm) {
        auto it = c->stores.find(a.root);
        if (it != c->stores.end()) it->second.pending -= 1;
        roots.push_back(a.root);
      }
  c->window.clear();
  std::sort(roots.begin(), roots.end());
  roots.erase(std::unique(roots.begin(), roots.end()), roots.end());
  for (int64_t r : roots) maybe_free(c, r);
}

// Window growth (Section 7.2): a full window that fused into one task
// doubles the window size, up to the configured cap.
void grow_window(dfs_ctx* c, const Plan& p) {
  const int cap = c->cfg.window_max > 0 ? c->cfg.window_max : 4096;
  if (c->cfg.window_growth && p.groups.size() == 1 && c->cfg.window_size < cap) {
    c->cfg.window_size = std::min(cap, 2 * c->cfg.window_size);
    c->st.window_growths += 1;
  }
}

int flush(dfs_ctx* c, bool size_trigger = false) {
  if (c->window.empty()) return DFS_OK;
  c->st.flushes += 1;
  const auto t0 = std::chrono::steady_clock::now();
  WindowInfo wi = window_info(c);
  CachedWindow* cw = nullptr;
  auto it = c->wcache.find(wi.key);
  if (it != c->wcache.end()) {
    c->st.plan_hits += 1;
    cw = it->second.get();
    if (size_trigger) grow_window(c, cw->plan);
  } else {
    c->st.plan_misses += 1;
    std::unique_ptr<CachedWindow> built;
    int rc = build_window(c, wi, built);
    if (rc) {
      release_window(c);
      return rc;
    }
    if (size_trigger) grow_window(c, built->plan);
    if (!c->device) {
      c->st.groups += (int64_t)built->plan.groups.size();
      release_window(c);
      return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context: window analysed, kernels compiled, not launched");
    }
    cw = built.get();
    c->wcache[wi.key] = std::move(built);
  }
  c->st.groups += (int64_t)cw->plan.groups.size();
  c->st.temporaries += (int64_t)cw->plan.temps.size();
  c->st.analysis_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (!cw->launches.empty()) c->last_source = cw->launches.back().source;
  int rc = run_window(c, *cw, wi);
  release_window(c);
  return rc;
}

// ------------------------------------------------------------- batching
// Root descriptions of one instance window, roots numbered by first use.
std::map<int64_t, RootInfo> root_infos(dfs_ctx* c, const std::vector<Task>& w, std::vector<int64_t>& order) {
  std::map<int64_t, RootInfo> m;
  for (const Task& t : w)
    for (const Arg& a : t.args) {
      if (a.imm || m.count(a.root)) continue;
      order.push_back(a.root);
      const StoreRec& r = c->stores.at(a.root);
      RootInfo ri;
      ri.root = a.root;
      ri.ndim = r.ndim;
      for (int d = 0; d < MAXD; ++d) ri.shape[d] = d < r.ndim ? r.shape[d] : 0;
      ri.app_live = r.app_refs > 0;
      ri.wrapped = r.wrapped;
      ri.valid = r.valid;
      m[a.root] = ri;
    }
  return m;
}

// Structure of one instance without its sizes: operations, privileges,
// dtypes, ranks, store liveness and the patterns of root, partition and
// launch-domain identity.  Equal keys mean the fusion pass treats the
// instances alike.
std::string batch_key(const std::vector<Task>& w, const std::map<int64_t, RootInfo>& roots) {
  std::map<int64_t, int64_t> rid;
  std::vector<NPart> parts;
  std::vector<const Task*> doms;
  std::string k;
  auto put = [&k](int64_t v) { k.append(reinterpret_cast<const char*>(&v), sizeof v); };
  for (const Task& t : w) {
    put(-1 - t.op);
    int64_t dc = -1;
    for (size_t i = 0; i < doms.size() && dc < 0; ++i)
      if (doms[i]->same_domain(t)) dc = (int64_t)i;
    if (dc < 0) {
      dc = (int64_t)doms.size();
      doms.push_back(&t);
    }
    put(dc);
    put(t.dnd);
    for (const Arg& a : t.args) {
      if (a.imm) {
        put(-7);
        continue;
      }
      auto it = rid.find(a.root);
      if (it == rid.end()) {
        const int64_t id = (int64_t)rid.size();
        rid[a.root] = id;
        const RootInfo& ri = roots.at(a.root);
        put(-8);
        put(a.dtype);
        put(ri.ndim);
        put((ri.app_live ? 1 : 0) | (ri.wrapped ? 2 : 0) | (ri.valid ? 4 : 0));
        put(id);
      } else {
        put(it->second);
      }
      put(a.priv * 16 + a.redop);
      int64_t pc = -1;
      for (size_t i = 0; i < parts.size() && pc < 0; ++i)
        if (parts[i] == a.part) pc = (int64_t)i;
      if (pc < 0) {
        pc = (int64_t)parts.size();
        parts.push_back(a.part);
      }
      put(pc);
      put(a.part.kind * 16 + a.part.nd);
    }
  }
  return k;
}

// One launch of a batched kernel (timing, statistics); also used by
// dfs_batch_repeat.
int launch_batched(dfs_ctx* c, const dfs_ctx::LastBatch& L) {
  const bool timing = c->cfg.time_launches && !c->capturing;
  dfs_ctx::Timed tm{nullptr, nullptr, L.name};
  if (timing) {
    for (cudaEvent_t* e : {&tm.a, &tm.b}) {
      if (!c->event_pool.empty()) {
        *e = c->event_pool.back();
        c->event_pool.pop_back();
      } else {
        CUDA_OK(cudaEventCreate(e));
      }
    }
    CUDA_OK(cudaEventRecord(tm.a, c->stream));
  }
  uint64_t blob[8];
  std::memcpy(blob, L.blob, sizeof blob);
  void* params[] = {blob};
  const unsigned sm = (unsigned)L.dyn_smem;
  CUresult cr = L.coop ? c->drv.LaunchCooperativeKernel(L.fn, L.grid, 1, 1, L.block, 1, 1, sm, (CUstream)c->stream, params)
                       : c->drv.LaunchKernel(L.fn, L.grid, 1, 1, L.block, 1, 1, sm, (CUstream)c->stream, params, nullptr);
  if (cr != CUDA_SUCCESS) {
    const char* es = nullptr;
    c->drv.GetErrorString(cr, &es);
    return fail(c, DFS_ERR_CUDA, std::string("batched launch: ") + (es ? es : "?"));
  }
  if (timing) {
    CUDA_OK(cudaEventRecord(tm.b, c->stream));
    c->timed.push_back(tm);
  }
  if (c->capturing)
    c->capture_launches += 1;
  else
    c->st.launches += 1;
  c->st.barriers += L.nbarriers;
  c->st.groups += L.groups;
  c->st.last_grid = L.grid;
  c->st.last_block = L.block;
  return DFS_OK;
}

int flush_batch(dfs_ctx* c) {
  const std::vector<Task>& w = c->window;
  std::vector<size_t> marks = c->batch_marks;
  if (marks.empty() || marks.back() != w.size()) marks.push_back(w.size());
  std::vector<std::pair<size_t, size_t>> inst;
  size_t s0 = 0;
  for (size_t m : marks) {
    if (m > s0) inst.push_back({s0, m});
    s0 = m;
  }
  auto fallback = [&](const std::string& why) {
    c->batch_fallbacks += 1;
    c->batch_fallback_reason = why;
    return flush(c);
  };
  // a single instance also takes the size-generic batched kernel: a stream
  // of one-off problems of new sizes then compiles nothing new
  if (inst.empty()) return flush(c);
  if (c->cfg.launch_mode != DFS_LAUNCH_PERSISTENT || !c->cfg.fusion) return fallback("batching runs fused, persistent launches");
  const int K = (int)inst.size();
  std::vector<std::vector<Task>> iw(K);
  std::vector<std::map<int64_t, RootInfo>> iroots(K);
  std::vector<std::vector<int64_t>> canon(K);
  for (int i = 0; i < K; ++i) {
    iw[i].assign(w.begin() + (long)inst[i].first, w.begin() + (long)inst[i].second);
    iroots[i] = root_infos(c, iw[i], canon[i]);
  }
  const std::string key0 = batch_key(iw[0], iroots[0]);
  for (int i = 1; i < K; ++i)
    if (batch_key(iw[i], iroots[i]) != key0) return fallback("instances are not isomorphic");
  // instances must be independent: a written root belongs to one instance
  {
    std::map<int64_t, int> writer, user;
    for (int i = 0; i < K; ++i)
      for (const Task& t : iw[i])
        for (const Arg& a : t.args) {
          if (a.imm) continue;
          auto u = user.find(a.root);
          if (u == user.end()) user[a.root] = i;
          if (a.is_w() || a.is_rd()) {
            auto wr = writer.find(a.root);
            if (wr != writer.end() && wr->second != i) return fallback("instances write a shared store");
            writer[a.root] = i;
          }
        }
    for (const auto& kv : writer)
      for (int i = 0; i < K; ++i)
        if (i != kv.second)
          for (const Task& t : iw[i])
            for (const Arg& a : t.args)
              if (!a.imm && a.root == kv.first) return fallback("an instance reads a store another writes");
  }
  // one plan for all: it must be the same for every instance
  const Plan p0 = analyse(iw[0], iroots[0], true, DFS_LAUNCH_PERSISTENT);
  if (p0.launches.size() != 1) return fallback("instance window longer than one launch");
  auto temps_canon = [&](const Plan& p, int i) {
    std::set<std::pair<int, int>> s;
    std::map<int64_t, int> ci;
    for (size_t k = 0; k < canon[i].size(); ++k) ci[canon[i][k]] = (int)k;
    for (const auto& tr : p.temps) s.insert({tr.first, ci.at(tr.second)});
    return s;
  };
  const auto t0c = temps_canon(p0, 0);
  for (int i = 1; i < K; ++i) {
    const Plan pi = analyse(iw[i], iroots[i], true, DFS_LAUNCH_PERSISTENT);
    bool same = pi.groups.size() == p0.groups.size();
    for (size_t g = 0; same && g < pi.groups.size(); ++g)
      same = pi.groups[g].begin == p0.groups[g].begin && pi.groups[g].end == p0.groups[g].end &&
             pi.groups[g].scalar == p0.groups[g].scalar;
    if (!same || temps_canon(pi, i) != t0c) return fallback("instance plans differ");
  }
  std::map<int64_t, bool> valid;
  for (const auto& kv : iroots[0]) valid[kv.first] = kv.second.valid;
  const LaunchSpec spec = make_spec(c, iw[0], iroots[0], p0, 0, (int)p0.groups.size(), valid);
  // vector width: every instance's streamed arrays must be 16-byte aligned
  size_t esz = 0;
  bool mixed = false;
  for (const Task& t : iw[0])
    for (size_t ai = 0; ai < t.args.size(); ++ai) {
      const Arg& a = t.args[ai];
      if (a.imm || a.nd == 0 || (t.op == DFS_OP_SPMV && ai != 4)) continue;
      if (esz && esz != dtype_size(a.dtype)) mixed = true;
      esz = dtype_size(a.dtype);
    }
  int vec = (esz && !mixed) ? (int)(16 / esz) : 1;
  for (int i = 0; i < K && vec > 1; ++i)
    for (const Task& t : iw[i])
      for (size_t ai = 0; ai < t.args.size(); ++ai) {
        const Arg& a = t.args[ai];
        if (a.imm || a.nd == 0 || (t.op == DFS_OP_SPMV && ai != 4)) continue;
        const StoreRec& r = c->stores.at(a.root);
        if ((r.ptr && (uintptr_t)r.ptr % 16) || a.part.tile[0] % vec || a.part.off[0] % vec || a.part.vlo[0] % vec)
          vec = 1;
      }
  // does some instance's SpMV share rows between lanes?
  bool lanes = false;
  for (int i = 0; i < K && !lanes; ++i)
    for (const Task& t : iw[i])
      if (t.op == DFS_OP_SPMV) {
        const NPart& cp = t.args[1].part;
        const NPart& rp = t.args[0].part;
        if (spmv_lanes(cp.vhi[0] - cp.vlo[0], rp.vhi[0] - rp.vlo[0] - 1) > 1) lanes = true;
      }
  // memoised kernel of this structure
  std::string ckey = key0;
  const int64_t cfgk[] = {vec, c->cfg.block_threads, c->cfg.unroll, c->cfg.debug_skip_arrival, lanes ? 1 : 0, c->cfg.ctas_per_sm};
  ckey.append(reinterpret_cast<const char*>(cfgk), sizeof cfgk);
  auto bit = c->bcache.find(ckey);
  dfs_ctx::BatchEntry* be = nullptr;
  if (bit != c->bcache.end()) {
    be = bit->second.get();
    c->st.plan_hits += 1;
  } else {
    c->st.plan_misses += 1;
    auto ne = std::make_unique<dfs_ctx::BatchEntry>();
    std::string why;
    if (!generate_batch(spec, vec, lanes, ne->code, why)) return fallback(why);
    std::string err;
    c->last_source = ne->code.source;
    if (!c->device) {
      // analysis-only: check that the batched kernel compiles, launch nothing
      const size_t ok = c->jit->compile_only(ne->code.source, ne->code.name, err);
      release_window(c);
      if (!ok) return fail(c, DFS_ERR_COMPILE, err);
      return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context: batched kernel compiled, not launched");
    }
    ne->k = c->jit->get(ne->code.source, ne->code.name, spec.block, err, ne->code.dyn_smem);
    if (!ne->k) {
      release_window(c);
      return fail(c, DFS_ERR_COMPILE, err);
    }
    ne->plan = p0;
    {
      std::map<int64_t, int> ci;
      for (size_t k = 0; k < canon[0].size(); ++k) ci[canon[0][k]] = (int)k;
      for (int64_t r : ne->code.ptr_roots) ne->ptr_canon.push_back(ci.at(r));
    }
    be = ne.get();
    c->bcache[ckey] = std::move(ne);
  }
  const BatchCode& bc = be->code;
  c->last_source = bc.source;  // cache hits too: the source of the most recent launch
  std::map<int64_t, int> ci0;
  for (size_t k = 0; k < canon[0].size(); ++k) ci0[canon[0][k]] = (int)k;
  const std::vector<int>& ptr_canon = be->ptr_canon;
  // descriptors and work lists
  const size_t NP = (size_t)std::max(1, bc.nptr), NIm = (size_t)std::max(1, bc.nimm), NV = (size_t)std::max(1, bc.nv);
  const size_t per = NP + NIm + NV;
  std::vector<int64_t> host((size_t)K * per + (size_t)bc.nprefix * (K + 1), 0);
  for (int i = 0; i < K; ++i) {
    int64_t* d = &host[(size_t)i * per];
    for (int k = 0; k < bc.nptr; ++k) {
      StoreRec& r = c->stores.at(canon[i][ptr_canon[k]]);
      const int rc = materialise(c, r);
      if (rc) {
        release_window(c);
        return rc;
      }
      std::memcpy(&d[k], &r.ptr, sizeof r.ptr);
    }
    for (int k = 0; k < bc.nimm; ++k) {
      const double v = iw[i][bc.imm_src[k].first].args[bc.imm_src[k].second].immv;
      std::memcpy(&d[NP + k], &v, sizeof v);
    }
    for (int k = 0; k < bc.nv; ++k) {
      const auto& src = bc.v_src[k];
      const Task& tk = iw[i][src.task];
      if (src.field == 4) {  // lanes per row of an SpMV task's matrix
        const NPart& cp = tk.args[1].part;
        const NPart& rp = tk.args[0].part;
        d[NP + NIm + k] = spmv_lanes(cp.vhi[0] - cp.vlo[0], rp.vhi[0] - rp.vlo[0] - 1);
        continue;
      }
      const NPart& p = tk.args[src.arg].part;
      const int64_t vals[] = {p.tile[0], p.off[0], p.vlo[0], p.vhi[0]};
      d[NP + NIm + k] = vals[src.field];
    }
  }
  int64_t red_stride = 1;
  for (int s = 0; s < bc.nprefix; ++s) {
    int64_t* pf = &host[(size_t)K * per + (size_t)s * (K + 1)];
    pf[0] = 0;
    for (int i = 0; i < K; ++i) pf[i + 1] = pf[i] + iw[i][bc.prefix_task[s]].npoints();
    red_stride = std::max(red_stride, pf[K]);
  }
  const std::string hkey(reinterpret_cast<const char*>(host.data()), host.size() * sizeof(int64_t));
  auto tit = c->tables.find(hkey);
  if (tit == c->tables.end()) {
    if (c->capturing) {
      release_window(c);
      return fail(c, DFS_ERR_STATE, "batch descriptors first seen inside a capture: run the batch once before");
    }
    if (c->tables.size() >= 256 && c->graphs.empty()) {
      for (auto& kv : c->tables) cudaFreeAsync(kv.second.dev, c->stream);
      c->tables.clear();
    }
    dfs_ctx::Table tb;
    tb.bytes = hkey.size();
    CUDA_OK(cudaMallocAsync(&tb.dev, tb.bytes, c->stream));
    CUDA_OK(cudaMemcpyAsync(tb.dev, host.data(), tb.bytes, cudaMemcpyHostToDevice, c->stream));
    tit = c->tables.emplace(hkey, tb).first;
  }
  const size_t sval_need = (size_t)K * (size_t)std::max(1, bc.nsval) * sizeof(double);
  const size_t part_need = (size_t)std::max(1, bc.nred) * (size_t)red_stride * 8;
  if (sval_need > c->sval_cap || part_need > c->partials_cap) {
    if (c->capturing) {
      release_window(c);
      return fail(c, DFS_ERR_STATE, "batch scratch would grow inside a capture: run the batch once before");
    }
    if (sval_need > c->sval_cap) {
      if (c->sval) cudaFreeAsync(c->sval, c->stream);
      CUDA_OK(cudaMallocAsync((void**)&c->sval, sval_need, c->stream));
      c->sval_cap = sval_need;
    }
    if (part_need > c->partials_cap) {
      if (c->partials) cudaFreeAsync(c->partials, c->stream);
      CUDA_OK(cudaMallocAsync(&c->partials, part_need, c->stream));
      c->partials_cap = part_need;
    }
  }
  // launch: struct BP { insts, prefix, sval, partials, ctl, timeout_ns, ninst, red_stride }
  uint64_t blob[8];
  void* insts = tit->second.dev;
  void* prefix = (char*)tit->second.dev + (size_t)K * per * 8;
  std::memcpy(&blob[0], &insts, 8);
  std::memcpy(&blob[1], &prefix, 8);
  std::memcpy(&blob[2], &c->sval, 8);
  std::memcpy(&blob[3], &c->partials, 8);
  std::memcpy(&blob[4], &c->ctl, 8);
  blob[5] = (uint64_t)(c->cfg.barrier_timeout_s * 1e9);
  const int64_t kk = K;
  std::memcpy(&blob[6], &kk, 8);
  std::memcpy(&blob[7], &red_stride, 8);
  int per_sm = be->k->occupancy > 0 ? be->k->occupancy : 1;
  if (c->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, c->cfg.ctas_per_sm);
  const int grid = std::max(1, per_sm * c->sms);
  const bool coop = bc.nbarriers > 0;
  if (coop && be->k->occupancy <= 0) {
    release_window(c);
    return fail(c, DFS_ERR_CUDA, "batched kernel cannot be resident for a cooperative launch");
  }
  dfs_ctx::LastBatch L;
  L.fn = be->k->fn;
  L.grid = grid;
  L.block = spec.block;
  L.dyn_smem = be->k->dyn_smem;
  L.coop = coop;
  L.nbarriers = bc.nbarriers;
  L.ninst = K;
  L.groups = (int64_t)p0.groups.size() * K;
  L.name = bc.name;
  L.source = &bc.source;
  std::memcpy(L.blob, blob, sizeof blob);
  c->lastb.ok = false;
  const int lrc = launch_batched(c, L);
  if (lrc) {
    release_window(c);
    return lrc;
  }
  c->st.last_regs = be->k->regs;
  c->st.last_occupancy = be->k->occupancy;
  // every written root that has memory now holds a value
  for (const LaunchRoot& lr : spec.roots) {
    if (lr.param < 0 || !lr.written) continue;
    const int k = ci0.at(lr.root);
    for (int i = 0; i < K; ++i) c->stores.at(canon[i][k]).valid = true;
  }
  c->batches += 1;
  c->batched_instances += K;
  // steady: every store of the batch held a value before it ran (or is a
  // temporary), so running the same kernel again is the same as submitting
  // the same instances again
  bool steady = !c->capturing;
  for (const LaunchRoot& lr : spec.roots)
    if (!lr.temp && !lr.valid_before) steady = false;
  if (steady) {
    c->lastb = L;
    c->lastb.ok = true;
  }
  release_window(c);
  return DFS_OK;
}

int write_json(const std::string& s, char* buf, size_t len, size_t* needed) {
  if (needed) *needed = s.size() + 1;
  if (!buf || len < s.size() + 1) {
    if (buf && len) buf[0] = 0;
    return DFS_ERR_BUFFER;
  }
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return DFS_OK;
}

}  // namespace
}  // namespace dfs

namespace dfs {
namespace {

// Checks of dfs_read_scalars and dfs_read_scalars_async; flushes.
int gather_check(dfs_ctx* c, int32_t n, const dfs_store* hs, const char* who) {
  if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
  if (c->capturing) return fail(c, DFS_ERR_STATE, std::string(who) + " while capturing");
  for (int32_t i = 0; i < n; ++i) {
    StoreRec* r = find_store(c, hs[i]);
    if (!r) return fail(c, DFS_ERR_STATE, "unknown or released store");
    if (r->ndim != 0) return fail(c, DFS_ERR_INVALID, std::string(who) + " takes 0-d stores");
  }
  int rc = flush(c);
  if (rc) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const StoreRec& r = *find_store(c, hs[i]);
    const StoreRec& root = c->stores.at(r.root);
    if (!root.ptr || !root.valid) return fail(c, DFS_ERR_STATE, "store has no value");
  }
  return DFS_OK;
}

// Grows the gather buffers to n scalars (synchronising the stream first, as
// the old buffers may still be in use).
int gather_reserve(dfs_ctx* c, int32_t n) {
  if ((size_t)n > c->gather_cap) {
    CUDA_OK(cudaStreamSynchronize(c->stream));
    if (c->gather_host) cudaFreeHost(c->gather_host);
    if (c->gather_dev) cudaFree(c->gather_dev);
    c->gather_host = nullptr;
    c->gather_dev = nullptr;
    c->gather_cap = 0;
    const size_t cap = std::max<size_t>(1024, (size_t)n);
    // per scalar: descriptor (address, dtype) then the gathered double
    CUDA_OK(cudaMallocHost((void**)&c->gather_host, cap * 3 * sizeof(int64_t)));
    CUDA_OK(cudaMalloc(&c->gather_dev, cap * 3 * sizeof(int64_t)));
    c->gather_cap = cap;
  }
  return DFS_OK;
}

// Enqueues the gather of n 0-d stores (n within the reserved capacity):
// descriptors (address, dtype) from desc_host (2 n int64, written here) to
// the device, the gather kernel, and the n doubles back to vals_host.  Both
// host buffers are page-locked and must stay untouched until the stream
// passes this point.
int gather_enqueue(dfs_ctx* c, int32_t n, const dfs_store* hs, int64_t* desc_host, double* vals_host) {
  for (int32_t i = 0; i < n; ++i) {
    const StoreRec& r = *find_store(c, hs[i]);
    const StoreRec& root = c->stores.at(r.root);
    const char* p = (const char*)root.ptr;
    for (int d = 0; d < root.ndim; ++d) p += (size_t)r.off[d] * root.stride[d] * dtype_size(r.dtype);
    desc_host[2 * i] = (int64_t)(uintptr_t)p;
    desc_host[2 * i + 1] = r.dtype;
  }
  int64_t* desc = static_cast<int64_t*>(c->gather_dev);
  double* vals = reinterpret_cast<double*>(desc + 2 * c->gather_cap);
  CUDA_OK(cudaMemcpyAsync(desc, desc_host, (size_t)n * 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(launch_gather_scalars(desc, n, vals, c->stream));
  CUDA_OK(cudaMemcpyAsync(vals_host, vals, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return DFS_OK;
}

bool page_locked(const void* p, size_t bytes) {
  cudaPointerAttributes a0{}, a1{};
  const char* last = (const char*)p + (bytes ? bytes - 1 : 0);
  const bool ok = cudaPointerGetAttributes(&a0, p) == cudaSuccess && a0.type == cudaMemoryTypeHost &&
                  cudaPointerGetAttributes(&a1, last) == cudaSuccess && a1.type == cudaMemoryTypeHost;
  if (!ok) cudaGetLastError();
  return ok;
}

cudaEvent_t* find_ticket(dfs_ctx* c, uint64_t t) {
  auto it = c->tickets.find(t);
  return it == c->tickets.end() ? nullptr : &it->second;
}

}  // namespace
}  // namespace dfs

namespace dfs {
namespace {

// Template recording: notes a store the recorded sequence uses; a store it
// did not create is an input of the template (first use fixes its dtype and
// shape, which every replay's store must match).
void rec_use(dfs_ctx* c, int64_t h) {
  if (c->rec_created.count(h)) return;
  for (int64_t e : c->rec.ext)
    if (e == h) return;
  const StoreRec* r = find_store(c, h);
  if (!r) return;
  std::array<int64_t, 2 + DFS_MAX_DIM> info{};
  info[0] = r->dtype;
  info[1] = r->ndim;
  for (int d = 0; d < r->ndim; ++d) info[2 + d] = r->shape[d];
  c->rec.ext.push_back(h);
  c->rec.ext_info.push_back(info);
}

// Entry points that a template cannot replay refuse to run while recording.
int refuse_recording(dfs_ctx* c, const char* who) {
  c->rec_fault = std::string(who) + " while recording a template";
  return fail(c, DFS_ERR_STATE, c->rec_fault);
}

}  // namespace
}  // namespace dfs

using namespace dfs;

// No C++ exception may cross the C ABI: an internal failure (a violated
// invariant surfacing as std::out_of_range, or std::bad_alloc) is reported
// as DFS_ERR_INVALID with its message in dfs_last_error.
static int internal_error(dfs_ctx* c, const char* what) {
  return fail(c, DFS_ERR_INVALID, std::string("internal error: ") + (what ? what : "?"));
}

extern "C" {

int dfs_version(void) { return 100; }

void dfs_config_default(dfs_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->fusion = 1;
  cfg->launch_mode = DFS_LAUNCH_PERSISTENT;
  cfg->window_size = 256;
  cfg->stream = nullptr;
  cfg->block_threads = 256;
  cfg->ctas_per_sm = 0;
  cfg->unroll = 2;
  cfg->barrier_timeout_s = 2.0;
  cfg->cache_dir = nullptr;
}

int dfs_init(dfs_ctx** out, const dfs_config* cfg_in) {
  try {
    if (!out) return DFS_ERR_INVALID;
    *out = nullptr;
    auto c = std::make_unique<dfs_ctx>();
    dfs_config cfg;
    dfs_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.window_size < 1) cfg.window_size = 1;
    if (cfg.block_threads == 0) cfg.block_threads = 256;
    if (cfg.block_threads != 128 && cfg.block_threads != 256 && cfg.block_threads != 512 && cfg.block_threads != 1024)
      return DFS_ERR_INVALID;
    if (cfg.unroll <= 0) cfg.unroll = 2;
    if (cfg.unroll > 8) cfg.unroll = 8;
    if (cfg.barrier_timeout_s <= 0) cfg.barrier_timeout_s = 2.0;
    if (cfg.launch_mode != DFS_LAUNCH_PER_TASK && cfg.launch_mode != DFS_LAUNCH_PERSISTENT) return DFS_ERR_INVALID;
    c->cfg = cfg;
    std::string cache_dir = cfg.cache_dir ? cfg.cache_dir : "";
    c->cfg.cache_dir = nullptr;
    if (cfg.device >= 0) {
      dfs_ctx* cp = c.get();
      int n = 0;
      cudaError_t e = cudaGetDeviceCount(&n);
      if (e != cudaSuccess || n <= cfg.device) return fail(nullptr, DFS_ERR_NO_DEVICE, "");
      if (cudaSetDevice(cfg.device) != cudaSuccess) return DFS_ERR_CUDA;
      cudaDeviceProp prop;
      if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) return DFS_ERR_CUDA;
      c->sms = prop.multiProcessorCount;
      std::string err;
      if (!driver_load(c->drv, err)) return DFS_ERR_CUDA;
      char arch[32];
      snprintf(arch, sizeof arch, "sm_%d%d%s", prop.major, prop.minor, prop.major >= 9 ? "a" : "");
      c->jit = std::make_unique<Jit>(&c->drv, arch, cache_dir);
      if (cfg.stream) {
        c->stream = (cudaStream_t)cfg.stream;
      } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return DFS_ERR_CUDA;
        c->own_stream = true;
      }
      // a failure from here on gives back the stream and control block
      auto undo = [&](int rc) {
        if (c->ctl) cudaFree(c->ctl);
        c->ctl = nullptr;
        if (c->own_stream) cudaStreamDestroy(c->stream);
        c->stream = nullptr;
        c->own_stream = false;
        return rc;
      };
      if (cudaMalloc(&c->ctl, sizeof(Ctl)) != cudaSuccess) {
        c->ctl = nullptr;
        return undo(DFS_ERR_OOM);
      }
      if (cudaMemset(c->ctl, 0, sizeof(Ctl)) != cudaSuccess) return undo(DFS_ERR_CUDA);
      if (cudaDeviceSynchronize() != cudaSuccess) return undo(DFS_ERR_CUDA);
      c->device = true;
      (void)cp;
    } else {
      // analysis-only: NVRTC still compiles generated kernels for sm_103a
      c->sms = 152;
      c->jit = std::make_unique<Jit>(&c->drv, "sm_103a", "");
    }
    *out = c.release();
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(nullptr, e_.what());
  } catch (...) {
    return internal_error(nullptr, "unknown exception");
  }
}

int dfs_shutdown(dfs_ctx* c) {
  try {
    if (!c) return DFS_OK;
    int rc = DFS_OK;
    if (c->device) {
      if (c->capturing) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(c->stream, &g);
        if (g) cudaGraphDestroy(g);
        c->capturing = false;
        for (void* p : c->capture_deferred) cudaFreeAsync(p, c->stream);
      }
      rc = flush(c);
      cudaStreamSynchronize(c->stream);
      for (auto& kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
        for (void* p : kv.second.owned) cudaFreeAsync(p, c->stream);
      }
      c->graphs.clear();
      for (auto& kv : c->stores)
        if (kv.second.owned && kv.second.ptr) cudaFreeAsync(kv.second.ptr, c->stream);
      if (c->partials) cudaFreeAsync(c->partials, c->stream);
      if (c->sval) cudaFreeAsync(c->sval, c->stream);
      for (auto& kv : c->tables) cudaFreeAsync(kv.second.dev, c->stream);
      c->tables.clear();
      cudaStreamSynchronize(c->stream);
      if (c->gather_host) cudaFreeHost(c->gather_host);
      if (c->gather_dev) cudaFree(c->gather_dev);
      for (auto& t : c->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
      }
      for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
      for (auto& kv : c->tickets) cudaEventDestroy(kv.second);
      for (cudaEvent_t e : c->ticket_pool) cudaEventDestroy(e);
      if (c->ctl) cudaFree(c->ctl);
      c->jit.reset();
      if (c->own_stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return rc;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

// Library-owned roots of rank >= 2 are pitched: every row (last dimension)
// starts on a 16-byte boundary, so row nests can use vector accesses even
// when the row length is not a multiple of the vector; wrapped memory keeps
// the caller's contiguous layout.
static int new_store(dfs_ctx* c, int32_t dtype, int32_t ndim, const int64_t* shape, dfs_store* out,
                     bool pitched) {
  if (!c || !out) return DFS_ERR_INVALID;
  if (dtype < DFS_F32 || dtype > DFS_I64) return fail(c, DFS_ERR_INVALID, "bad dtype");
  if (ndim < 0 || ndim > MAXD || (ndim > 0 && !shape)) return fail(c, DFS_ERR_INVALID, "bad ndim");
  StoreRec r;
  r.handle = c->next_handle++;
  r.dtype = dtype;
  r.ndim = ndim;
  r.root = r.handle;
  for (int d = 0; d < ndim; ++d) {
    if (shape[d] < 0) return fail(c, DFS_ERR_INVALID, "negative extent");
    r.shape[d] = shape[d];
  }
  int64_t s = 1;
  for (int d = ndim - 1; d >= 0; --d) {
    r.stride[d] = s;
    s *= r.shape[d];
    if (pitched && d == ndim - 1 && ndim >= 2) {
      const int64_t v = (int64_t)(16 / dtype_size(dtype));
      s = (r.shape[d] + v - 1) / v * v;  // row pitch in elements
    }
  }
  r.nbytes = r.nelem() ? (size_t)(ndim ? r.shape[0] * r.stride[0] : 1) * dtype_size(dtype) : 0;
  r.app_refs = 1;
  c->stores[r.handle] = r;
  *out = r.handle;
  return DFS_OK;
}

int dfs_store_create(dfs_ctx* c, int32_t dtype, int32_t ndim, const int64_t* shape, dfs_store* out) {
  try {
    const int rc = new_store(c, dtype, ndim, shape, out, true);
    if (rc == DFS_OK && c->recording) {
      dfs_ctx::RecEv ev;
      ev.kind = 0;
      ev.h = *out;
      ev.dtype = dtype;
      ev.ndim = ndim;
      for (int d = 0; d < ndim; ++d) ev.shape[d] = shape[d];
      c->rec.evs.push_back(ev);
      c->rec_created.insert(*out);
      c->rec_live.insert(*out);
    }
    return rc;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_store_wrap(dfs_ctx* c, int32_t dtype, int32_t ndim, const int64_t* shape, void* dev_ptr, dfs_store* out) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_store_wrap");
    if (!dev_ptr) return fail(c, DFS_ERR_INVALID, "null device pointer");
    int rc = new_store(c, dtype, ndim, shape, out, false);
    if (rc) return rc;
    StoreRec& r = c->stores.at(*out);
    r.ptr = dev_ptr;
    r.wrapped = true;
    r.valid = true;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_store_wrap_host(dfs_ctx* c, int32_t dtype, int32_t ndim, const int64_t* shape, void* host_ptr,
                        dfs_store* out) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_store_wrap_host");
    if (!host_ptr || !out) return fail(c, DFS_ERR_INVALID, "null pointer");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    if (dtype < DFS_F32 || dtype > DFS_I64 || ndim < 0 || ndim > MAXD || (ndim > 0 && !shape))
      return fail(c, DFS_ERR_INVALID, "bad dtype or shape");
    size_t n = 1;
    for (int d = 0; d < ndim; ++d) {
      if (shape[d] < 0) return fail(c, DFS_ERR_INVALID, "negative extent");
      n *= (size_t)shape[d];
    }
    const size_t bytes = n * dtype_size(dtype);
    void* dev = nullptr;
    void* dev_last = nullptr;
    char* last = (char*)host_ptr + (bytes ? bytes - 1 : 0);
    // only page-locked host memory (cudaHostAlloc / cudaHostRegister): its
    // pages stay resident; pageable memory can be unmapped under a kernel
    cudaPointerAttributes a0{}, a1{};
    if (cudaPointerGetAttributes(&a0, host_ptr) != cudaSuccess || a0.type != cudaMemoryTypeHost ||
        cudaPointerGetAttributes(&a1, last) != cudaSuccess || a1.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return fail(c, DFS_ERR_INVALID, "not page-locked host memory");
    }
    if (cudaHostGetDevicePointer(&dev, host_ptr, 0) != cudaSuccess || !dev ||
        cudaHostGetDevicePointer(&dev_last, last, 0) != cudaSuccess ||
        (char*)dev_last - (char*)dev != last - (char*)host_ptr) {
      cudaGetLastError();  // clear the sticky-free error of the failed query
      return fail(c, DFS_ERR_INVALID, "not mapped page-locked host memory over the whole range");
    }
    int rc = new_store(c, dtype, ndim, shape, out, false);
    if (rc) return rc;
    StoreRec& r = c->stores.at(*out);
    r.ptr = dev;
    r.wrapped = true;
    r.valid = true;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_host_alloc(size_t bytes, void** out) {
  if (!out) return DFS_ERR_INVALID;
  *out = nullptr;
  if (!bytes) return DFS_OK;
  if (cudaHostAlloc(out, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess || !*out) {
    cudaGetLastError();
    *out = nullptr;
    return DFS_ERR_OOM;
  }
  return DFS_OK;
}

int dfs_host_free(void* p) {
  if (p && cudaFreeHost(p) != cudaSuccess) {
    cudaGetLastError();
    return DFS_ERR_CUDA;
  }
  return DFS_OK;
}

int dfs_store_view(dfs_ctx* c, dfs_store parent, const int64_t* offset, const int64_t* shape, dfs_store* out) {
  try {
    if (!c || !out) return DFS_ERR_INVALID;
    StoreRec* p = find_store(c, parent);
    if (!p) return fail(c, DFS_ERR_STATE, "unknown or released parent store");
    if (p->ndim > 0 && (!offset || !shape)) return fail(c, DFS_ERR_INVALID, "view needs offset and shape");
    StoreRec v;
    v.handle = c->next_handle++;
    v.dtype = p->dtype;
    v.ndim = p->ndim;
    v.root = p->root;
    for (int d = 0; d < p->ndim; ++d) {
      if (offset[d] < 0 || shape[d] < 0 || offset[d] + shape[d] > p->shape[d])
        return fail(c, DFS_ERR_INVALID, "view box outside its parent");
      v.shape[d] = shape[d];
      v.off[d] = p->off[d] + offset[d];
    }
    StoreRec& root = c->stores.at(p->root);
    root.app_refs += 1;
    c->stores[v.handle] = v;
    *out = v.handle;
    if (c->recording) {
      rec_use(c, parent);
      dfs_ctx::RecEv ev;
      ev.kind = 1;
      ev.h = v.handle;
      ev.parent = parent;
      ev.ndim = v.ndim;
      for (int d = 0; d < v.ndim; ++d) {
        ev.off[d] = offset[d];
        ev.shape[d] = shape[d];
      }
      c->rec.evs.push_back(ev);
      c->rec_created.insert(v.handle);
      c->rec_live.insert(v.handle);
    }
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_store_release(dfs_ctx* c, dfs_store s) {
  try {
    if (!c) return DFS_ERR_INVALID;
    StoreRec* r = find_store(c, s);
    if (!r) return fail(c, DFS_ERR_STATE, "unknown or already released store");
    if (c->recording) {
      if (!c->rec_created.count(s)) {
        c->rec_fault = "a template may release only stores it created";
      } else {
        dfs_ctx::RecEv ev;
        ev.kind = 3;
        ev.h = s;
        c->rec.evs.push_back(ev);
        c->rec_live.erase(s);
      }
    }
    const int64_t root = r->root;
    r->released = true;
    StoreRec& rr = c->stores.at(root);
    rr.app_refs -= 1;
    if (r->handle != root) c->stores.erase(s);
    maybe_free(c, root);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_store_write(dfs_ctx* c, dfs_store s, const void* host_src, size_t bytes) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_store_write");
    StoreRec* r = find_store(c, s);
    if (!r) return fail(c, DFS_ERR_STATE, "unknown or released store");
    if (r->root != r->handle) return fail(c, DFS_ERR_INVALID, "write a root store, not a view");
    const size_t es = dtype_size(r->dtype);
    if (bytes != (size_t)r->nelem() * es) return fail(c, DFS_ERR_INVALID, "byte count does not match the store");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    int rc = flush(c);
    if (rc) return rc;
    rc = materialise(c, *r);
    if (rc) return rc;
    const int nd = r->ndim;
    if (nd >= 2 && r->stride[nd - 2] != r->shape[nd - 1]) {
      // pitched rows: one 2-D copy over every row of every plane
      const size_t w = (size_t)r->shape[nd - 1] * es;
      const size_t h = bytes ? bytes / w : 0;
      if (h) CUDA_OK(cudaMemcpy2DAsync(r->ptr, (size_t)r->stride[nd - 2] * es, host_src, w, w, h,
                                       cudaMemcpyHostToDevice, c->stream));
    } else if (bytes) {
      CUDA_OK(cudaMemcpyAsync(r->ptr, host_src, bytes, cudaMemcpyHostToDevice, c->stream));
    }
    r->valid = true;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

static int check_device_error(dfs_ctx* c) {
  Ctl h;
  CUDA_OK(cudaMemcpy(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost));
  if (h.err != 0) {
    cudaMemset(c->ctl, 0, sizeof(Ctl));
    cudaDeviceSynchronize();
    if (h.err == 2)
      return fail(c, DFS_ERR_BARRIER_TIMEOUT, "a staged SpMV copy of x did not complete in time");
    return fail(c, DFS_ERR_BARRIER_TIMEOUT, "a grid barrier timed out (barrier " + std::to_string(h.err_where) + ")");
  }
  return DFS_OK;
}

int dfs_store_read(dfs_ctx* c, dfs_store s, void* host_dst, size_t bytes) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_store_read");
    StoreRec* r = find_store(c, s);
    if (!r) return fail(c, DFS_ERR_STATE, "unknown or released store");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    if (c->capturing) return fail(c, DFS_ERR_STATE, "dfs_store_read while capturing");
    const size_t es = dtype_size(r->dtype);
    if (bytes != (size_t)r->nelem() * es) return fail(c, DFS_ERR_INVALID, "byte count does not match the store");
    int rc = flush(c);
    if (rc) return rc;
    StoreRec& root = c->stores.at(r->root);
    if (!root.ptr) return fail(c, DFS_ERR_STATE, "store has no value");
    if (bytes) {
      if (r->ndim <= 1) {
        const char* src = (const char*)root.ptr + (size_t)(r->ndim ? r->off[0] : 0) * es;
        CUDA_OK(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
      } else if (r->ndim == 2) {
        const char* src = (const char*)root.ptr + ((size_t)r->off[0] * root.stride[0] + (size_t)r->off[1]) * es;
        CUDA_OK(cudaMemcpy2DAsync(host_dst, (size_t)r->shape[1] * es, src, (size_t)root.stride[0] * es,
                                  (size_t)r->shape[1] * es, (size_t)r->shape[0], cudaMemcpyDeviceToHost, c->stream));
      } else {
        for (int64_t i = 0; i < r->shape[0]; ++i) {
          const char* src = (const char*)root.ptr +
                            ((size_t)(r->off[0] + i) * root.stride[0] + (size_t)r->off[1] * root.stride[1] + (size_t)r->off[2]) * es;
          CUDA_OK(cudaMemcpy2DAsync((char*)host_dst + (size_t)i * r->shape[1] * r->shape[2] * es, (size_t)r->shape[2] * es,
                                    src, (size_t)root.stride[1] * es, (size_t)r->shape[2] * es, (size_t)r->shape[1],
                                    cudaMemcpyDeviceToHost, c->stream));
        }
      }
    }
    CUDA_OK(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_store_device_ptr(dfs_ctx* c, dfs_store s, void** out) {
  try {
    if (!c || !out) return DFS_ERR_INVALID;
    StoreRec* r = find_store(c, s);
    if (!r) return fail(c, DFS_ERR_STATE, "unknown or released store");
    int rc = flush(c);
    if (rc) return rc;
    StoreRec& root = c->stores.at(r->root);
    rc = materialise(c, root);
    if (rc) return rc;
    size_t off = 0;
    for (int d = 0; d < r->ndim; ++d) off += (size_t)r->off[d] * root.stride[d];
    *out = (char*)root.ptr + off * dtype_size(r->dtype);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_partition_none(dfs_ctx* c, dfs_partition* out) {
  try {
    if (!c || !out) return DFS_ERR_INVALID;
    PartRec p;
    p.kind = 0;
    const int64_t h = c->next_handle++;
    c->parts[h] = p;
    *out = h;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_partition_tiling(dfs_ctx* c, int32_t ndim, const int64_t* tile, const int64_t* offset, const int32_t* proj,
                         dfs_partition* out) {
  try {
    if (!c || !out) return DFS_ERR_INVALID;
    if (ndim < 1 || ndim > MAXD || !tile) return fail(c, DFS_ERR_INVALID, "bad tiling rank");
    PartRec p;
    p.kind = 1;
    p.ndim = ndim;
    for (int d = 0; d < ndim; ++d) {
      if (tile[d] <= 0) return fail(c, DFS_ERR_INVALID, "tile extents must be positive");
      p.tile[d] = tile[d];
      p.off[d] = offset ? offset[d] : 0;
      p.proj[d] = proj ? proj[d] : d;
      if (p.proj[d] < 0 || p.proj[d] >= MAXD) return fail(c, DFS_ERR_INVALID, "bad projection");
    }
    const int64_t h = c->next_handle++;
    c->parts[h] = p;
    *out = h;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_submit(dfs_ctx* c, int32_t op, int32_t ndim, const int64_t* dom, int32_t nargs, const dfs_arg* args) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!arity_ok(op, nargs) || !args) return fail(c, DFS_ERR_INVALID, "unknown op or wrong argument count");
    if (ndim < 1 || ndim > MAXD || !dom) return fail(c, DFS_ERR_INVALID, "launch domain rank must be 1..3");
    Task t;
    t.op = op;
    t.dnd = ndim;
    for (int d = 0; d < ndim; ++d) {
      if (dom[d] < 1) return fail(c, DFS_ERR_INVALID, "launch domain extents must be >= 1");
      t.dom[d] = dom[d];
    }
    t.seq = c->seq;
    for (int i = 0; i < nargs; ++i) {
      const dfs_arg& in = args[i];
      Arg a;
      if (in.privilege == DFS_PRIV_IMM) {
        a.imm = true;
        a.immv = in.imm;
        a.priv = DFS_PRIV_IMM;
        t.args.push_back(a);
        continue;
      }
      if (in.privilege != DFS_PRIV_R && in.privilege != DFS_PRIV_W && in.privilege != DFS_PRIV_RW &&
          in.privilege != DFS_PRIV_RD)
        return fail(c, DFS_ERR_INVALID, "bad privilege");
      if (in.privilege == DFS_PRIV_RD && in.redop != DFS_REDOP_SUM) return fail(c, DFS_ERR_INVALID, "RD needs a reduction operator");
      StoreRec* s = find_store(c, in.store);
      if (!s) return fail(c, DFS_ERR_STATE, "task names an unknown or released store");
      auto pit = c->parts.find(in.partition);
      if (pit == c->parts.end()) return fail(c, DFS_ERR_STATE, "task names an unknown partition");
      const PartRec& P = pit->second;
      a.store = in.store;
      a.root = s->root;
      a.priv = in.privilege;
      a.redop = in.redop;
      a.dtype = s->dtype;
      a.nd = s->ndim;
      a.part.kind = P.kind;
      a.part.nd = s->ndim;
      if (P.kind == 1 && P.ndim != s->ndim) return fail(c, DFS_ERR_INVALID, "tiling rank differs from the store's");
      for (int d = 0; d < s->ndim; ++d) {
        a.part.vlo[d] = s->off[d];
        a.part.vhi[d] = s->off[d] + s->shape[d];
        if (P.kind == 1) {
          a.part.tile[d] = P.tile[d];
          a.part.off[d] = s->off[d] + P.off[d];
          a.part.proj[d] = P.proj[d];
        }
      }
      t.args.push_back(a);
    }
    int rc = validate(c, t);
    if (rc) return rc;
    if (c->recording) {
      dfs_ctx::RecEv ev;
      ev.kind = 2;
      ev.op = op;
      ev.ndim = ndim;
      for (int d = 0; d < ndim; ++d) ev.dom[d] = dom[d];
      ev.args.assign(args, args + nargs);
      for (int i = 0; i < nargs; ++i)
        if (args[i].privilege != DFS_PRIV_IMM) rec_use(c, args[i].store);
      c->rec.evs.push_back(std::move(ev));
    }
    for (const Arg& a : t.args)
      if (!a.imm) c->stores.at(a.root).pending += 1;
    c->window.push_back(std::move(t));
    c->seq += 1;
    c->st.tasks += 1;
    if ((int)c->window.size() >= c->cfg.window_size && !c->batching) return flush(c, true);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_flush(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    return flush(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_sync(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!c->device) return DFS_OK;
    if (c->capturing) return fail(c, DFS_ERR_STATE, "dfs_sync while capturing");
    int rc = flush(c);
    if (rc) return rc;
    CUDA_OK(cudaStreamSynchronize(c->stream));
    for (auto& t : c->timed) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
        auto& kt = c->ktime[t.name];
        kt.first += ms;
        kt.second += 1;
      }
      c->event_pool.push_back(t.a);
      c->event_pool.push_back(t.b);
    }
    c->timed.clear();
    return check_device_error(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_capture_begin(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_capture_begin");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    if (c->capturing) return fail(c, DFS_ERR_STATE, "already capturing");
    int rc = flush(c);
    if (rc) return rc;
    c->lastb.ok = false;
    // reduction scratch cannot be reallocated inside a capture: reserve 1 MB
    const size_t want = 1 << 20;
    if (c->partials_cap < want) {
      if (c->partials) cudaFreeAsync(c->partials, c->stream);
      c->partials = nullptr;
      CUDA_OK(cudaMallocAsync(&c->partials, want, c->stream));
      c->partials_cap = want;
    }
    CUDA_OK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->captured_allocs.clear();
    c->capture_deferred.clear();
    c->capture_launches = 0;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_capture_end(dfs_ctx* c, dfs_graph* out) {
  try {
    if (!c || !out) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_capture_end");
    if (!c->capturing) return fail(c, DFS_ERR_STATE, "not capturing");
    int rc = flush(c);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->capturing = false;
    std::vector<void*> deferred;
    deferred.swap(c->capture_deferred);
    auto give_back = [&]() {
      for (void* p : deferred) cudaFreeAsync(p, c->stream);
      // addresses handed out inside an abandoned capture belong to no live
      // allocation: those stores lose their memory (and value)
      for (int64_t r : c->captured_allocs) {
        auto it = c->stores.find(r);
        if (it == c->stores.end()) continue;
        it->second.ptr = nullptr;
        it->second.owned = false;
        it->second.valid = false;
      }
      c->captured_allocs.clear();
    };
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      give_back();
      return rc;
    }
    if (e != cudaSuccess || !graph) {
      give_back();
      return fail(c, DFS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    if (!c->captured_allocs.empty()) {
      cudaGraphDestroy(graph);
      give_back();
      return fail(c, DFS_ERR_STATE, "a store created inside the captured region is still referenced");
    }
    dfs_ctx::GraphRec g;
    g.graph = graph;
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      give_back();
      return fail(c, DFS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    g.owned.swap(deferred);
    g.launches = c->capture_launches;
    const int64_t h = c->next_handle++;
    c->graphs[h] = std::move(g);
    *out = h;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_graph_launch(dfs_ctx* c, dfs_graph h) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_graph_launch");
    auto it = c->graphs.find(h);
    if (it == c->graphs.end()) return fail(c, DFS_ERR_STATE, "unknown graph");
    if (c->capturing) return fail(c, DFS_ERR_STATE, "cannot launch a graph while capturing");
    int rc = flush(c);
    if (rc) return rc;
    c->lastb.ok = false;
    CUDA_OK(cudaGraphLaunch(it->second.exec, c->stream));
    c->st.launches += it->second.launches;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_graph_destroy(dfs_ctx* c, dfs_graph h) {
  try {
    if (!c) return DFS_ERR_INVALID;
    auto it = c->graphs.find(h);
    if (it == c->graphs.end()) return fail(c, DFS_ERR_STATE, "unknown graph");
    cudaGraphExecDestroy(it->second.exec);
    cudaGraphDestroy(it->second.graph);
    for (void* p : it->second.owned) cudaFreeAsync(p, c->stream);
    c->graphs.erase(it);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_batch_begin(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_batch_begin");
    if (c->batching) return fail(c, DFS_ERR_STATE, "already batching");
    const int rc = flush(c);
    if (rc) return rc;
    c->batching = true;
    c->batch_marks.clear();
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_batch_next(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_batch_next");
    if (!c->batching) return fail(c, DFS_ERR_STATE, "dfs_batch_next outside a batch");
    c->batch_marks.push_back(c->window.size());
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_batch_end(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_batch_end");
    if (!c->batching) return fail(c, DFS_ERR_STATE, "dfs_batch_end outside a batch");
    c->batching = false;
    const int rc = flush_batch(c);
    c->batch_marks.clear();
    return rc;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_batch_repeat(dfs_ctx* c, int32_t n) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_batch_repeat");
    if (n < 0) return fail(c, DFS_ERR_INVALID, "negative repeat count");
    if (c->batching) return fail(c, DFS_ERR_STATE, "dfs_batch_repeat inside a batch");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    const int rc = flush(c);
    if (rc) return rc;
    if (!c->lastb.ok) return fail(c, DFS_ERR_STATE, "no steady batch to repeat");
    if (n > 0 && c->lastb.source) c->last_source = *c->lastb.source;
    for (int32_t i = 0; i < n; ++i) {
      const int lrc = launch_batched(c, c->lastb);
      if (lrc) {
        c->lastb.ok = false;
        return lrc;
      }
      c->batches += 1;
      c->batch_repeats += 1;
      c->batched_instances += c->lastb.ninst;
    }
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_read_scalars(dfs_ctx* c, int32_t n, const dfs_store* hs, double* out) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_read_scalars");
    if (n < 0 || (n > 0 && (!hs || !out))) return fail(c, DFS_ERR_INVALID, "bad arguments");
    int rc = gather_check(c, n, hs, "dfs_read_scalars");
    if (rc) return rc;
    if (n == 0) {
      CUDA_OK(cudaStreamSynchronize(c->stream));
      return check_device_error(c);
    }
    rc = gather_reserve(c, n);
    if (rc) return rc;
    double* hv = reinterpret_cast<double*>(c->gather_host + 2 * c->gather_cap);
    rc = gather_enqueue(c, n, hs, c->gather_host, hv);
    if (rc) return rc;
    CUDA_OK(cudaStreamSynchronize(c->stream));
    std::memcpy(out, hv, (size_t)n * sizeof(double));
    return check_device_error(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_read_scalars_async(dfs_ctx* c, int32_t n, const dfs_store* hs, int64_t* host_work, double* host_vals) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_read_scalars_async");
    if (n < 0 || (n > 0 && (!hs || !host_work || !host_vals))) return fail(c, DFS_ERR_INVALID, "bad arguments");
    if (n > 0 && (!page_locked(host_work, (size_t)n * 2 * sizeof(int64_t)) ||
                  !page_locked(host_vals, (size_t)n * sizeof(double))))
      return fail(c, DFS_ERR_INVALID, "host buffers must be page-locked");
    int rc = gather_check(c, n, hs, "dfs_read_scalars_async");
    if (rc || n == 0) return rc;
    rc = gather_reserve(c, n);
    if (rc) return rc;
    return gather_enqueue(c, n, hs, host_work, host_vals);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_record(dfs_ctx* c, uint64_t* ticket) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return refuse_recording(c, "dfs_record");
    if (!ticket) return fail(c, DFS_ERR_INVALID, "null ticket");
    if (!c->device) return fail(c, DFS_ERR_NO_DEVICE, "analysis-only context");
    if (c->capturing) return fail(c, DFS_ERR_STATE, "dfs_record while capturing");
    int rc = flush(c);
    if (rc) return rc;
    cudaEvent_t ev;
    if (!c->ticket_pool.empty()) {
      ev = c->ticket_pool.back();
      c->ticket_pool.pop_back();
    } else {
      CUDA_OK(cudaEventCreate(&ev));
    }
    const cudaError_t e = cudaEventRecord(ev, c->stream);
    if (e != cudaSuccess) {
      c->ticket_pool.push_back(ev);
      return fail(c, DFS_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
    }
    const uint64_t t = c->next_ticket++;
    c->tickets[t] = ev;
    *ticket = t;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_wait(dfs_ctx* c, uint64_t ticket) {
  try {
    if (!c) return DFS_ERR_INVALID;
    cudaEvent_t* ev = find_ticket(c, ticket);
    if (!ev) return fail(c, DFS_ERR_STATE, "unknown ticket");
    CUDA_OK(cudaEventSynchronize(*ev));
    return check_device_error(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_poll(dfs_ctx* c, uint64_t ticket, int32_t* done) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!done) return fail(c, DFS_ERR_INVALID, "null result");
    cudaEvent_t* ev = find_ticket(c, ticket);
    if (!ev) return fail(c, DFS_ERR_STATE, "unknown ticket");
    const cudaError_t e = cudaEventQuery(*ev);
    if (e == cudaErrorNotReady) {
      *done = 0;
      return DFS_OK;
    }
    CUDA_OK(e);
    *done = 1;
    return check_device_error(c);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_ticket_elapsed_ms(dfs_ctx* c, uint64_t from, uint64_t to, float* ms) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!ms) return fail(c, DFS_ERR_INVALID, "null result");
    cudaEvent_t* a = find_ticket(c, from);
    cudaEvent_t* b = find_ticket(c, to);
    if (!a || !b) return fail(c, DFS_ERR_STATE, "unknown ticket");
    const cudaError_t e = cudaEventElapsedTime(ms, *a, *b);
    if (e == cudaErrorNotReady) {
      cudaGetLastError();
      return fail(c, DFS_ERR_STATE, "ticket not complete");
    }
    CUDA_OK(e);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_ticket_release(dfs_ctx* c, uint64_t ticket) {
  try {
    if (!c) return DFS_ERR_INVALID;
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) return fail(c, DFS_ERR_STATE, "unknown ticket");
    c->ticket_pool.push_back(it->second);
    c->tickets.erase(it);
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_template_begin(dfs_ctx* c) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (c->recording) return fail(c, DFS_ERR_STATE, "already recording a template");
    if (c->capturing) return fail(c, DFS_ERR_STATE, "dfs_template_begin while capturing");
    c->recording = true;
    c->rec = dfs_ctx::Template{};
    c->rec_created.clear();
    c->rec_live.clear();
    c->rec_fault.clear();
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_template_end(dfs_ctx* c, uint64_t* id) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!c->recording) return fail(c, DFS_ERR_STATE, "not recording a template");
    c->recording = false;
    std::string why = c->rec_fault;
    if (why.empty() && !c->rec_live.empty()) why = "the recorded sequence did not release every store it created";
    if (why.empty() && !id) why = "null template id";
    if (!why.empty()) {
      c->rec = dfs_ctx::Template{};
      return fail(c, id ? DFS_ERR_STATE : DFS_ERR_INVALID, why);
    }
    const uint64_t t = c->next_template++;
    c->templates[t] = std::move(c->rec);
    c->rec = dfs_ctx::Template{};
    *id = t;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_template_inputs(dfs_ctx* c, uint64_t id, int32_t cap, dfs_store* out, int32_t* n) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!n || (cap > 0 && !out) || cap < 0) return fail(c, DFS_ERR_INVALID, "bad arguments");
    auto it = c->templates.find(id);
    if (it == c->templates.end()) return fail(c, DFS_ERR_STATE, "unknown template");
    const auto& ext = it->second.ext;
    *n = (int32_t)ext.size();
    for (int32_t i = 0; i < cap && i < (int32_t)ext.size(); ++i) out[i] = ext[i];
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_template_replay(dfs_ctx* c, uint64_t id, int32_t n, const dfs_store* from, const dfs_store* to) {
  // stores this replay created and has not released yet: if a step fails,
  // their application references are dropped, so nothing the caller cannot
  // name stays allocated (tasks already issued keep what they use alive)
  std::vector<dfs_store> live;
  auto undo = [&]() {
    if (!c || live.empty()) return;
    const std::string why = c->err;
    for (auto h = live.rbegin(); h != live.rend(); ++h)
      if (find_store(c, *h)) dfs_store_release(c, *h);
    c->err = why;
  };
  try {
    if (!c) return DFS_ERR_INVALID;
    if (n < 0 || (n > 0 && (!from || !to))) return fail(c, DFS_ERR_INVALID, "bad arguments");
    if (c->recording) return fail(c, DFS_ERR_STATE, "dfs_template_replay while recording a template");
    auto it = c->templates.find(id);
    if (it == c->templates.end()) return fail(c, DFS_ERR_STATE, "unknown template");
    const dfs_ctx::Template& T = it->second;
    std::unordered_map<int64_t, int64_t> m;
    for (int32_t i = 0; i < n; ++i) m[from[i]] = to[i];
    // every input mapped to a live store of the recorded dtype and shape,
    // checked before anything is issued
    for (size_t k = 0; k < T.ext.size(); ++k) {
      auto mi = m.find(T.ext[k]);
      if (mi == m.end()) return fail(c, DFS_ERR_INVALID, "a template input is not mapped");
      const StoreRec* r = find_store(c, mi->second);
      if (!r) return fail(c, DFS_ERR_STATE, "a template input maps to an unknown or released store");
      const auto& info = T.ext_info[k];
      bool same = r->dtype == info[0] && r->ndim == info[1];
      for (int d = 0; same && d < r->ndim; ++d) same = r->shape[d] == info[2 + d];
      if (!same) return fail(c, DFS_ERR_INVALID, "a template input maps to a store of another dtype or shape");
    }
    std::vector<dfs_arg> args;
    for (const dfs_ctx::RecEv& ev : T.evs) {
      int rc = DFS_OK;
      if (ev.kind == 0) {
        dfs_store h = 0;
        rc = new_store(c, ev.dtype, ev.ndim, ev.shape, &h, true);
        m[ev.h] = h;
        if (!rc) live.push_back(h);
      } else if (ev.kind == 1) {
        dfs_store h = 0;
        rc = dfs_store_view(c, m.at(ev.parent), ev.off, ev.shape, &h);
        m[ev.h] = h;
        if (!rc) live.push_back(h);
      } else if (ev.kind == 2) {
        args = ev.args;
        for (dfs_arg& a : args)
          if (a.privilege != DFS_PRIV_IMM) a.store = m.at(a.store);
        rc = dfs_submit(c, ev.op, ev.ndim, ev.dom, (int32_t)args.size(), args.data());
      } else {
        const dfs_store h = m.at(ev.h);
        rc = dfs_store_release(c, h);
        if (!rc) {
          auto li = std::find(live.begin(), live.end(), h);
          if (li != live.end()) live.erase(li);
        }
      }
      if (rc) {
        // the error message names the failing step; earlier tasks stay issued
        undo();
        return rc;
      }
    }
    return DFS_OK;
  } catch (const std::exception& e_) {
    const int rc = internal_error(c, e_.what());
    undo();
    return rc;
  } catch (...) {
    const int rc = internal_error(c, "unknown exception");
    undo();
    return rc;
  }
}

int dfs_template_free(dfs_ctx* c, uint64_t id) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (!c->templates.erase(id)) return fail(c, DFS_ERR_STATE, "unknown template");
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_set_launch_config(dfs_ctx* c, int32_t block_threads, int32_t unroll, int32_t ctas_per_sm) {
  try {
    if (!c) return DFS_ERR_INVALID;
    if (block_threads != 128 && block_threads != 256 && block_threads != 512 && block_threads != 1024)
      return fail(c, DFS_ERR_INVALID, "block_threads must be 128, 256, 512 or 1024");
    if (unroll < 1 || unroll > 8) return fail(c, DFS_ERR_INVALID, "unroll must be in 1..8");
    if (ctas_per_sm < 0) return fail(c, DFS_ERR_INVALID, "negative ctas_per_sm");
    if (c->batching || c->capturing) return fail(c, DFS_ERR_STATE, "inside a batch or a capture");
    const int rc = flush(c);
    if (rc) return rc;
    c->cfg.block_threads = block_threads;
    c->cfg.unroll = unroll;
    c->cfg.ctas_per_sm = ctas_per_sm;
    c->lastb.ok = false;
    return DFS_OK;
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  }
}

const char* dfs_last_error(dfs_ctx* c) { return c ? c->err.c_str() : "null context"; }

int dfs_plan_json(dfs_ctx* c, char* buf, size_t len, size_t* needed) {
  try {
    if (!c) return DFS_ERR_INVALID;
    WindowInfo wi = window_info(c);
    Plan p = analyse(c->window, wi.roots, c->cfg.fusion != 0, c->cfg.launch_mode);
    std::string s = plan_json(p, c->window, wi);
    s.insert(s.size() - 1, ", \"key\": \"" + std::to_string(std::hash<std::string>{}(wi.key)) + "\"");
    return write_json(s, buf, len, needed);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_stats_json(dfs_ctx* c, char* buf, size_t len, size_t* needed) {
  try {
    if (!c) return DFS_ERR_INVALID;
    std::ostringstream o;
    const Stats& s = c->st;
    o << "{\"tasks\": " << s.tasks << ", \"groups\": " << s.groups << ", \"launches\": " << s.launches
      << ", \"barriers\": " << s.barriers << ", \"flushes\": " << s.flushes << ", \"plan_hits\": " << s.plan_hits
      << ", \"plan_misses\": " << s.plan_misses << ", \"temporaries\": " << s.temporaries
      << ", \"bytes_allocated\": " << s.bytes_allocated << ", \"allocations\": " << s.allocations
      << ", \"analysis_s\": " << s.analysis_s;
    if (c->jit)
      o << ", \"compile_s\": " << c->jit->compile_seconds() << ", \"kernels_compiled\": " << c->jit->compiles()
        << ", \"kernel_cache_hits\": " << c->jit->hits() << ", \"kernel_disk_hits\": " << c->jit->disk_hits();
    o << ", \"last_regs\": " << s.last_regs << ", \"last_occupancy\": " << s.last_occupancy
      << ", \"last_grid\": " << s.last_grid << ", \"last_block\": " << s.last_block;
    o << ", \"kernel_times\": {";
    bool first = true;
    for (const auto& kv : c->ktime) {
      o << (first ? "" : ", ") << "\"" << kv.first << "\": {\"ms\": " << kv.second.first
        << ", \"launches\": " << kv.second.second << "}";
      first = false;
    }
    o << "}";
    o << ", \"batches\": " << c->batches << ", \"batched_instances\": " << c->batched_instances
      << ", \"window_size\": " << c->cfg.window_size << ", \"window_growths\": " << s.window_growths
      << ", \"stores\": " << c->stores.size()
    << ", \"batch_repeats\": " << c->batch_repeats << ", \"batch_fallbacks\": " << c->batch_fallbacks << ", \"batch_fallback_reason\": \"" << c->batch_fallback_reason
      << "\"";
    o << ", \"sms\": " << c->sms << "}";
    return write_json(o.str(), buf, len, needed);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

int dfs_last_kernel_source(dfs_ctx* c, char* buf, size_t len, size_t* needed) {
  try {
    if (!c) return DFS_ERR_INVALID;
    return write_json(c->last_source, buf, len, needed);
  } catch (const std::exception& e_) {
    return internal_error(c, e_.what());
  } catch (...) {
    return internal_error(c, "unknown exception");
  }
}

}  // extern "C"
