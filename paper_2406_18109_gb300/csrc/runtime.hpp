// runtime.hpp -- internal data model of the fusion runtime.
//
// Stores, views, partitions and index tasks follow the paper's IR (Section 3,
// Fig. 2a).  Every analysis works on ROOT stores: a view is a box of its root,
// and an argument's partition is normalised into root coordinates, so that
// "same parent" (Def. 1) is root equality and partition equality is a
// constant-time structural comparison (Section 4.2.1).
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <ostream>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/diffuse.h"

namespace dfs {

constexpr int MAXD = DFS_MAX_DIM;

size_t dtype_size(int dt);
const char* dtype_cname(int dt);  // "float", "double", "int", "long long"
bool dtype_is_float(int dt);

struct StoreRec {
  int64_t handle = 0;
  int dtype = 0;
  int ndim = 0;
  int64_t shape[MAXD] = {0, 0, 0};
  int64_t root = 0;                 // handle of the root store
  int64_t off[MAXD] = {0, 0, 0};    // origin of this store in root coordinates
  bool released = false;            // this handle's application reference dropped
  // ---- root-only state
  void* ptr = nullptr;              // device memory (nullptr until materialised)
  bool owned = false;               // library allocation
  bool wrapped = false;             // caller-owned memory
  bool valid = false;               // holds a value (written, uploaded or wrapped)
  int64_t app_refs = 0;             // live application handles: the root and its views
  int64_t pending = 0;              // buffered tasks referencing the root
  int64_t stride[MAXD] = {0, 0, 0}; // element strides (row-major)
  size_t nbytes = 0;
  int64_t nelem() const;
};

struct PartRec {
  int kind = 0;  // 0 = None, 1 = Tiling
  int ndim = 0;
  int64_t tile[MAXD] = {0, 0, 0};
  int64_t off[MAXD] = {0, 0, 0};
  int32_t proj[MAXD] = {0, 1, 2};
};

// Partition of one task argument in root coordinates.  sub-store of point p
// (Fig. 3e): [proj(p)*tile, (proj(p)+1)*tile) + off, clipped to [vlo, vhi).
struct NPart {
  int kind = 0;  // 0 = None, 1 = Tiling
  int nd = 0;
  int64_t tile[MAXD] = {0, 0, 0};
  int64_t off[MAXD] = {0, 0, 0};
  int32_t proj[MAXD] = {0, 0, 0};
  int64_t vlo[MAXD] = {0, 0, 0};
  int64_t vhi[MAXD] = {0, 0, 0};
  bool operator==(const NPart& o) const;
  bool operator!=(const NPart& o) const { return !(*this == o); }
  std::string key() const;
};

struct Arg {
  bool imm = false;
  double immv = 0.0;
  int64_t store = 0;  // handle as submitted (root or view)
  int64_t root = 0;
  int priv = 0;
  int redop = 0;
  int dtype = 0;
  int nd = 0;         // root ndim
  NPart part;
  bool is_r() const { return priv == DFS_PRIV_R || priv == DFS_PRIV_RW; }
  bool is_w() const { return priv == DFS_PRIV_W || priv == DFS_PRIV_RW; }
  bool is_rd() const { return priv == DFS_PRIV_RD; }
};

struct Task {
  int op = 0;
  int dnd = 0;
  int64_t dom[MAXD] = {1, 1, 1};
  std::vector<Arg> args;
  int64_t seq = 0;
  int64_t npoints() const;
  bool same_domain(const Task& o) const;
  bool scalar() const;  // every store argument is 0-d
};

// Host mirror of the device control block (dfs_device.cuh, struct Ctl).
struct Ctl {
  uint32_t bar_arrive;
  uint32_t exit_arrive;
  int32_t err;
  int32_t err_where;
  uint64_t pad[2];
  uint64_t ticket[16];
};

// ------------------------------------------------------------------ analysis
struct Group {  // one fused task (a fusible prefix, Section 4.2.2)
  int begin = 0, end = 0;
  bool scalar = false;
};

struct Plan {
  std::vector<Group> groups;
  std::set<std::pair<int, int64_t>> temps;  // (group, root): temporary in that group (Def. 4)
  std::vector<std::pair<int, int>> launches;  // [first group, last group + 1)
  std::string key;                          // canonical window key (Section 5.2)
};

struct RootInfo {  // what the analysis needs to know about a root
  int64_t root;
  int ndim;
  int64_t shape[MAXD];
  bool app_live;
  bool wrapped;
  bool valid;
};

// Fusion pass over a window.  `roots` describes every root the window uses.
// launch_mode selects how groups are packed into launches.
Plan analyse(const std::vector<Task>& window, const std::map<int64_t, RootInfo>& roots,
             bool fusion, int launch_mode);

// Longest prefix of window[start..] meeting the four constraints of Fig. 5.
int longest_fusible_prefix(const std::vector<Task>& window, int start);

// Def. 4 for the fused group [b, e) of the window.
bool is_temporary(const std::vector<Task>& window, int b, int e, int64_t root, const RootInfo& ri);

bool covers(const NPart& p, const Task& t, const RootInfo& ri);

std::string iteration_space_key(const Task& t);

std::string canonical_key(const std::vector<Task>& window, const std::map<int64_t, RootInfo>& roots);

// ------------------------------------------------------------------ codegen
struct LaunchRoot {  // one root buffer used by a launch
  int64_t root;
  int dtype;
  int ndim;
  int64_t shape[MAXD];
  int64_t stride[MAXD];
  bool zero_d;
  bool temp;          // eliminated: lives in registers only
  bool written;       // written (W/RW) or reduced by some task of the launch
  bool read;          // read by some task of the launch
  bool valid_before;  // holds a value before the launch
  bool live_out;      // 0-d: value must be written back to memory
  bool aligned16;     // device pointer 16-byte aligned
  int param;          // index of its pointer in the kernel parameters (-1: none)
};

struct LaunchSpec {
  std::vector<Task> tasks;         // tasks of the launch in program order
  std::vector<Group> groups;       // re-based on `tasks`
  std::vector<LaunchRoot> roots;   // indexed through root_index
  std::map<int64_t, int> root_index;
  int block = 256;
  int unroll = 2;
  bool persistent = false;
  int debug_skip = 0;  // test hook: CTA 0 withholds its arrival at this barrier
  int min_blocks = 0;  // > 0: __launch_bounds__ minimum resident CTAs per SM (caps registers)
};

struct KernelCode {
  std::string name;
  std::string source;
  std::string key;      // canonical (store-renamed) key of the generated code
  int nptr = 0;         // pointer params (roots) -- param order: ptrs, imms, partials, ctl
  int nimm = 0;
  int nred = 0;         // reduction slots
  int64_t max_points = 1;
  bool has_flat = false;    // some group sweeps a flat range
  bool has_points = false;  // some group deals points to CTAs (max_points of them)
  int nbarriers = 0;
  std::vector<int64_t> red_points;  // points of each reduction slot
  std::vector<double> imms;         // immediate values in parameter order
  std::vector<std::pair<int, int>> imm_src;  // (task, arg) of each immediate param
  std::vector<int64_t> ptr_roots;   // root handle of each pointer param
  size_t partial_bytes = 0;
  int dyn_smem = 0;                 // dynamic shared memory per CTA (staged SpMV x windows)
};

KernelCode generate(const LaunchSpec& spec);

// Device template of an element-wise op ("op_add", ...), nullptr otherwise.
const char* op_device_fn(int op);

// The element operations of one lane of a fused body, emitted as straight-line
// code.  ERF is odd by definition (op_erf(a) = copysign(erf(|a|), a)), so
// when a body takes erf of a value and of its negation (NEG then ERF or NCDF,
// as in N(d) and N(-d) of the Black-Scholes chain) erf(|.|) is evaluated
// once and both results keep the exact bits each task computes alone.  One
// instance per lane: names are the lane's value expressions.
//
// Invariant: every expression handed to emit (an operand or a result) names
// an immutable per-lane value -- a `const` load, an immediate, a 0-d register
// that no task of the loop nest writes, or an earlier result `v<task>_...`.
// A store rewritten inside the window gets a new result name, so sharing
// keyed by these strings can never reuse a stale value.  emit refuses (throws)
// a result name it has already defined.
class LaneOps {
 public:
  // Emits `const T res = op(in...)` (possibly in several statements).
  void emit(std::ostream& o, const std::string& pad, const std::string& T, int op, const std::string& res,
            const std::vector<std::string>& in);
  // For callers that evaluate ERF or NCDF on two lanes at once: the name of
  // an erf magnitude this lane already has for argument in0 (or for its
  // negation), empty if none; and the record of the one the caller computed.
  std::string mag_of(int op, const std::string& in0) const;
  void set_mag(int op, const std::string& in0, const std::string& m);
  // Registers `res` as defined by the caller (an operation it emitted itself).
  void define(const std::string& res);

 private:
  std::string shared(const std::map<std::string, std::string>& m, const std::string& a) const;
  std::map<std::string, std::string> neg_;   // value -> a value equal to its negation
  std::map<std::string, std::string> mag_;   // ERF argument -> erf(|argument|)
  std::map<std::string, std::string> nmag_;  // NCDF argument x -> erf(|x / sqrt 2|)
  std::set<std::string> defined_;            // result names emitted so far
};

// ------------------------------------------------------ batched execution
// One size-generic kernel for K isomorphic instances of a window.  Sizes,
// pointers and immediates come from per-instance descriptors:
//   struct Inst { void* p[nptr]; double imm[nimm]; i64 v[nv]; }
// and every vector group walks a work list (prefix offsets of the instances'
// point counts).  Stores are 0-d or 1-D.
struct BatchCode {
  std::string name, source;
  int nptr = 0, nimm = 0, nv = 0, nsval = 0, nprefix = 0, nred = 0, nbarriers = 0;
  int vec = 1;
  std::vector<int64_t> ptr_roots;              // instance-0 root of each pointer slot
  std::vector<std::pair<int, int>> imm_src;    // (task, arg) of each immediate slot
  struct VSrc {
    int task, arg, field;                      // field: 0 tile, 1 off, 2 vlo, 3 vhi, 4 SpMV lanes per row
  };
  std::vector<VSrc> v_src;
  std::vector<int> prefix_task;                // first task of the group each prefix array serves
  int dyn_smem = 0;                            // dynamic shared memory per CTA (staged SpMV x windows)
};

// Lanes per row of the warp-cooperative SpMV (spmv_warp) for a CSR matrix
// of nnz entries over nrows rows: the largest power of two K <= 32 with
// 16 K <= nnz / nrows, so rows share lanes only from 32 entries on (measured
// on GB300: 7-entry rows ran 30 % slower on two lanes than on one, 16-entry
// random rows 7 % faster on four); 1 (one row per lane) below.  A property of
// the matrix alone, so every path that multiplies by it sums its rows in one
// order.
inline int spmv_lanes(int64_t nnz, int64_t nrows) {
  const int64_t avg = nrows > 0 ? nnz / nrows : 0;
  int k = 1;
  while (k < 32 && 16 * (2 * k) <= avg) k *= 2;
  return k;
}

// Returns false (with a reason) when the launch cannot be batched.
// coop: some instance's SpMV shares rows between lanes (spmv_lanes > 1);
// without it SpMV nests keep one row per lane and the unrolled loops.
bool generate_batch(const LaunchSpec& spec, int vec, bool coop, BatchCode& out, std::string& why);

}  // namespace dfs
