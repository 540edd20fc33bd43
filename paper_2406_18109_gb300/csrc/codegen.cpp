// codegen.cpp -- CUDA source for one launch group.
//
// The fused task body is the composition of the task bodies in program order
// (Section 4.2.2); loops of consecutive tasks with the same iteration space
// are fused and their temporaries become registers (Section 6.3, Fig. 8:
// compose, eliminate temporaries, fuse and parallelise loops, remove local
// allocations).  On the GPU:
//   * the launch domain is the set of work units (points); CTAs take points
//     in grid-stride order, so a fused group needs no communication between
//     CTAs (the fusion constraints guarantee point-wise dependencies);
//   * a launch holding several fused groups (persistent mode) separates them
//     by grid barriers wherever the previous group was not a replicated
//     scalar group; scalar groups (all stores 0-d) run redundantly in every
//     CTA on register copies of the 0-d values (after a barrier, on warp 0
//     with a shared-memory broadcast to the rest of the CTA);
//   * reductions keep one partial per point, finished in a fixed order after
//     the next barrier (or by the last CTA to exit), so every result is
//     reproducible and identical between fused and unfused execution.
// Every shape, tile and offset is a compile-time constant of the generated
// source; pointers and immediate values are kernel parameters, so isomorphic
// windows share one compiled kernel (Section 5.2).
#include <algorithm>
#include <cstdio>
#include <functional>
#include <sstream>
#include <stdexcept>

#include "runtime.hpp"

namespace dfs {

size_t dtype_size(int dt) {
  switch (dt) {
    case DFS_F32: return 4;
    case DFS_F64: return 8;
    case DFS_I32: return 4;
    case DFS_I64: return 8;
  }
  return 0;
}
const char* dtype_cname(int dt) {
  switch (dt) {
    case DFS_F32: return "float";
    case DFS_F64: return "double";
    case DFS_I32: return "int";
    case DFS_I64: return "long long";
  }
  return "void";
}
bool dtype_is_float(int dt) { return dt == DFS_F32 || dt == DFS_F64; }

namespace {

const char* op_fn(int op) {
  switch (op) {
    case DFS_OP_COPY: return "op_copy";
    case DFS_OP_NEG: return "op_neg";
    case DFS_OP_ABS: return "op_abs";
    case DFS_OP_EXP: return "op_exp";
    case DFS_OP_LOG: return "op_log";
    case DFS_OP_SQRT: return "op_sqrt";
    case DFS_OP_ERF: return "op_erf";
    case DFS_OP_NCDF: return "op_ncdf";
    case DFS_OP_ADD: return "op_add";
    case DFS_OP_SUB: return "op_sub";
    case DFS_OP_MUL: return "op_mul";
    case DFS_OP_DIV: return "op_div";
    case DFS_OP_POW: return "op_pow";
    case DFS_OP_MAX: return "op_max";
    case DFS_OP_MIN: return "op_min";
  }
  return nullptr;
}

bool is_elementwise(int op) { return op_fn(op) != nullptr; }
bool is_reduction(int op) { return op == DFS_OP_DOT || op == DFS_OP_SUM; }

// The argument whose sub-store drives the task's loop.
const Arg& space_arg(const Task& t) {
  if (is_reduction(t.op)) return t.args[0];
  if (t.op == DFS_OP_SPMV) return t.args[4];
  return t.args.back();
}

std::string akey(const Arg& a) { return std::to_string(a.root) + "@" + a.part.key(); }

struct Nest {
  int first, last;  // task indices [first, last)
  int dims;         // 1 (flat) or 2 (row loop)
  int vec;          // elements per vector access
  int rank = 1;     // rank of the iteration space (rows of a 3-D space are (plane, row) pairs)
  bool coop = false;  // an SpMV of the nest uses several lanes per row (spmv_warp)
  // realigned rows: vectors in the frame of the written views (`head` scalar
  // columns first); a read view whose column origin is `shift` elements past
  // that frame is loaded as two aligned vectors
  bool realign = false;
  int head = 0;
  std::map<std::string, int> shift;
};

// Lanes per row of an SpMV task's matrix (col and rowptr extents).
int spmv_k(const Task& t) {
  const NPart& c = t.args[1].part;
  const NPart& r = t.args[0].part;
  return spmv_lanes(c.vhi[0] - c.vlo[0], r.vhi[0] - r.vlo[0] - 1);
}

class Gen {
 public:
  explicit Gen(const LaunchSpec& s) : S(s) {}

  KernelCode run();

 private:
  const LaunchSpec& S;
  std::ostringstream o;
  KernelCode kc;
  std::map<int64_t, int> ptr_of;          // root -> pointer param index
  std::map<int64_t, std::string> sreg;    // 0-d root -> register name
  std::map<int64_t, bool> have;           // 0-d root holds a value in registers
  struct Red { int slot; int64_t root; int dtype; int64_t points; };
  std::vector<Red> pending_red;           // reductions awaiting finalisation
  int nbar = 0;
  int nbc = 0;  // shared broadcast slots of finished reductions
  bool stage = false;  // some per-point SpMV nest stages x windows in shared memory

  const LaunchRoot& R(int64_t root) const { return S.roots[S.root_index.at(root)]; }
  bool temp_in(int g, int64_t root) const;
  std::string ptr(int64_t root) const { return "r" + std::to_string(ptr_of.at(root)); }
  std::string T(int dt) const { return dtype_cname(dt); }

  void emit_params();
  void emit_prologue();
  void emit_group(int g);
  void emit_scalar_group(int g);
  void emit_vector_group(int g);
  void emit_nest(int g, const Nest& n, const std::string& red_pt, bool flat);
  // Which tasks of nest n run two lanes per instruction in a body of w lanes
  // (index: task - n.first).
  std::vector<char> packed_tasks(const Nest& n, int w) const;
  void emit_finalise(const char* indent);
  int emit_warp0_scalars(int g);
  void realign(Nest& n, int vec);
  std::vector<Nest> nests_of(int g);
  std::string imm_expr(int task, int arg, int dt);
};

bool Gen::temp_in(int g, int64_t root) const {
  (void)g;
  const LaunchRoot& r = R(root);
  return r.temp;
}

std::string Gen::imm_expr(int task, int arg, int dt) {
  const int k = kc.nimm++;
  kc.imms.push_back(S.tasks[task].args[arg].immv);
  kc.imm_src.push_back({task, arg});
  return "((" + T(dt) + ")P.imm[" + std::to_string(k) + "])";
}

void Gen::emit_params() {
  // pointer params: every root with memory
  for (const LaunchRoot& r : S.roots) {
    if (r.param < 0) continue;
    ptr_of[r.root] = r.param;
  }
  kc.nptr = 0;
  for (const LaunchRoot& r : S.roots)
    if (r.param >= 0) kc.nptr = std::max(kc.nptr, r.param + 1);
  kc.ptr_roots.assign(kc.nptr, 0);
  for (const LaunchRoot& r : S.roots)
    if (r.param >= 0) kc.ptr_roots[r.param] = r.root;
}

void Gen::emit_prologue() {
  // typed root pointers
  for (const LaunchRoot& r : S.roots) {
    if (r.param < 0) continue;
    o << "  " << T(r.dtype) << "* __restrict__ " << ptr(r.root) << " = (" << T(r.dtype) << "*)P.p["
      << r.param << "];\n";
  }
  // 0-d registers
  int k = 0;
  for (const LaunchRoot& r : S.roots) {
    if (!r.zero_d) continue;
    const std::string nm = "s" + std::to_string(k++);
    sreg[r.root] = nm;
    const bool load = r.valid_before && r.param >= 0;
    o << "  " << T(r.dtype) << " " << nm << " = " << (load ? "ld(" + ptr(r.root) + ")" : T(r.dtype) + "(0)")
      << ";\n";
    have[r.root] = load;
  }
}

// Row nests whose views start at different column offsets (the shifted
// views of a stencil) still use vector accesses when every root row is a
// whole number of aligned vectors and no reduction's summation order would
// change: the nest iterates in the vector frame of its written views.
void Gen::realign(Nest& n, int vec) {
  int mw = -1, mr = -1;
  size_t esz = 0;
  std::map<std::string, int> phase;
  for (int t = n.first; t < n.last; ++t) {
    const Task& tk = S.tasks[t];
    if (tk.scalar()) continue;
    if (is_reduction(tk.op) || tk.op == DFS_OP_SPMV) return;
    for (size_t ai = 0; ai < tk.args.size(); ++ai) {
      const Arg& a = tk.args[ai];
      if (a.imm || a.nd == 0) continue;
      const LaunchRoot& r = R(a.root);
      if (r.temp) continue;  // lives in registers
      if (esz && esz != dtype_size(a.dtype)) return;
      esz = dtype_size(a.dtype);
      const int cd = a.nd - 1;
      if (!r.aligned16 || a.part.kind != 1 || tk.dom[a.part.proj[cd]] != 1) return;
      for (int d = 0; d < cd; ++d)
        if (r.stride[d] % vec) return;
      const int64_t c0 = std::max(a.part.off[cd], a.part.vlo[cd]);
      const int ph = (int)(((c0 % vec) + vec) % vec);
      phase[akey(a)] = ph;
      const bool out = is_elementwise(tk.op) && ai + 1 == tk.args.size();
      if (out) {
        if (mw >= 0 && mw != ph) return;
        mw = ph;
      } else if (mr < 0) {
        mr = ph;
      }
    }
  }
  if (!esz || (int)(16 / esz) != vec) return;
  n.realign = true;
  n.vec = vec;
  n.head = (vec - (mw >= 0 ? mw : std::max(mr, 0))) % vec;
  for (const auto& kv : phase) n.shift[kv.first] = (kv.second + n.head) % vec;
}

std::vector<Nest> Gen::nests_of(int g) {
  const Group& G = S.groups[g];
  std::vector<Nest> v;
  int i = G.begin;
  while (i < G.end && S.tasks[i].scalar()) ++i;  // scalar tasks are hoisted
  while (i < G.end) {
    const std::string key = iteration_space_key(S.tasks[i]);
    int j = i + 1;
    while (j < G.end && (S.tasks[j].scalar() || iteration_space_key(S.tasks[j]) == key)) ++j;
    Nest n;
    n.first = i;
    n.last = j;
    // dimensionality and vector width
    const Arg& sa = space_arg(S.tasks[i]);
    const int nd = sa.nd;
    // collapse a 2-D or 3-D space into a flat one when every access spans
    // whole root rows (and planes): its elements are then contiguous
    bool flat = nd <= 1;
    if (nd >= 2) {
      flat = true;
      for (int t = i; t < j && flat; ++t)
        for (const Arg& a : S.tasks[t].args) {
          if (a.imm || a.nd == 0) continue;
          if (S.tasks[t].op == DFS_OP_SPMV && &a != &S.tasks[t].args[4]) continue;
          const LaunchRoot& r = R(a.root);
          if (a.part.kind != 1) flat = false;
          for (int d = 1; d < nd && flat; ++d)
            if (a.part.vlo[d] != 0 || a.part.vhi[d] != r.shape[d] || a.part.off[d] > 0 ||
                a.part.tile[d] < r.shape[d] || r.stride[d - 1] != r.shape[d] * r.stride[d])  // no row padding
              flat = false;
        }
    }
    if (nd > 3) throw std::runtime_error("iteration spaces of rank > 3 are not supported");
    // rows mode: ext0 rows (2-D) or ext0 x ext1 rows (3-D) of the last dimension
    n.dims = flat ? 1 : 2;
    n.rank = nd;
    // widest element over the memory accesses of the nest
    size_t esz = 0;
    bool aligned = true;
    for (int t = i; t < j; ++t) {
      const Task& tk = S.tasks[t];
      for (size_t ai = 0; ai < tk.args.size(); ++ai) {
        const Arg& a = tk.args[ai];
        if (a.imm || a.nd == 0) continue;
        if (tk.op == DFS_OP_SPMV && ai != 4) continue;  // gathered, not streamed
        esz = std::max(esz, dtype_size(a.dtype));
      }
    }
    int vec = esz ? (int)(16 / esz) : 1;
    for (int t = i; t < j && vec > 1; ++t) {
      const Task& tk = S.tasks[t];
      for (size_t ai = 0; ai < tk.args.size(); ++ai) {
        const Arg& a = tk.args[ai];
        if (a.imm || a.nd == 0) continue;
        if (tk.op == DFS_OP_SPMV && ai != 4) continue;
        const LaunchRoot& r = R(a.root);
        if ((int)(16 / dtype_size(a.dtype)) != vec) aligned = false;
        if (!r.temp && !r.aligned16) aligned = false;
        if (n.dims == 1) {
          for (int d = 0; d < a.nd; ++d) {
            const int64_t st = r.stride[d];
            if ((a.part.tile[d] * st) % vec || (a.part.off[d] * st) % vec || (a.part.vlo[d] * st) % vec)
              aligned = false;
          }
        } else {
          const int cd = a.nd - 1;  // the column dimension
          for (int d = 0; d < cd; ++d)
            if (r.stride[d] % vec) aligned = false;
          if (a.part.tile[cd] % vec || a.part.off[cd] % vec || a.part.vlo[cd] % vec ||
              (a.part.vhi[cd] - a.part.vlo[cd]) % vec)
            aligned = false;
        }
      }
    }
    n.vec = aligned ? vec : 1;
    if (!aligned && vec > 1 && n.dims == 2) realign(n, vec);
    for (int t = i; t < j; ++t)
      if (S.tasks[t].op == DFS_OP_SPMV && spmv_k(S.tasks[t]) > 1) n.coop = true;
    v.push_back(n);
    i = j;
    while (i < G.end && S.tasks[i].scalar()) ++i;
  }
  return v;
}

void Gen::emit_group(int g) {
  if (S.groups[g].scalar)
    emit_scalar_group(g);
  else
    emit_vector_group(g);
}

// A group of scalar tasks, evaluated on the register copies of the 0-d
// stores: by every thread at the start of a launch, by warp 0 after a grid
// barrier (emit_warp0_scalars).
void Gen::emit_scalar_group(int g) {
  const Group& G = S.groups[g];
  o << "    { // group " << g << " (scalar)\n";
  for (int i = G.begin; i < G.end; ++i) {
    const Task& t = S.tasks[i];
    const Arg& out = t.args.back();
    const int dt = out.dtype;
    std::vector<std::string> ins;
    for (size_t k = 0; k + 1 < t.args.size(); ++k) {
      const Arg& a = t.args[k];
      if (a.imm) ins.push_back(imm_expr(i, (int)k, dt));
      else ins.push_back("(" + T(dt) + ")" + sreg.at(a.root));
    }
    o << "      " << sreg.at(out.root) << " = " << op_fn(t.op) << "(";
    for (size_t k = 0; k < ins.size(); ++k) o << (k ? ", " : "") << ins[k];
    o << ");\n";
    have[out.root] = true;
  }
  o << "    }\n";
}

void Gen::emit_vector_group(int g) {
  const Group& G = S.groups[g];
  const Task& t0 = S.tasks[G.begin];
  const int64_t npts = t0.npoints();
  // Scalar tasks can share a group with vector tasks when the launch domain
  // has a single point.  They read and write 0-d values only, so every CTA
  // evaluates them first, in program order (the one point may run anywhere);
  // this is exact unless a vector task earlier in the group reads a value a
  // later scalar task overwrites.
  for (int i = G.begin; i < G.end; ++i) {
    if (!S.tasks[i].scalar()) continue;
    const int64_t out = S.tasks[i].args.back().root;
    for (int j = G.begin; j < i; ++j)
      if (!S.tasks[j].scalar())
        for (const Arg& a : S.tasks[j].args)
          if (!a.imm && a.root == out)
            throw std::runtime_error("a scalar task overwrites a value read earlier in its group");
    const Task& t = S.tasks[i];
    const int dt = t.args.back().dtype;
    std::vector<std::string> ins;
    for (size_t k = 0; k + 1 < t.args.size(); ++k) {
      const Arg& a = t.args[k];
      ins.push_back(a.imm ? imm_expr(i, (int)k, dt) : "(" + T(dt) + ")" + sreg.at(a.root));
    }
    o << "    " << sreg.at(t.args.back().root) << " = " << op_fn(t.op) << "(";
    for (size_t k = 0; k < ins.size(); ++k) o << (k ? ", " : "") << ins[k];
    o << ");\n";
    have[t.args.back().root] = true;
  }
  std::vector<Nest> nests = nests_of(g);
  // A group with one loop nest and no reduction needs no per-point
  // structure: the union of the points' sub-stores is one rectangle of
  // contiguous tiles (every operand has the same tile shape and offsets
  // relative to its view), so it is swept as one range with a grid stride,
  // which balances the work across CTAs at element granularity.
  bool flat = nests.size() == 1;
  for (int i = G.begin; i < G.end && flat; ++i)
    if (is_reduction(S.tasks[i].op)) flat = false;
  if (flat && space_arg(t0).nd > 3) flat = false;
  if (flat) {
    kc.has_flat = true;
    o << "    { // group " << g << ": tasks " << G.begin << ".." << G.end - 1 << ", one flat nest over "
      << npts << " points\n";
    emit_nest(g, nests[0], "", true);
    o << "    }\n";
    return;
  }
  kc.has_points = true;
  kc.max_points = std::max(kc.max_points, npts);
  o << "    { // group " << g << ": tasks " << G.begin << ".." << G.end - 1 << ", " << nests.size()
    << " loop nest(s), " << npts << " points\n";
  o << "      for (i64 pt = blockIdx.x; pt < " << npts << "LL; pt += gridDim.x) {\n";
  // point coordinates
  {
    int64_t rem = 1;
    for (int d = t0.dnd - 1; d >= 0; --d) {
      o << "        const i64 q" << d << " = (pt / " << rem << "LL) % " << t0.dom[d] << "LL;\n";
      rem *= t0.dom[d];
    }
  }
  for (size_t k = 0; k < nests.size(); ++k) {
    if (k) o << "        __syncthreads();\n";
    emit_nest(g, nests[k], "pt", false);
  }
  o << "      }\n";
  o << "    }\n";
}

// FP32 element-wise ADD, NCDF, ERF and LOG tasks run two lanes per
// instruction (pk_add, pk_ncdf_*, erf_mag2, log_f32x2) when that cannot change
// a bit.  The compiler contracts a packed product whose value reaches a sum
// into a fused multiply-add, so an NCDF (whose last step multiplies) whose
// value, possibly negated or copied on the way, reaches a sum of the body
// (ADD, SUB, a SUM reduction) keeps both operations scalar, and so does a sum
// of a MUL.  ERF and LOG are neither products nor sums (inside, their products
// reach sums only through explicit fused multiply-adds), so they always pair
// up.  MUL itself stays on single lanes: a packed multiply saves an issue slot
// but waits on the packed pipe, and measured on the fused Black-Scholes
// window, multiplies on lane pairs made the kernel 0.9 % slower.  Values
// loaded from memory or computed outside the body are not products of the
// body.
std::vector<char> Gen::packed_tasks(const Nest& n, int w) const {
  std::vector<char> pk(n.last - n.first, 0);
  if (w < 2 || w % 2) return pk;
  std::map<std::string, int> product_of;  // akey -> task whose product the value is
  std::vector<char> blocked(n.last - n.first, 0);
  for (int i = n.first; i < n.last; ++i) {
    const Task& t = S.tasks[i];
    if (t.scalar()) continue;
    const bool sum = t.op == DFS_OP_ADD || t.op == DFS_OP_SUB || t.op == DFS_OP_SUM;
    const size_t nin = t.op == DFS_OP_SPMV ? 0 : t.args.size() - 1;
    int carried = -1;  // a product passed on by NEG or COPY
    for (size_t ai = 0; ai < nin; ++ai) {
      const Arg& a = t.args[ai];
      if (a.imm || a.nd == 0) continue;
      auto it = product_of.find(akey(a));
      if (it == product_of.end()) continue;
      if (sum) {
        blocked[it->second - n.first] = 1;
        blocked[i - n.first] = 1;
      }
      if (t.op == DFS_OP_NEG || t.op == DFS_OP_COPY) carried = it->second;
    }
    if (!is_elementwise(t.op)) continue;
    const std::string out = akey(t.args.back());
    product_of.erase(out);
    if (t.op == DFS_OP_MUL || t.op == DFS_OP_NCDF) product_of[out] = i;
    else if (carried >= 0) product_of[out] = carried;
  }
  for (int i = n.first; i < n.last; ++i) {
    const Task& t = S.tasks[i];
    if (t.scalar() || blocked[i - n.first] || space_arg(t).dtype != DFS_F32) continue;
    pk[i - n.first] = t.op == DFS_OP_ADD || t.op == DFS_OP_NCDF || t.op == DFS_OP_ERF || t.op == DFS_OP_LOG;
  }
  return pk;
}

void Gen::emit_nest(int g, const Nest& n, const std::string& ptvar, bool flat) {
  const int BD = S.block;
  const int U = std::max(1, S.unroll);
  const int V = n.vec;
  const Task& first = S.tasks[n.first];
  const Arg& sa = space_arg(first);
  const int nd = sa.nd;
  const std::string ind = "        ";
  o << ind << "{ // nest: tasks " << n.first << ".." << n.last - 1 << ", vec " << V << ", "
    << (n.dims == 1 ? "flat" : "rows") << "\n";
  // ---- per-access base offsets (root coordinates flattened)
  std::map<std::string, std::string> base;  // akey -> base variable
  int nb = 0;
  auto box_lo = [&](const Arg& a, int d) {
    std::ostringstream s;
    if (a.part.kind == 0) {
      s << a.part.vlo[d] << "LL";
    } else if (flat) {
      s << std::max(a.part.off[d], a.part.vlo[d]) << "LL";
    } else {
      s << "max(q" << a.part.proj[d] << " * " << a.part.tile[d] << "LL + (" << a.part.off[d] << "LL), "
        << a.part.vlo[d] << "LL)";
    }
    return s.str();
  };
  auto need_base = [&](const Arg& a) {
    const std::string k = akey(a);
    if (base.count(k)) return base[k];
    const std::string nm = "b" + std::to_string(nb++);
    const LaunchRoot& r = R(a.root);
    o << ind << "  const i64 " << nm << " = ";
    for (int d = 0; d < a.nd; ++d) o << (d ? " + " : "") << "(" << box_lo(a, d) << ") * " << r.stride[d] << "LL";
    if (a.nd == 0) o << "0";
    o << ";\n";
    base[k] = nm;
    return nm;
  };
  // ---- extents of the iteration space
  int64_t flat_cells = 1;  // elements of a flat range (constant)
  for (int d = 0; d < nd; ++d) {
    if (sa.part.kind == 0) {
      flat_cells *= std::max<int64_t>(0, sa.part.vhi[d] - sa.part.vlo[d]);
      o << ind << "  const i64 ext" << d << " = " << (sa.part.vhi[d] - sa.part.vlo[d]) << "LL;\n";
    } else if (flat) {
      const int64_t cnt = first.dom[sa.part.proj[d]];
      const int64_t lo = std::max(sa.part.off[d], sa.part.vlo[d]);
      const int64_t hi = std::min(cnt * sa.part.tile[d] + sa.part.off[d], sa.part.vhi[d]);
      flat_cells *= std::max<int64_t>(0, hi - lo);
      o << ind << "  const i64 ext" << d << " = " << std::max<int64_t>(0, hi - lo) << "LL;\n";
    } else {
      o << ind << "  const i64 ext" << d << " = min(q" << sa.part.proj[d] << " * " << sa.part.tile[d]
        << "LL + (" << sa.part.off[d] << "LL) + " << sa.part.tile[d] << "LL, " << sa.part.vhi[d]
        << "LL) - max(q" << sa.part.proj[d] << " * " << sa.part.tile[d] << "LL + (" << sa.part.off[d]
        << "LL), " << sa.part.vlo[d] << "LL);\n";
    }
  }
  // ---- classify accesses
  // reads from memory: distinct (root, partition) read before any in-nest write of it
  struct Rd { std::string key; const Arg* a; std::string var; bool ro; };
  std::vector<Rd> reads;
  std::map<std::string, int> read_idx;
  std::set<std::string> written_keys;
  // reduction accumulators
  struct Acc { int task; int slot; std::string var; int dt; };
  std::vector<Acc> accs;
  for (int i = n.first; i < n.last; ++i) {
    const Task& t = S.tasks[i];
    if (t.scalar()) continue;
    for (size_t ai = 0; ai < t.args.size(); ++ai) {
      const Arg& a = t.args[ai];
      if (a.imm || a.nd == 0) continue;
      if (t.op == DFS_OP_SPMV && ai != 4) continue;
      const std::string k = akey(a);
      if (a.is_r() && !(t.op != DFS_OP_SPMV && is_elementwise(t.op) && ai + 1 == t.args.size())) {
        if (!written_keys.count(k) && !read_idx.count(k)) {
          read_idx[k] = (int)reads.size();
          const LaunchRoot& r = R(a.root);
          reads.push_back({k, &a, "m" + std::to_string(reads.size()), !r.written});
          need_base(a);
        }
      }
      const bool is_out = (is_elementwise(t.op) && ai + 1 == t.args.size()) || (t.op == DFS_OP_SPMV && ai == 4);
      if (is_out) {
        written_keys.insert(k);
        // an SpMV output's offset also gives its row index, temporary or not
        if (!R(a.root).temp || t.op == DFS_OP_SPMV) need_base(a);
      }
    }
    if (is_reduction(t.op)) {
      const Arg& out = t.args.back();
      Acc ac;
      ac.task = i;
      ac.slot = kc.nred++;
      ac.var = "acc" + std::to_string(ac.slot);
      ac.dt = out.dtype;
      accs.push_back(ac);
      kc.red_points.push_back(t.npoints());
      pending_red.push_back({ac.slot, out.root, out.dtype, t.npoints()});
      o << ind << "  " << T(ac.dt) << " " << ac.var << " = " << T(ac.dt) << "(0);\n";
    }
  }
  // SpMV gathered operands: bases of rowptr/col/val/x (None partitions)
  for (int i = n.first; i < n.last; ++i) {
    const Task& t = S.tasks[i];
    if (t.scalar()) continue;
    if (t.op != DFS_OP_SPMV) continue;
    for (int ai = 0; ai < 4; ++ai) need_base(t.args[ai]);
  }
  // the first SpMV of a per-point nest that carries x windows: stage them for
  // this point (every thread of the CTA is here, at the same point)
  int staged = -1;
  if (stage && !flat && n.dims == 1 && !n.coop)
    for (int i = n.first; i < n.last && staged < 0; ++i)
      if (S.tasks[i].op == DFS_OP_SPMV && S.tasks[i].args.size() == 6) staged = i;
  if (staged >= 0) {
    const Task& t = S.tasks[staged];
    const Arg& x = t.args[3];
    const std::string tn = T(x.dtype);
    const std::string wb = need_base(t.args[5]);
    o << ind << "  const XWin xw_ = xstage<" << tn << ">((" << tn << "*)dfs_xs_raw, "
      << DFS_SPMV_STAGE_BYTES / (int)dtype_size(x.dtype) << ", " << ptr(x.root) << " + " << base.at(akey(x)) << ", "
      << (x.part.vhi[0] - x.part.vlo[0]) << "LL, (const int*)" << ptr(t.args[5].root) << " + " << wb
      << ", &xs_mbar_, xs_ph_, xs_live_, ctl, P.timeout_ns);\n";
  }
  // immediates hoisted once per nest
  std::map<std::pair<int, int>, std::string> immv;
  for (int i = n.first; i < n.last; ++i) {
    const Task& t = S.tasks[i];
    if (t.scalar()) continue;
    const int dt = t.args.back().dtype;
    for (size_t ai = 0; ai < t.args.size(); ++ai) {
      const Arg& a = t.args[ai];
      if (!a.imm) continue;
      const std::string nm = "k" + std::to_string(i) + "_" + std::to_string(ai);
      o << ind << "  const " << T(dt) << " " << nm << " = " << imm_expr(i, (int)ai, dt) << ";\n";
      immv[{i, (int)ai}] = nm;
    }
  }

  std::map<int, std::string> spre;  // SpMV task -> value computed before the body (warp-cooperative rows)
  // ---- body generator for one element group: `u` unroll slot, lanes V,
  // element offset expression `eoff` (flat) or (row, col) expressions
  auto addr = [&](const Arg& a, const std::string& e_flat, const std::string& row, const std::string& col) {
    const LaunchRoot& r = R(a.root);
    if (n.dims == 1) return ptr(a.root) + " + " + base.at(akey(a)) + " + " + e_flat;
    if (n.rank == 3)
      return ptr(a.root) + " + " + base.at(akey(a)) + " + ((" + row + ") / ext1) * " + std::to_string(r.stride[0]) +
             "LL + ((" + row + ") % ext1) * " + std::to_string(r.stride[1]) + "LL + " + col;
    return ptr(a.root) + " + " + base.at(akey(a)) + " + (" + row + ") * " + std::to_string(r.stride[0]) + "LL + " + col;
  };
  // emits loads for slot u (vector width w), compute, stores; returns nothing
  auto body = [&](int w, const std::vector<std::string>& slots, const std::vector<std::string>& eflat,
                  const std::vector<std::string>& erow, const std::vector<std::string>& ecol,
                  const std::string& pad) {
    const int ns = (int)slots.size();
    // loads
    for (int s = 0; s < ns; ++s) {
      for (const Rd& rd : reads) {
        const Arg& a = *rd.a;
        const std::string ad = addr(a, eflat[s], erow[s], ecol[s]);
        const std::string v = rd.var + "_" + slots[s];
        const int sh = (w > 1 && n.realign) ? n.shift.at(rd.key) : 0;
        if (sh && w == 4 && a.dtype == DFS_F32) {
          o << pad << "const f32x4 " << v << " = " << (rd.ro ? "ld4sro<" : "ld4s<") << sh << ">(" << ad << " - " << sh
            << ");\n";
        } else if (sh && w == 2 && a.dtype == DFS_F64) {
          o << pad << "const f64x2 " << v << " = " << (rd.ro ? "ld2sro<" : "ld2s<") << sh << ">(" << ad << " - " << sh
            << ");\n";
        } else if (w == 4 && a.dtype == DFS_F32) {
          o << pad << "const f32x4 " << v << " = " << (rd.ro ? "ld4ro(" : "ld4(") << ad << ");\n";
        } else if (w == 2 && a.dtype == DFS_F64) {
          o << pad << "const f64x2 " << v << " = " << (rd.ro ? "ld2ro(" : "ld2(") << ad << ");\n";
        } else {
          o << pad << "const " << T(a.dtype) << " " << v << " = " << (rd.ro ? "ldro(" : "ld(") << ad << ");\n";
        }
      }
    }
    // compute: per slot, tasks in program order, each over the lanes
    const std::vector<char> pk = packed_tasks(n, w);
    std::map<std::string, std::vector<std::string>> outvars;  // akey -> per (slot*w+lane) value
    for (int s = 0; s < ns; ++s) {
      std::vector<std::map<std::string, std::string>> curs(w);  // per lane: akey -> value expr
      std::vector<LaneOps> lanes(w);
      for (int l = 0; l < w; ++l)
        for (const Rd& rd : reads) {
          const std::string v = rd.var + "_" + slots[s];
          curs[l][rd.key] = (w > 1) ? v + ".v[" + std::to_string(l) + "]" : v;
        }
      for (int i = n.first; i < n.last; ++i) {
        const Task& t = S.tasks[i];
        if (t.scalar()) continue;
        const int dt = space_arg(t).dtype;   // the output's (y for an SpMV, whose last arg may be its windows)
        auto res_of = [&](int l) { return "v" + std::to_string(i) + "_" + slots[s] + "_" + std::to_string(l); };
        auto val_of = [&](int l, size_t ai) -> std::string {
          const Arg& a = t.args[ai];
          if (a.imm) return immv.at({i, (int)ai});
          if (a.nd == 0) return "(" + T(dt) + ")" + sreg.at(a.root);
          return curs[l].at(akey(a));
        };
        if (pk[i - n.first]) {
          // two lanes per instruction
          for (int l = 0; l < w; l += 2) {
            const std::string r0 = res_of(l), r1 = res_of(l + 1), pr = r0 + "_p";
            if (t.op == DFS_OP_NCDF || t.op == DFS_OP_ERF) {
              lanes[l].define(r0);
              lanes[l + 1].define(r1);
              const std::string a0 = val_of(l, 0), a1 = val_of(l + 1, 0);
              // the argument of erf: x / sqrt 2 for NCDF, x itself for ERF
              std::string y0 = a0, y1 = a1;
              if (t.op == DFS_OP_NCDF) {
                const std::string y = r0 + "_y2";
                o << pad << "const float2 " << y << " = pk_ncdf_arg(" << a0 << ", " << a1 << ");\n";
                y0 = y + ".x";
                y1 = y + ".y";
              }
              // erf(|y|) of both lanes in one packed evaluation, unless the
              // lanes reuse the magnitude of a negation (both do, or neither)
              std::string m0 = lanes[l].mag_of(t.op, a0), m1 = lanes[l + 1].mag_of(t.op, a1);
              if (m0.empty() && m1.empty()) {
                o << pad << "const float2 " << r0 << "_m2 = erf_mag2(" << y0 << ", " << y1 << ");\n";
                m0 = r0 + "_m2.x";
                m1 = r0 + "_m2.y";
              } else {
                if (m0.empty()) {
                  m0 = r0 + "_m";
                  o << pad << "const float " << m0 << " = erf_mag(" << y0 << ");\n";
                }
                if (m1.empty()) {
                  m1 = r1 + "_m";
                  o << pad << "const float " << m1 << " = erf_mag(" << y1 << ");\n";
                }
              }
              lanes[l].set_mag(t.op, a0, m0);
              lanes[l + 1].set_mag(t.op, a1, m1);
              if (t.op == DFS_OP_NCDF)
                o << pad << "const float2 " << pr << " = pk_ncdf_of_erf(erf_sign(" << m0 << ", " << y0 << "), erf_sign("
                  << m1 << ", " << y1 << "));\n";
              else
                o << pad << "const float2 " << pr << " = make_float2(erf_sign(" << m0 << ", " << y0 << "), erf_sign("
                  << m1 << ", " << y1 << "));\n";
            } else if (t.op == DFS_OP_LOG) {
              lanes[l].define(r0);
              lanes[l + 1].define(r1);
              o << pad << "const float2 " << pr << " = log_f32x2(" << val_of(l, 0) << ", " << val_of(l + 1, 0) << ");\n";
            } else {
              lanes[l].define(r0);
              lanes[l + 1].define(r1);
              o << pad << "const float2 " << pr << " = pk_add(" << val_of(l, 0) << ", " << val_of(l + 1, 0) << ", "
                << val_of(l, 1) << ", " << val_of(l + 1, 1) << ");\n";
            }
            o << pad << "const float " << r0 << " = " << pr << ".x;\n";
            o << pad << "const float " << r1 << " = " << pr << ".y;\n";
            curs[l][akey(t.args.back())] = r0;
            curs[l + 1][akey(t.args.back())] = r1;
          }
          continue;
        }
        for (int l = 0; l < w; ++l) {
          auto& cur = curs[l];
          LaneOps& lane = lanes[l];
          auto val = [&](size_t ai) { return val_of(l, ai); };
          const std::string res = res_of(l);
          if (is_elementwise(t.op)) {
            std::vector<std::string> in{val(0)};
            if (t.args.size() == 3) in.push_back(val(1));
            lane.emit(o, pad, T(dt), t.op, res, in);
            cur[akey(t.args.back())] = res;
          } else if (t.op == DFS_OP_SPMV && spre.count(i)) {
            o << pad << "const " << T(dt) << " " << res << " = " << spre.at(i) << "_" << l << ";\n";
            cur[akey(t.args[4])] = res;
          } else if (t.op == DFS_OP_SPMV) {
            const Arg& y = t.args[4];
            const std::string row = "(" + base.at(akey(y)) + " - " + std::to_string(y.part.vlo[0]) + "LL + " +
                                    eflat[s] + " + " + std::to_string(l) + ")";
            o << pad << "const " << T(dt) << " " << res << " = " << (i == staged ? "spmv_row_xs<" : "spmv_row<")
              << T(dt) << ">(" << ptr(t.args[0].root) << " + " << base.at(akey(t.args[0])) << ", "
              << ptr(t.args[1].root) << " + " << base.at(akey(t.args[1])) << ", " << ptr(t.args[2].root) << " + "
              << base.at(akey(t.args[2])) << ", " << ptr(t.args[3].root) << " + " << base.at(akey(t.args[3])) << ", "
              << row << (i == staged ? ", (const " + T(dt) + "*)dfs_xs_raw, xw_" : std::string()) << ");\n";
            cur[akey(y)] = res;
          } else if (is_reduction(t.op)) {
            const Acc* ac = nullptr;
            for (const Acc& x : accs)
              if (x.task == i) ac = &x;
            if (t.op == DFS_OP_DOT)
              o << pad << ac->var << " = red_fma(" << val(0) << ", " << val(1) << ", " << ac->var << ");\n";
            else
              o << pad << ac->var << " = " << ac->var << " + " << val(0) << ";\n";
          }
        }
      }
      // collect outputs to store
      for (int l = 0; l < w; ++l)
        for (int i = n.first; i < n.last; ++i) {
          const Task& t = S.tasks[i];
          if (t.scalar()) continue;
          const Arg* out = nullptr;
          if (is_elementwise(t.op)) out = &t.args.back();
          if (t.op == DFS_OP_SPMV) out = &t.args[4];
          if (!out || R(out->root).temp) continue;
          const std::string k = akey(*out);
          auto& vv = outvars[k];
          if (vv.size() < (size_t)(ns * w)) vv.resize(ns * w);
          vv[s * w + l] = curs[l].at(k);
        }
    }
    // stores (the last value written to each (root, partition) in the nest)
    for (auto& kv : outvars) {
      const Arg* a = nullptr;
      for (int i = n.first; i < n.last && !a; ++i) {
        const Task& t = S.tasks[i];
        if (t.scalar()) continue;
        for (size_t ai = 0; ai < t.args.size(); ++ai)
          if (!t.args[ai].imm && akey(t.args[ai]) == kv.first) a = &t.args[ai];
      }
      for (int s = 0; s < ns; ++s) {
        const std::string ad = addr(*a, eflat[s], erow[s], ecol[s]);
        if (w == 4 && a->dtype == DFS_F32) {
          o << pad << "st4(" << ad << ", f32x4{{" << kv.second[s * w] << ", " << kv.second[s * w + 1] << ", "
            << kv.second[s * w + 2] << ", " << kv.second[s * w + 3] << "}});\n";
        } else if (w == 2 && a->dtype == DFS_F64) {
          o << pad << "st2(" << ad << ", f64x2{{" << kv.second[s * w] << ", " << kv.second[s * w + 1] << "}});\n";
        } else {
          o << pad << "*(" << ad << ") = " << kv.second[s * w] << ";\n";
        }
      }
    }
  };

  // block-stride loops inside a point, grid-stride loops over a flat range
  const std::string st0 = flat ? "((i64)blockIdx.x * " + std::to_string(BD) + " + threadIdx.x)" : "(i64)threadIdx.x";
  const std::string stp = flat ? "gs" : std::to_string(BD);
  if (flat) o << ind << "  const i64 gs = (i64)gridDim.x * " << BD << ";\n";
  auto slot_off = [&](int u) { return flat ? std::to_string(u) + " * gs" : std::to_string(u * BD); };
  if (n.dims == 1 && n.coop) {
    // SpMV rows shared by lanes (spmv_warp).  Elements are dealt to threads
    // exactly as in the plain loops (vectors of V in thread order, then the
    // scalar tail), so reductions fused here sum in the same order; each trip
    // a warp takes 32 consecutive vectors, so all its lanes run the same trips
    o << ind << "  const i64 n = ";
    for (int d = 0; d < nd; ++d) o << (d ? " * " : "") << "ext" << d;
    o << ";\n";
    o << ind << "  const int lane_ = threadIdx.x & 31;\n";
    auto coop_spmv = [&](int w, const std::string& first, const std::string& pad) {
      for (int i = n.first; i < n.last; ++i) {
        const Task& t = S.tasks[i];
        if (t.op != DFS_OP_SPMV) continue;
        const Arg& y = t.args[4];
        const int dt = y.dtype;
        for (int l = 0; l < w; ++l)
          o << pad << "const " << T(dt) << " sp" << i << "_" << l << " = spmv_warp<" << T(dt) << ">("
            << ptr(t.args[0].root) << " + " << base.at(akey(t.args[0])) << ", " << ptr(t.args[1].root) << " + "
            << base.at(akey(t.args[1])) << ", " << ptr(t.args[2].root) << " + " << base.at(akey(t.args[2])) << ", "
            << ptr(t.args[3].root) << " + " << base.at(akey(t.args[3])) << ", (" << base.at(akey(y)) << " - "
            << y.part.vlo[0] << "LL + " << first << " + " << l << "), act_, " << spmv_k(t) << ");\n";
        spre[i] = "sp" + std::to_string(i);
      }
    };
    if (V > 1) {
      o << ind << "  const i64 nv = n / " << V << ";\n";
      o << ind << "  for (i64 wb = " << st0 << " - lane_; wb < nv; wb += " << stp << ") {\n";
      o << ind << "    const i64 v = wb + lane_;\n";
      o << ind << "    const bool act_ = v < nv;\n";
      coop_spmv(V, "v * " + std::to_string(V), ind + "    ");
      o << ind << "    if (act_) {\n";
      body(V, {"r"}, {"(v) * " + std::to_string(V)}, {""}, {""}, ind + "      ");
      o << ind << "    }\n";
      o << ind << "  }\n";
      o << ind << "  for (i64 wb = " << st0 << " - lane_; nv * " << V << " + wb < n; wb += " << stp << ") {\n";
      o << ind << "    const i64 e = nv * " << V << " + wb + lane_;\n";
    } else {
      o << ind << "  for (i64 wb = " << st0 << " - lane_; wb < n; wb += " << stp << ") {\n";
      o << ind << "    const i64 e = wb + lane_;\n";
    }
    o << ind << "    const bool act_ = e < n;\n";
    coop_spmv(1, "e", ind + "    ");
    o << ind << "    if (act_) {\n";
    body(1, {"t"}, {"e"}, {""}, {""}, ind + "      ");
    o << ind << "    }\n";
    o << ind << "  }\n";
  } else if (n.dims == 1) {
    // n elements in one contiguous range; vectors of V; main loop unrolled U
    o << ind << "  const i64 n = ";
    for (int d = 0; d < nd; ++d) o << (d ? " * " : "") << "ext" << d;
    o << ";\n";
    o << ind << "  if (n > 0) {\n";
    const std::string it = V > 1 ? "v" : "e";
    const std::string lim = V > 1 ? "nv" : "n";
    if (V > 1) o << ind << "    const i64 nv = n / " << V << ";\n";
    o << ind << "    i64 " << it << " = " << st0 << ";\n";
    auto flat_e = [&](const std::string& x) { return V > 1 ? "(" + x + ") * " + std::to_string(V) : "(" + x + ")"; };
    if (U > 1) {
      o << ind << "    for (; " << it << " + " << slot_off(U - 1) << " < " << lim << "; " << it << " += " << U
        << " * " << stp << ") {\n";
      std::vector<std::string> sl, ef, er, ec;
      for (int u = 0; u < U; ++u) {
        sl.push_back("u" + std::to_string(u));
        ef.push_back(flat_e(it + " + " + slot_off(u)));
        er.push_back("");
        ec.push_back("");
      }
      body(V, sl, ef, er, ec, ind + "      ");
      o << ind << "    }\n";
    }
    o << ind << "    for (; " << it << " < " << lim << "; " << it << " += " << stp << ") {\n";
    body(V, {"r"}, {flat_e(it)}, {""}, {""}, ind + "      ");
    o << ind << "    }\n";
    if (V > 1) {
      o << ind << "    for (i64 e = nv * " << V << " + " << st0 << "; e < n; e += " << stp << ") {\n";
      body(1, {"t"}, {"e"}, {""}, {""}, ind + "      ");
      o << ind << "    }\n";
    }
    o << ind << "  }\n";
  } else if (flat) {
    // a rectangle of nrows rows x ncols columns swept as one range of
    // (row, vector) cells with a grid stride; realigned rows start their
    // vectors after `hd` scalar columns and end with a scalar tail
    o << ind << "  const i64 nrows = " << (n.rank == 3 ? "ext0 * ext1" : "ext0") << ";\n";
    o << ind << "  const i64 ncols = " << (n.rank == 3 ? "ext2" : "ext1") << ";\n";
    o << ind << "  const i64 hd = " << (n.realign ? "min((i64)" + std::to_string(n.head) + ", ncols)" : "0") << ";\n";
    o << ind << "  const i64 nvr = (ncols - hd) / " << V << ";\n";
    o << ind << "  const i64 ncell = nrows * nvr;\n";
    o << ind << "  i64 c = " << st0 << ";\n";
    // 32-bit division by the constant row length when the range allows it
    const bool narrow = flat_cells < (int64_t(1) << 31);
    auto cell = [&](const std::string& cv, const std::string& sfx) {
      if (narrow)
        o << ind << "      const i64 i" << sfx << " = (i64)((u32)(" << cv << ") / (u32)nvr);\n";
      else
        o << ind << "      const i64 i" << sfx << " = (" << cv << ") / nvr;\n";
      o << ind << "      const i64 j" << sfx << " = hd + ((" << cv << ") - i" << sfx << " * nvr) * " << V << ";\n";
    };
    if (U > 1) {
      o << ind << "  for (; c + " << slot_off(U - 1) << " < ncell; c += " << U << " * gs) {\n";
      std::vector<std::string> sl, ef, er, ec;
      for (int u = 0; u < U; ++u) {
        cell("c + " + slot_off(u), std::to_string(u));
        sl.push_back("u" + std::to_string(u));
        ef.push_back("");
        er.push_back("i" + std::to_string(u));
        ec.push_back("j" + std::to_string(u));
      }
      body(V, sl, ef, er, ec, ind + "      ");
      o << ind << "  }\n";
    }
    o << ind << "  for (; c < ncell; c += gs) {\n";
    cell("c", "r");
    body(V, {"r"}, {""}, {"ir"}, {"jr"}, ind + "      ");
    o << ind << "  }\n";
    if (n.realign) {
      // the scalar head and tail columns of every row
      o << ind << "  const i64 nrem = ncols - nvr * " << V << ";\n";
      o << ind << "  if (nrem > 0) {\n";
      o << ind << "    for (i64 c2 = " << st0 << "; c2 < nrows * nrem; c2 += gs) {\n";
      o << ind << "      const i64 is = c2 / nrem;\n";
      o << ind << "      const i64 ks = c2 - is * nrem;\n";
      o << ind << "      const i64 js = ks < hd ? ks : hd + nvr * " << V << " + (ks - hd);\n";
      body(1, {"s"}, {""}, {"is"}, {"js"}, ind + "      ");
      o << ind << "    }\n";
      o << ind << "  }\n";
    }
  } else {
    // rows: each row of ncols elements is swept by the whole block
    o << ind << "  const i64 nrows = " << (n.rank == 3 ? "ext0 * ext1" : "ext0") << ";\n";
    o << ind << "  const i64 ncols = " << (n.rank == 3 ? "ext2" : "ext1") << ";\n";
    o << ind << "  for (i64 i = 0; i < nrows; ++i) {\n";
    if (V > 1 && n.realign) {
      o << ind << "    const i64 hd = min((i64)" << n.head << ", ncols);\n";
      o << ind << "    const i64 nv = (ncols - hd) / " << V << ";\n";
      o << ind << "    for (i64 v = threadIdx.x; v < nv; v += " << BD << ") {\n";
      body(V, {"r"}, {""}, {"i"}, {"hd + v * " + std::to_string(V)}, ind + "      ");
      o << ind << "    }\n";
      o << ind << "    for (i64 k = threadIdx.x; k < ncols - nv * " << V << "; k += " << BD << ") {\n";
      o << ind << "      const i64 js = k < hd ? k : hd + nv * " << V << " + (k - hd);\n";
      body(1, {"t"}, {""}, {"i"}, {"js"}, ind + "      ");
      o << ind << "    }\n";
    } else if (V > 1) {
      o << ind << "    const i64 nv = ncols / " << V << ";\n";
      o << ind << "    for (i64 v = threadIdx.x; v < nv; v += " << BD << ") {\n";
      body(V, {"r"}, {""}, {"i"}, {"v * " + std::to_string(V)}, ind + "      ");
      o << ind << "    }\n";
    } else {
      o << ind << "    i64 j = threadIdx.x;\n";
      if (U > 1) {
        o << ind << "    for (; j + " << (U - 1) * BD << " < ncols; j += " << U * BD << ") {\n";
        std::vector<std::string> sl, ef, er, ec;
        for (int u = 0; u < U; ++u) {
          sl.push_back("u" + std::to_string(u));
          ef.push_back("");
          er.push_back("i");
          ec.push_back("(j + " + std::to_string(u * BD) + ")");
        }
        body(1, sl, ef, er, ec, ind + "      ");
        o << ind << "    }\n";
      }
      o << ind << "    for (; j < ncols; j += " << BD << ") {\n";
      body(1, {"t"}, {""}, {"i"}, {"j"}, ind + "      ");
      o << ind << "    }\n";
    }
    o << ind << "  }\n";
  }
  // per-point partials of the reductions
  for (const Acc& ac : accs) {
    o << ind << "  { const " << T(ac.dt) << " tot = block_sum(" << ac.var << ", (" << T(ac.dt) << "*)red_buf);\n";
    o << ind << "    if (threadIdx.x == 0) ((" << T(ac.dt) << "*)P.partials)[" << ac.slot << "LL * P.red_stride + "
      << ptvar << "] = tot; }\n";
  }
  o << ind << "}\n";
  (void)g;
}

// Finishes every pending reduction: sum of the per-point partials in point
// order, folded into the register copy of the target.  Warp 0 sums (the
// order of sum_partials) and hands the totals to the CTA through shared
// memory: FP64 arithmetic is scarce on GB300 (about two lane operations per
// SM and clock), and every warp repeating the same sum cost about 0.5 us per
// reduction in an L2-resident CG iteration.  Called where every thread of the
// CTA arrives (after a grid barrier, or in the last CTA).
void Gen::emit_finalise(const char* ind) {
  if (pending_red.empty()) return;
  std::vector<std::string> bc;
  for (const Red& r : pending_red) {
    bc.push_back("bc" + std::to_string(nbc++));
    o << ind << "__shared__ " << T(r.dtype) << " " << bc.back() << ";\n";
  }
  o << ind << "if (threadIdx.x < 32) {\n";
  for (size_t j = 0; j < pending_red.size(); ++j) {
    const Red& r = pending_red[j];
    o << ind << "  const " << T(r.dtype) << " " << bc[j] << "_t = sum_partials((const " << T(r.dtype)
      << "*)P.partials + " << r.slot << "LL * P.red_stride, " << r.points << "LL);\n";
    o << ind << "  if (threadIdx.x == 0) " << bc[j] << " = " << bc[j] << "_t;\n";
  }
  o << ind << "}\n" << ind << "__syncthreads();\n";
  for (size_t j = 0; j < pending_red.size(); ++j) {
    const Red& r = pending_red[j];
    const std::string nm = sreg.at(r.root);
    if (have[r.root])
      o << ind << nm << " = op_add(" << nm << ", " << bc[j] << ");\n";
    else
      o << ind << nm << " = " << bc[j] << ";\n";
    have[r.root] = true;
  }
  pending_red.clear();
}

// After a grid barrier: the pending reductions and the scalar groups that
// follow (g, g+1, ... while scalar) run on warp 0 alone, and every 0-d value
// they set reaches the CTA's other warps through shared memory.  The values
// are those every thread would compute (the same operations on the same
// register copies); only the repetition goes.  FP64 arithmetic is scarce on
// GB300 (about two lane operations per SM and clock), and eight warps
// repeating a 128-partial sum and an IEEE division cost about 1 us per CG
// phase at 256^2.  Returns the first group after the scalar run.
int Gen::emit_warp0_scalars(int g) {
  int h = g;
  while (h < (int)S.groups.size() && S.groups[h].scalar) ++h;
  std::vector<int64_t> set;
  auto add = [&](int64_t r) {
    if (std::find(set.begin(), set.end(), r) == set.end()) set.push_back(r);
  };
  for (const Red& r : pending_red) add(r.root);
  for (int k = g; k < h; ++k)
    for (int i = S.groups[k].begin; i < S.groups[k].end; ++i) add(S.tasks[i].args.back().root);
  if (set.empty()) return g;
  std::map<int64_t, std::string> bc;
  for (int64_t r : set) {
    bc[r] = "bc" + std::to_string(nbc++);
    o << "    __shared__ " << T(R(r).dtype) << " " << bc[r] << ";\n";
  }
  o << "    if (threadIdx.x < 32) {\n";
  for (const Red& r : pending_red) {
    const std::string nm = sreg.at(r.root);
    o << "      { const " << T(r.dtype) << " tot = sum_partials((const " << T(r.dtype) << "*)P.partials + "
      << r.slot << "LL * P.red_stride, " << r.points << "LL);\n";
    if (have[r.root])
      o << "        " << nm << " = op_add(" << nm << ", tot); }\n";
    else
      o << "        " << nm << " = tot; }\n";
    have[r.root] = true;
  }
  pending_red.clear();
  for (int k = g; k < h; ++k) emit_scalar_group(k);
  o << "      if (threadIdx.x == 0) {\n";
  for (int64_t r : set) o << "        " << bc[r] << " = " << sreg.at(r) << ";\n";
  o << "      }\n    }\n    __syncthreads();\n";
  for (int64_t r : set) o << "    " << sreg.at(r) << " = " << bc[r] << ";\n";
  return h;
}

KernelCode Gen::run() {
  emit_params();
  std::ostringstream body;
  // the kernel body is generated into `o`; header assembled afterwards
  // x windows are staged by per-point nests whose SpMV rows are not shared
  // between lanes (the same test emit_vector_group and emit_nest apply)
  for (int g = 0; g < (int)S.groups.size() && !stage; ++g) {
    if (S.groups[g].scalar) continue;
    const std::vector<Nest> ns = nests_of(g);
    bool flat = ns.size() == 1;
    for (int i = S.groups[g].begin; i < S.groups[g].end && flat; ++i)
      if (is_reduction(S.tasks[i].op)) flat = false;
    if (flat && space_arg(S.tasks[S.groups[g].begin]).nd > 3) flat = false;
    for (const Nest& n : ns)
      if (!flat && n.dims == 1 && !n.coop)
        for (int i = n.first; i < n.last; ++i)
          if (S.tasks[i].op == DFS_OP_SPMV && S.tasks[i].args.size() == 6) stage = true;
  }
  o << "  __shared__ double red_buf[" << S.block << "];\n";
  o << "  Ctl* ctl = P.ctl;\n";
  if (stage) {
    kc.dyn_smem = DFS_SPMV_STAGE_BYTES;
    o << "  extern __shared__ __align__(128) unsigned char dfs_xs_raw[];\n";
    o << "  __shared__ __align__(8) u64 xs_mbar_;\n  u32 xs_ph_ = 0;\n  bool xs_live_ = true;\n";
    o << "  xstage_init(&xs_mbar_);\n";
  }
  emit_prologue();
  o << "  do {\n";
  for (int g = 0; g < (int)S.groups.size(); ++g) {
    if (g > 0 && !S.groups[g - 1].scalar) {
      ++nbar;
      o << "    if (!grid_barrier(ctl, " << nbar << "u, P.timeout_ns"
        << (S.debug_skip == nbar ? ", blockIdx.x != 0" : "") << ")) break;\n";
      const int h = emit_warp0_scalars(g);
      if (h > g) {
        g = h - 1;
        continue;
      }
    }
    emit_group(g);
  }
  o << "  } while (0);\n";
  o << "  if (last_cta(ctl)) {\n";
  if (!pending_red.empty()) {
    o << "    if (ld_relaxed_int(&ctl->err) == 0) {\n";
    emit_finalise("      ");
    o << "    }\n";
  }
  o << "    if (threadIdx.x == 0) {\n";
  for (const LaunchRoot& r : S.roots) {
    if (!r.zero_d || !r.live_out || r.param < 0) continue;
    o << "      *" << ptr(r.root) << " = " << sreg.at(r.root) << ";\n";
  }
  o << "    }\n";
  o << "    ctl_reset(ctl);\n";
  o << "  }\n";
  kc.nbarriers = nbar;

  std::ostringstream src;
  src << "#include \"dfs_device.cuh\"\nusing namespace dfs;\n";
  src << "struct Params {\n  void* p[" << std::max(1, kc.nptr) << "];\n  double imm[" << std::max(1, kc.nimm)
      << "];\n  void* partials;\n  Ctl* ctl;\n  u64 timeout_ns;\n  i64 red_stride;\n};\n";
  const std::string body_s = o.str();
  const size_t h = std::hash<std::string>{}(body_s);
  char nm[64];
  snprintf(nm, sizeof nm, "dfs_k%016zx", h);
  kc.name = nm;
  src << "extern \"C\" __global__ void __launch_bounds__(" << S.block << (S.min_blocks > 0 ? ", " + std::to_string(S.min_blocks) : std::string()) << ") " << kc.name
      << "(const __grid_constant__ Params P) {\n"
      << body_s << "}\n";
  kc.source = src.str();
  kc.key = kc.source;
  int64_t stride = 1;
  for (int64_t p : kc.red_points) stride = std::max(stride, p);
  kc.partial_bytes = (size_t)kc.nred * (size_t)stride * 8;
  return kc;
}

}  // namespace

const char* op_device_fn(int op) { return op_fn(op); }

std::string LaneOps::shared(const std::map<std::string, std::string>& m, const std::string& a) const {
  auto it = m.find(a);
  if (it != m.end()) return it->second;
  auto ng = neg_.find(a);
  if (ng != neg_.end()) {
    it = m.find(ng->second);
    if (it != m.end()) return it->second;
  }
  return std::string();
}

void LaneOps::emit(std::ostream& o, const std::string& pad, const std::string& T, int op, const std::string& res,
                   const std::vector<std::string>& in) {
  define(res);
  if (op == DFS_OP_ERF) {
    // |-a| = |a| bit for bit, so erf(|a|) serves a and its negation
    std::string m = shared(mag_, in[0]);
    if (m.empty()) {
      m = res + "_m";
      o << pad << "const " << T << " " << m << " = erf_mag(" << in[0] << ");\n";
    }
    mag_[in[0]] = m;
    o << pad << "const " << T << " " << res << " = erf_sign(" << m << ", " << in[0] << ");\n";
    return;
  }
  if (op == DFS_OP_NCDF) {
    // the scaled arguments of a and -a differ only in sign (round to
    // nearest is symmetric), so they share erf of their magnitude
    const std::string y = res + "_y";
    o << pad << "const " << T << " " << y << " = ncdf_arg(" << in[0] << ");\n";
    std::string m = shared(nmag_, in[0]);
    if (m.empty()) {
      m = res + "_m";
      o << pad << "const " << T << " " << m << " = erf_mag(" << y << ");\n";
    }
    nmag_[in[0]] = m;
    o << pad << "const " << T << " " << res << " = ncdf_of_erf(erf_sign(" << m << ", " << y << "));\n";
    return;
  }
  o << pad << "const " << T << " " << res << " = " << op_fn(op) << "(" << in[0];
  for (size_t k = 1; k < in.size(); ++k) o << ", " << in[k];
  o << ");\n";
  if (op == DFS_OP_NEG) {
    neg_.emplace(res, in[0]);
    neg_.emplace(in[0], res);
  }
}

std::string LaneOps::mag_of(int op, const std::string& in0) const {
  return shared(op == DFS_OP_NCDF ? nmag_ : mag_, in0);
}

void LaneOps::set_mag(int op, const std::string& in0, const std::string& m) {
  (op == DFS_OP_NCDF ? nmag_ : mag_)[in0] = m;
}

void LaneOps::define(const std::string& res) {
  if (!defined_.insert(res).second)
    throw std::runtime_error("code generator: value " + res + " defined twice in one loop body");
}

KernelCode generate(const LaunchSpec& spec) {
  Gen g(spec);
  return g.run();
}

}  // namespace dfs
