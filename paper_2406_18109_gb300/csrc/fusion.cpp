// fusion.cpp -- the host fusion pass.
//
//  * longest_fusible_prefix: the greedy forward dataflow of Section 4.2.2
//    applying the four constraints of Fig. 5 (launch-domain equivalence,
//    true dependence, anti-dependence, reduction) with constant-time partition
//    comparisons (Section 4.2.1).
//  * is_temporary: Def. 4 (temporary stores), with covers() evaluated in
//    closed form for affine tilings.
//  * analyse: cuts the window into fused groups, finds the temporaries of
//    each group and packs groups into launches (one per group, or one
//    persistent kernel per flush with grid barriers at the cuts).
//  * canonical_key: the alpha-renamed, De Bruijn-like window form of
//    Section 5.2, used to memoise analysis and code generation.
#include <algorithm>
#include <cstdio>
#include <sstream>

#include "runtime.hpp"

namespace dfs {

bool NPart::operator==(const NPart& o) const {
  if (kind != o.kind || nd != o.nd) return false;
  for (int d = 0; d < nd; ++d) {
    if (vlo[d] != o.vlo[d] || vhi[d] != o.vhi[d]) return false;
    if (kind == 1 && (tile[d] != o.tile[d] || off[d] != o.off[d] || proj[d] != o.proj[d]))
      return false;
  }
  return true;
}

std::string NPart::key() const {
  std::ostringstream s;
  s << (kind ? "T" : "N") << nd;
  for (int d = 0; d < nd; ++d) {
    s << "[" << vlo[d] << ":" << vhi[d];
    if (kind) s << "|" << tile[d] << "," << off[d] << "," << proj[d];
    s << "]";
  }
  return s.str();
}

int64_t Task::npoints() const {
  int64_t n = 1;
  for (int d = 0; d < dnd; ++d) n *= dom[d];
  return n;
}

bool Task::same_domain(const Task& o) const {
  if (dnd != o.dnd) return false;
  for (int d = 0; d < dnd; ++d)
    if (dom[d] != o.dom[d]) return false;
  return true;
}

bool Task::scalar() const {
  for (const Arg& a : args)
    if (!a.imm && a.nd != 0) return false;
  return true;
}

// ----------------------------------------------------------- Section 4.2.2
int longest_fusible_prefix(const std::vector<Task>& w, int start) {
  struct Access {
    int64_t root;
    const NPart* part;
  };
  std::vector<Access> writes, reads;
  std::set<int64_t> reduced, accessed;
  int f = start;
  for (int j = start; j < (int)w.size(); ++j) {
    const Task& t = w[j];
    bool ok = true;
    if (j > start) {
      // launch-domain equivalence
      if (!t.same_domain(w[start])) ok = false;
      for (const Arg& b : t.args) {
        if (b.imm || !ok) continue;
        if (b.is_r() || b.is_w()) {
          // true dependence: an earlier write of (S, P), then R/W of (S, P'), P != P'
          for (const Access& a : writes)
            if (a.root == b.root && *a.part != b.part) ok = false;
          // reduction: an earlier reduction to S, then R/W of S
          if (reduced.count(b.root)) ok = false;
        }
        // anti-dependence: an earlier read of (S, P), then a write of (S, P'), P != P'
        if (b.is_w())
          for (const Access& a : reads)
            if (a.root == b.root && *a.part != b.part) ok = false;
        // reduction: an earlier R/W of S, then a reduction to S
        if (b.is_rd() && accessed.count(b.root)) ok = false;
      }
    }
    if (!ok) break;
    for (const Arg& b : t.args) {
      if (b.imm) continue;
      if (b.is_w()) writes.push_back({b.root, &b.part});
      if (b.is_r()) reads.push_back({b.root, &b.part});
      if (b.is_rd()) reduced.insert(b.root);
      if (b.is_r() || b.is_w()) accessed.insert(b.root);
    }
    f = j + 1;
  }
  return f - start;
}

// ------------------------------------------------------------- Section 5.1
// covers(S, P): the union of the sub-stores over the launch domain is all of
// S.  For None this is "the view is the whole root".  For an affine tiling the
// union is a product of per-dimension intervals, each a run of contiguous
// tiles [off, off + tile * count) clipped to the view.
bool covers(const NPart& p, const Task& t, const RootInfo& ri) {
  for (int d = 0; d < p.nd; ++d)
    if (p.vlo[d] != 0 || p.vhi[d] != ri.shape[d]) return false;
  if (p.kind == 0) return true;
  for (int d = 0; d < p.nd; ++d) {
    const int c = p.proj[d];
    if (c < 0 || c >= t.dnd) return false;
    const int64_t count = t.dom[c];
    if (p.tile[d] <= 0 || count <= 0) return false;
    const int64_t lo = p.off[d], hi = p.off[d] + p.tile[d] * count;
    if (lo > 0 || hi < ri.shape[d]) return false;
  }
  return true;
}

bool is_temporary(const std::vector<Task>& w, int b, int e, int64_t root, const RootInfo& ri) {
  // (3) no live application reference; caller-owned memory is always kept
  if (ri.app_live || ri.wrapped) return false;
  // (2) no task after the prefix reads or reduces to S
  for (int k = e; k < (int)w.size(); ++k)
    for (const Arg& a : w[k].args)
      if (!a.imm && a.root == root && (a.is_r() || a.is_rd())) return false;
  // (1) every read is preceded by a covering write through the same partition
  for (int j = b; j < e; ++j) {
    for (const Arg& r : w[j].args) {
      if (r.imm || r.root != root || !r.is_r()) continue;
      bool ok = false;
      for (int i = b; i < j && !ok; ++i)
        for (const Arg& a : w[i].args)
          if (!a.imm && a.root == root && a.is_w() && a.part == r.part && covers(a.part, w[i], ri)) {
            ok = true;
            break;
          }
      if (!ok) return false;
    }
  }
  return true;
}

// Iteration space of a task: the per-point sub-store shape of the argument
// that drives its loop (the output of an element-wise task, the input of a
// reduction, the rows of an SpMV).  Tasks with equal keys can share one
// loop nest; a temporary shared by tasks with different keys is stored.
std::string iteration_space_key(const Task& t) {
  const Arg* s = nullptr;
  if (t.op == DFS_OP_DOT || t.op == DFS_OP_SUM) {
    s = &t.args[0];
  } else if (t.op == DFS_OP_SPMV) {
    s = &t.args[4];
  } else {
    s = &t.args.back();
  }
  std::ostringstream o;
  o << "d" << t.dnd;
  for (int d = 0; d < t.dnd; ++d) o << "," << t.dom[d];
  o << ";n" << s->nd;
  if (s->nd == 0) return o.str();
  const NPart& p = s->part;
  o << (p.kind ? "T" : "N");
  for (int d = 0; d < p.nd; ++d) {
    o << "[" << (p.vhi[d] - p.vlo[d]);
    if (p.kind) o << "|" << p.tile[d] << "," << (p.off[d] - p.vlo[d]) << "," << p.proj[d];
    o << "]";
  }
  return o.str();
}

Plan analyse(const std::vector<Task>& w, const std::map<int64_t, RootInfo>& roots, bool fusion,
             int launch_mode) {
  Plan plan;
  const int n = (int)w.size();
  int s = 0;
  while (s < n) {
    const int f = fusion ? longest_fusible_prefix(w, s) : 1;
    Group g;
    g.begin = s;
    g.end = s + f;
    g.scalar = true;
    for (int i = g.begin; i < g.end; ++i)
      if (!w[i].scalar()) g.scalar = false;
    plan.groups.push_back(g);
    s += f;
  }
  if (fusion) {
    for (int gi = 0; gi < (int)plan.groups.size(); ++gi) {
      const Group& g = plan.groups[gi];
      std::set<int64_t> seen;
      for (int i = g.begin; i < g.end; ++i)
        for (const Arg& a : w[i].args)
          if (!a.imm) seen.insert(a.root);
      for (int64_t r : seen) {
        const RootInfo& ri = roots.at(r);
        if (!is_temporary(w, g.begin, g.end, r, ri)) continue;
        // registers only when every access of r in the group shares one loop nest
        std::set<std::string> spaces;
        for (int i = g.begin; i < g.end; ++i)
          for (const Arg& a : w[i].args)
            if (!a.imm && a.root == r) spaces.insert(iteration_space_key(w[i]));
        if (ri.ndim == 0 || spaces.size() == 1) plan.temps.insert({gi, r});
      }
    }
  }
  const int ng = (int)plan.groups.size();
  if (launch_mode == DFS_LAUNCH_PERSISTENT) {
    const int max_phases = 64;
    for (int g = 0; g < ng; g += max_phases) plan.launches.push_back({g, std::min(ng, g + max_phases)});
  } else {
    for (int g = 0; g < ng; ++g) plan.launches.push_back({g, g + 1});
  }
  return plan;
}

// ------------------------------------------------------------- Section 5.2
// The key is a compact binary string (raw 64-bit words): task ops and
// domains, and per argument the first-occurrence number of its root, the
// privilege and the normalised partition; each root's dtype, shape and
// liveness bits are recorded at its first occurrence.  Immediate values and
// store identities are left out, so isomorphic windows share a key.
std::string canonical_key(const std::vector<Task>& w, const std::map<int64_t, RootInfo>& roots) {
  std::map<int64_t, int64_t> ids;
  std::string o;
  o.reserve(w.size() * 256);
  auto put = [&o](int64_t v) { o.append(reinterpret_cast<const char*>(&v), sizeof v); };
  for (const Task& t : w) {
    put(-1 - t.op);
    put(t.dnd);
    for (int d = 0; d < t.dnd; ++d) put(t.dom[d]);
    put((int64_t)t.args.size());
    for (const Arg& a : t.args) {
      if (a.imm) {
        put(-7);
        continue;
      }
      auto it = ids.find(a.root);
      if (it == ids.end()) {
        const int64_t id = (int64_t)ids.size();
        ids[a.root] = id;
        const RootInfo& ri = roots.at(a.root);
        put(-8);
        put(a.dtype);
        put(ri.ndim);
        for (int d = 0; d < ri.ndim; ++d) put(ri.shape[d]);
        put((ri.app_live ? 1 : 0) | (ri.wrapped ? 2 : 0) | (ri.valid ? 4 : 0));
        put(id);
      } else {
        put(it->second);
      }
      put(a.priv * 16 + a.redop);
      const NPart& p = a.part;
      put(p.kind * 16 + p.nd);
      for (int d = 0; d < p.nd; ++d) {
        put(p.vlo[d]);
        put(p.vhi[d]);
        if (p.kind) {
          put(p.tile[d]);
          put(p.off[d]);
          put(p.proj[d]);
        }
      }
    }
  }
  return o;
}

}  // namespace dfs
