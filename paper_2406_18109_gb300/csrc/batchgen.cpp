// batchgen.cpp -- one size-generic kernel for K isomorphic instances of a
// launch (batched execution of the fused plan of Section 4.2.2).
//
// The fused groups of the plan run in program order, exactly as in a single
// launch, but every vector group processes the points of all instances: a
// device work list holds, per group, the prefix offsets of the instances'
// point counts, and each CTA locates the instance of a global point by
// binary search.  Sizes, tiles, offsets, store addresses and immediates are
// read from the instance's descriptor; nothing instance-specific is compiled
// in, so one kernel serves problems of any size.
//
// 0-d values of an instance live in a per-instance slot array: scalar groups
// and the finishing of reductions run one warp per instance (lanes compute
// redundantly, lane 0 stores), between grid barriers.  A reduction's partials
// are indexed by global point, so instance i's partials are a contiguous run
// summed in point order by the same routine a single launch uses -- batched
// results are bit-identical to running each instance alone.
#include <algorithm>
#include <sstream>

#include "runtime.hpp"

namespace dfs {
namespace {

bool is_ew(int op) { return op_device_fn(op) != nullptr; }
bool is_red(int op) { return op == DFS_OP_DOT || op == DFS_OP_SUM; }

const Arg& space(const Task& t) {
  if (is_red(t.op)) return t.args[0];
  if (t.op == DFS_OP_SPMV) return t.args[4];
  return t.args.back();
}

std::string akey(const Arg& a) { return std::to_string(a.root) + "@" + a.part.key(); }

class BatchGen {
 public:
  BatchGen(const LaunchSpec& s, int vec, bool co) : S(s), V(vec), coop(co) {}
  bool run(BatchCode& out, std::string& why);

 private:
  const LaunchSpec& S;
  const int V;
  const bool coop;  // some instance's SpMV shares rows between lanes
  std::ostringstream o;
  BatchCode bc;
  std::map<int64_t, int> ptr_of;          // root -> pointer slot
  std::map<int64_t, int> sslot;           // 0-d root -> scalar slot
  std::map<std::string, int> vbase;       // akey -> first v slot (tile, off, vlo, vhi or vlo, vhi)
  std::map<int, int> kbase;               // SpMV task -> slot of its lanes per row
  int nticket = 0;                        // dynamically dealt phases so far
  std::map<int64_t, bool> produced;       // 0-d root holds a kernel-produced value
  std::map<int64_t, std::string> local;   // 0-d root -> register inside the open scalar phase
  struct Pending { int slot; int64_t root; int dtype; int pslot; };
  std::vector<Pending> pending;
  std::map<int, int> group_pslot;         // vector group -> prefix slot
  int nbar = 0;
  int nreg = 0;
  bool stage = false;  // some SpMV carries x windows, staged in shared memory

  const LaunchRoot& R(int64_t r) const { return S.roots[S.root_index.at(r)]; }
  std::string T(int dt) const { return dtype_cname(dt); }
  int vslots(const Task& t, size_t ai);
  int kslot(const Task& t);
  std::string imm(int task, int arg, int dt);
  std::string zero_d_read(int64_t root, int dt, bool in_scalar);
  void vector_group(int g);
  void open_scalar(const char* ind);
  void close_scalar(const char* ind);
  void scalar_tasks(int g, const char* ind);
  void finals(const char* ind);
  void barrier();
};

// One descriptor slot holding the instance's lanes per row (spmv_lanes) of
// an SpMV task's matrix.
int BatchGen::kslot(const Task& t) {
  const int task = (int)(&t - &S.tasks[0]);
  auto it = kbase.find(task);
  if (it != kbase.end()) return it->second;
  const int b = bc.nv;
  bc.v_src.push_back({task, 1, 4});
  bc.nv += 1;
  kbase[task] = b;
  return b;
}

int BatchGen::vslots(const Task& t, size_t ai) {
  const Arg& a = t.args[ai];
  const std::string k = akey(a);
  auto it = vbase.find(k);
  if (it != vbase.end()) return it->second;
  const int b = bc.nv;
  const int task = (int)(&t - &S.tasks[0]);
  if (a.part.kind == 1) {
    for (int f = 0; f < 4; ++f) bc.v_src.push_back({task, (int)ai, f});
    bc.nv += 4;
  } else {
    bc.v_src.push_back({task, (int)ai, 2});
    bc.v_src.push_back({task, (int)ai, 3});
    bc.nv += 2;
  }
  vbase[k] = b;
  return b;
}

std::string BatchGen::imm(int task, int arg, int dt) {
  const int k = bc.nimm++;
  bc.imm_src.push_back({task, arg});
  return "((" + T(dt) + ")D.imm[" + std::to_string(k) + "])";
}

// Value of a 0-d store as seen at this point of the kernel.
std::string BatchGen::zero_d_read(int64_t root, int dt, bool in_scalar) {
  const std::string cast = "(" + T(dt) + ")";
  if (in_scalar && local.count(root)) return local.at(root);
  if (produced[root]) return cast + "ld(sv + " + std::to_string(sslot.at(root)) + ")";
  const LaunchRoot& r = R(root);
  if (r.valid_before && r.param >= 0)
    return cast + "ld((const " + T(r.dtype) + "*)D.p[" + std::to_string(ptr_of.at(root)) + "])";
  return cast + "0";
}

void BatchGen::barrier() {
  ++nbar;
  // test hook: CTA 0 withholds its arrival at barrier number debug_skip
  o << "    if (!grid_barrier(ctl, " << nbar << "u, P.timeout_ns" << (S.debug_skip == nbar ? ", blockIdx.x != 0" : "")
    << ")) break;\n";
}

void BatchGen::open_scalar(const char* ind) {
  o << ind << "{ // per-instance scalars: one warp per instance\n";
  o << ind << "  const int lane = threadIdx.x & 31;\n";
  o << ind << "  for (i64 inst = ((i64)blockIdx.x * " << S.block << " + threadIdx.x) >> 5; inst < NI; inst += ((i64)gridDim.x * "
    << S.block << ") >> 5) {\n";
  o << ind << "    const Inst& D = P.insts[inst];\n";
  o << ind << "    double* sv = P.sval + inst * " << std::max(1, bc.nsval) << "LL;\n";
  local.clear();
  finals(ind);
}

void BatchGen::close_scalar(const char* ind) {
  o << ind << "    if (lane == 0) {\n";
  for (const auto& kv : local) o << ind << "      sv[" << sslot.at(kv.first) << "] = (double)" << kv.second << ";\n";
  o << ind << "    }\n";
  for (const auto& kv : local) produced[kv.first] = true;
  local.clear();
  o << ind << "  }\n" << ind << "}\n";
}

// Finishes the pending reductions of the open scalar phase's instance.
void BatchGen::finals(const char* ind) {
  for (const Pending& p : pending) {
    const std::string nm = "f" + std::to_string(nreg++);
    const std::string t = T(p.dtype);
    o << ind << "    const " << t << " " << nm << "_t = sum_partials((const " << t << "*)P.partials + " << p.slot
      << "LL * P.red_stride + P.prefix[" << p.pslot << "LL * (NI + 1) + inst], P.prefix[" << p.pslot
      << "LL * (NI + 1) + inst + 1] - P.prefix[" << p.pslot << "LL * (NI + 1) + inst]);\n";
    const LaunchRoot& r = R(p.root);
    const bool old = produced[p.root] || local.count(p.root) || (r.valid_before && r.param >= 0);
    if (old)
      o << ind << "    const " << t << " " << nm << " = op_add(" << zero_d_read(p.root, p.dtype, true) << ", " << nm
        << "_t);\n";
    else
      o << ind << "    const " << t << " " << nm << " = " << nm << "_t;\n";
    local[p.root] = nm;
  }
  pending.clear();
}

void BatchGen::scalar_tasks(int g, const char* ind) {
  const Group& G = S.groups[g];
  for (int i = G.begin; i < G.end; ++i) {
    const Task& t = S.tasks[i];
    const Arg& out = t.args.back();
    const int dt = out.dtype;
    std::vector<std::string> ins;
    for (size_t k = 0; k + 1 < t.args.size(); ++k) {
      const Arg& a = t.args[k];
      ins.push_back(a.imm ? imm(i, (int)k, dt) : zero_d_read(a.root, dt, true));
    }
    const std::string nm = "x" + std::to_string(nreg++);
    o << ind << "    const " << T(dt) << " " << nm << " = " << op_device_fn(t.op) << "(";
    for (size_t k = 0; k < ins.size(); ++k) o << (k ? ", " : "") << ins[k];
    o << ");\n";
    local[out.root] = nm;
  }
}

void BatchGen::vector_group(int g) {
  const Group& G = S.groups[g];
  const int ps = bc.nprefix++;
  bc.prefix_task.push_back(G.begin);
  group_pslot[g] = ps;
  const int BD = S.block;
  const int U = std::max(1, S.unroll);
  o << "    { // group " << g << ": tasks " << G.begin << ".." << G.end - 1 << ", points of every instance\n";
  o << "      const i64* pf = P.prefix + " << ps << "LL * (NI + 1);\n";
  o << "      const i64 tot = pf[NI];\n";
  // points are dealt dynamically (one ticket counter per phase, up to
  // kTickets phases): uneven points finish their phase together
  if (nticket < 16) {
    const int q = nticket++;
    o << "      for (i64 gp = take_ticket(ctl, " << q << ", &s_ticket); gp < tot; gp = take_ticket(ctl, " << q
      << ", &s_ticket)) {\n";
  } else {
    o << "      for (i64 gp = blockIdx.x; gp < tot; gp += gridDim.x) {\n";
  }
  o << "        const i64 inst = find_inst(pf, NI, gp);\n";
  o << "        const i64 q0 = gp - pf[inst];\n";
  o << "        const Inst& D = P.insts[inst];\n";
  o << "        const double* sv = P.sval + inst * " << std::max(1, bc.nsval) << "LL;\n";
  const std::string ind = "        ";
  // loop nests: runs of consecutive tasks with one iteration space
  int i = G.begin;
  int nest_no = 0;
  while (i < G.end) {
    const std::string key = iteration_space_key(S.tasks[i]);
    int j = i + 1;
    while (j < G.end && iteration_space_key(S.tasks[j]) == key) ++j;
    if (nest_no++) o << ind << "__syncthreads();\n";
    o << ind << "{\n";
    // descriptors of the accesses
    std::map<std::string, std::string> base;
    int nb = 0;
    auto need_base = [&](const Task& t, size_t ai) {
      const Arg& a = t.args[ai];
      const std::string k = akey(a);
      if (base.count(k)) return base[k];
      const int vb = vslots(t, ai);
      const std::string nm = "b" + std::to_string(nb++);
      if (a.part.kind == 1) {
        o << ind << "  const i64 " << nm << " = max(q0 * D.v[" << vb << "] + D.v[" << vb + 1 << "], D.v[" << vb + 2
          << "]);\n";
      } else {
        o << ind << "  const i64 " << nm << " = D.v[" << vb << "];\n";
      }
      base[k] = nm;
      return nm;
    };
    const Task& t0 = S.tasks[i];
    const size_t sai = is_red(t0.op) ? 0 : (t0.op == DFS_OP_SPMV ? 4 : t0.args.size() - 1);
    {
      const int vb = vslots(t0, sai);
      o << ind << "  const i64 n = min(q0 * D.v[" << vb << "] + D.v[" << vb + 1 << "] + D.v[" << vb << "], D.v[" << vb + 3
        << "]) - max(q0 * D.v[" << vb << "] + D.v[" << vb + 1 << "], D.v[" << vb + 2 << "]);\n";
    }
    // typed pointers used by the nest
    std::set<int64_t> roots;
    for (int k = i; k < j; ++k)
      for (const Arg& a : S.tasks[k].args)
        if (!a.imm && a.nd > 0 && ptr_of.count(a.root)) roots.insert(a.root);
    for (int64_t r : roots)
      o << ind << "  " << T(R(r).dtype) << "* __restrict__ r" << ptr_of.at(r) << " = (" << T(R(r).dtype) << "*)D.p["
        << ptr_of.at(r) << "];\n";
    auto P_ = [&](int64_t r) { return "r" + std::to_string(ptr_of.at(r)); };
    // memory reads, in-nest writes, reductions
    struct Rd { std::string key, var; const Task* t; size_t ai; bool ro; };
    std::vector<Rd> reads;
    std::set<std::string> written, read_keys;
    struct Acc { int task; int slot; std::string var; int dt; };
    std::vector<Acc> accs;
    for (int k = i; k < j; ++k) {
      const Task& t = S.tasks[k];
      for (size_t ai = 0; ai < t.args.size(); ++ai) {
        const Arg& a = t.args[ai];
        if (a.imm || a.nd == 0) continue;
        if (t.op == DFS_OP_SPMV && ai != 4) continue;
        const std::string key = akey(a);
        const bool is_out = (is_ew(t.op) && ai + 1 == t.args.size()) || (t.op == DFS_OP_SPMV && ai == 4);
        if (!is_out && !written.count(key) && !read_keys.count(key)) {
          read_keys.insert(key);
          reads.push_back({key, "m" + std::to_string(reads.size()), &t, ai, !R(a.root).written});
          need_base(t, ai);
        }
        if (is_out) {
          written.insert(key);
          if (!R(a.root).temp || t.op == DFS_OP_SPMV) need_base(t, ai);
        }
      }
      if (t.op == DFS_OP_SPMV)
        for (size_t ai = 0; ai < t.args.size(); ++ai)
          if (ai != 4) need_base(t, ai);
      if (is_red(t.op)) {
        const Arg& out = t.args.back();
        Acc ac{k, bc.nred++, "acc" + std::to_string(bc.nred), out.dtype};
        accs.push_back(ac);
        o << ind << "  " << T(ac.dt) << " " << ac.var << " = " << T(ac.dt) << "(0);\n";
      }
    }
    // immediates
    std::map<std::pair<int, int>, std::string> immv;
    for (int k = i; k < j; ++k) {
      const Task& t = S.tasks[k];
      const int dt = t.args.back().dtype;
      for (size_t ai = 0; ai < t.args.size(); ++ai)
        if (t.args[ai].imm) {
          const std::string nm = "k" + std::to_string(k) + "_" + std::to_string(ai);
          o << ind << "  const " << T(dt) << " " << nm << " = " << imm(k, (int)ai, dt) << ";\n";
          immv[{k, (int)ai}] = nm;
        }
    }
    // 0-d operands, read once per point
    std::map<std::pair<int, int>, std::string> zv;
    for (int k = i; k < j; ++k) {
      const Task& t = S.tasks[k];
      const int dt = t.args.back().dtype;
      for (size_t ai = 0; ai < t.args.size(); ++ai) {
        const Arg& a = t.args[ai];
        if (a.imm || a.nd != 0 || a.is_rd()) continue;
        const std::string nm = "z" + std::to_string(k) + "_" + std::to_string(ai);
        o << ind << "  const " << T(dt) << " " << nm << " = " << zero_d_read(a.root, dt, false) << ";\n";
        zv[{k, (int)ai}] = nm;
      }
    }
    std::map<int, std::string> spre;  // SpMV task -> value computed before the body
    // the first SpMV of the nest that carries x windows: stage them for this
    // point (every thread of the CTA is here, at the same point)
    int staged = -1;
    for (int k = i; k < j && stage && staged < 0; ++k)
      if (S.tasks[k].op == DFS_OP_SPMV && S.tasks[k].args.size() == 6) staged = k;
    if (staged >= 0) {
      const Task& t = S.tasks[staged];
      const Arg& x = t.args[3];
      const int xb = vslots(t, 3);
      const std::string tn = T(x.dtype);
      o << ind << "  const XWin xw_ = xstage<" << tn << ">((" << tn << "*)dfs_xs_raw, " << DFS_SPMV_STAGE_BYTES / (int)dtype_size(x.dtype)
        << ", " << P_(x.root) << " + " << base.at(akey(x)) << ", D.v[" << xb + 1 << "] - D.v[" << xb
        << "], (const int*)" << P_(t.args[5].root) << " + " << base.at(akey(t.args[5]))
        << ", &xs_mbar_, xs_ph_, xs_live_, ctl, P.timeout_ns);\n";
    }
    auto body = [&](int w, const std::vector<std::string>& slots, const std::vector<std::string>& ef,
                    const std::string& pad) {
      const int ns = (int)slots.size();
      for (int s = 0; s < ns; ++s)
        for (const Rd& rd : reads) {
          const Arg& a = rd.t->args[rd.ai];
          const std::string ad = P_(a.root) + " + " + base.at(rd.key) + " + " + ef[s];
          const std::string v = rd.var + "_" + slots[s];
          if (w == 4 && a.dtype == DFS_F32)
            o << pad << "const f32x4 " << v << " = " << (rd.ro ? "ld4ro(" : "ld4(") << ad << ");\n";
          else if (w == 2 && a.dtype == DFS_F64)
            o << pad << "const f64x2 " << v << " = " << (rd.ro ? "ld2ro(" : "ld2(") << ad << ");\n";
          else
            o << pad << "const " << T(a.dtype) << " " << v << " = " << (rd.ro ? "ldro(" : "ld(") << ad << ");\n";
        }
      std::map<std::string, std::vector<std::string>> outv;
      std::map<std::string, const Arg*> outarg;
      for (int s = 0; s < ns; ++s)
        for (int l = 0; l < w; ++l) {
          std::map<std::string, std::string> cur;
          for (const Rd& rd : reads) {
            const std::string v = rd.var + "_" + slots[s];
            cur[rd.key] = w > 1 ? v + ".v[" + std::to_string(l) + "]" : v;
          }
          LaneOps lane;
          for (int k = i; k < j; ++k) {
            const Task& t = S.tasks[k];
            const int dt = space(t).dtype;   // the output's (y for an SpMV, whose last arg may be its windows)
            auto val = [&](size_t ai) -> std::string {
              const Arg& a = t.args[ai];
              if (a.imm) return immv.at({k, (int)ai});
              if (a.nd == 0) return zv.at({k, (int)ai});
              return cur.at(akey(a));
            };
            const std::string res = "v" + std::to_string(k) + "_" + slots[s] + "_" + std::to_string(l);
            if (is_ew(t.op)) {
              std::vector<std::string> in{val(0)};
              if (t.args.size() == 3) in.push_back(val(1));
              lane.emit(o, pad, T(dt), t.op, res, in);
              cur[akey(t.args.back())] = res;
            } else if (t.op == DFS_OP_SPMV && spre.count(k)) {
              o << pad << "const " << T(dt) << " " << res << " = " << spre.at(k) << "_" << l << ";\n";
              cur[akey(t.args[4])] = res;
            } else if (t.op == DFS_OP_SPMV) {
              const Arg& y = t.args[4];
              const int yb = vslots(t, 4);
              const std::string row = "(" + base.at(akey(y)) + " - D.v[" + std::to_string(yb + 2) + "] + " + ef[s] +
                                      " + " + std::to_string(l) + ")";
              o << pad << "const " << T(dt) << " " << res << " = " << (k == staged ? "spmv_row_xs<" : "spmv_row<")
                << T(dt) << ">(" << P_(t.args[0].root) << " + " << base.at(akey(t.args[0])) << ", "
                << P_(t.args[1].root) << " + " << base.at(akey(t.args[1])) << ", " << P_(t.args[2].root) << " + "
                << base.at(akey(t.args[2])) << ", " << P_(t.args[3].root) << " + " << base.at(akey(t.args[3])) << ", "
                << row << (k == staged ? ", (const " + T(dt) + "*)dfs_xs_raw, xw_" : std::string()) << ");\n";
              cur[akey(y)] = res;
            } else if (is_red(t.op)) {
              const Acc* ac = nullptr;
              for (const Acc& x : accs)
                if (x.task == k) ac = &x;
              if (t.op == DFS_OP_DOT)
                o << pad << ac->var << " = red_fma(" << val(0) << ", " << val(1) << ", " << ac->var << ");\n";
              else
                o << pad << ac->var << " = " << ac->var << " + " << val(0) << ";\n";
            }
          }
          for (int k = i; k < j; ++k) {
            const Task& t = S.tasks[k];
            const Arg* out = nullptr;
            if (is_ew(t.op)) out = &t.args.back();
            if (t.op == DFS_OP_SPMV) out = &t.args[4];
            if (!out || R(out->root).temp) continue;
            const std::string key = akey(*out);
            auto& vv = outv[key];
            if (vv.size() < (size_t)(ns * w)) vv.resize(ns * w);
            vv[s * w + l] = cur.at(key);
            outarg[key] = out;
          }
        }
      for (auto& kv : outv) {
        const Arg* a = outarg[kv.first];
        for (int s = 0; s < ns; ++s) {
          const std::string ad = P_(a->root) + " + " + base.at(kv.first) + " + " + ef[s];
          if (w == 4 && a->dtype == DFS_F32)
            o << pad << "st4(" << ad << ", f32x4{{" << kv.second[s * 4] << ", " << kv.second[s * 4 + 1] << ", "
              << kv.second[s * 4 + 2] << ", " << kv.second[s * 4 + 3] << "}});\n";
          else if (w == 2 && a->dtype == DFS_F64)
            o << pad << "st2(" << ad << ", f64x2{{" << kv.second[s * 2] << ", " << kv.second[s * 2 + 1] << "}});\n";
          else
            o << pad << "*(" << ad << ") = " << kv.second[s * w] << ";\n";
        }
      }
    };
    bool has_spmv = false;
    for (int k = i; k < j; ++k) has_spmv = has_spmv || (coop && S.tasks[k].op == DFS_OP_SPMV);
    if (has_spmv) {
      // SpMV rows shared by lanes (spmv_warp, lanes per row from the
      // instance's descriptor).  Elements are dealt to threads as in the
      // plain loops (vectors of V, then the scalar tail), so fused reductions
      // sum in the same order; a warp takes 32 consecutive vectors per trip
      o << ind << "  const int lane_ = threadIdx.x & 31;\n";
      auto coop_spmv = [&](int w, const std::string& first, const std::string& pad) {
        for (int k = i; k < j; ++k) {
          const Task& t = S.tasks[k];
          if (t.op != DFS_OP_SPMV) continue;
          const Arg& y = t.args[4];
          const int yb = vslots(t, 4);
          const int dt = y.dtype;
          for (int l = 0; l < w; ++l)
            o << pad << "const " << T(dt) << " sp" << k << "_" << l << " = spmv_warp<" << T(dt) << ">("
              << P_(t.args[0].root) << " + " << base.at(akey(t.args[0])) << ", " << P_(t.args[1].root) << " + "
              << base.at(akey(t.args[1])) << ", " << P_(t.args[2].root) << " + " << base.at(akey(t.args[2])) << ", "
              << P_(t.args[3].root) << " + " << base.at(akey(t.args[3])) << ", (" << base.at(akey(y)) << " - D.v["
              << yb + 2 << "] + " << first << " + " << l << "), act_, (int)D.v[" << kslot(t) << "]);\n";
          spre[k] = "sp" + std::to_string(k);
        }
      };
      if (V > 1) {
        o << ind << "  const i64 nv = n / " << V << ";\n";
        o << ind << "  for (i64 wb = (i64)threadIdx.x - lane_; wb < nv; wb += " << BD << ") {\n";
        o << ind << "    const i64 v = wb + lane_;\n";
        o << ind << "    const bool act_ = v < nv;\n";
        coop_spmv(V, "v * " + std::to_string(V), ind + "    ");
        o << ind << "    if (act_) {\n";
        body(V, {"r"}, {"(v) * " + std::to_string(V)}, ind + "      ");
        o << ind << "    }\n";
        o << ind << "  }\n";
        o << ind << "  for (i64 wb = (i64)threadIdx.x - lane_; nv * " << V << " + wb < n; wb += " << BD << ") {\n";
        o << ind << "    const i64 e = nv * " << V << " + wb + lane_;\n";
      } else {
        o << ind << "  for (i64 wb = (i64)threadIdx.x - lane_; wb < n; wb += " << BD << ") {\n";
        o << ind << "    const i64 e = wb + lane_;\n";
      }
      o << ind << "    const bool act_ = e < n;\n";
      coop_spmv(1, "e", ind + "    ");
      o << ind << "    if (act_) {\n";
      body(1, {"t"}, {"e"}, ind + "      ");
      o << ind << "    }\n";
      o << ind << "  }\n";
    }
    if (!has_spmv) {
      // block-stride loop over the point's n elements
      o << ind << "  if (n > 0) {\n";
      const std::string it = V > 1 ? "v" : "e";
      const std::string lim = V > 1 ? "nv" : "n";
      auto fe = [&](const std::string& x) { return V > 1 ? "(" + x + ") * " + std::to_string(V) : "(" + x + ")"; };
      if (V > 1) o << ind << "    const i64 nv = n / " << V << ";\n";
      o << ind << "    i64 " << it << " = threadIdx.x;\n";
      if (U > 1) {
        o << ind << "    for (; " << it << " + " << (U - 1) * BD << " < " << lim << "; " << it << " += " << U * BD << ") {\n";
        std::vector<std::string> sl, ef;
        for (int u = 0; u < U; ++u) {
          sl.push_back("u" + std::to_string(u));
          ef.push_back(fe(it + " + " + std::to_string(u * BD)));
        }
        body(V, sl, ef, ind + "      ");
        o << ind << "    }\n";
      }
      o << ind << "    for (; " << it << " < " << lim << "; " << it << " += " << BD << ") {\n";
      body(V, {"r"}, {fe(it)}, ind + "      ");
      o << ind << "    }\n";
      if (V > 1) {
        o << ind << "    for (i64 e = nv * " << V << " + threadIdx.x; e < n; e += " << BD << ") {\n";
        body(1, {"t"}, {"e"}, ind + "      ");
        o << ind << "    }\n";
      }
      o << ind << "  }\n";
    }
    for (const Acc& ac : accs) {
      o << ind << "  { const " << T(ac.dt) << " tot = block_sum(" << ac.var << ", (" << T(ac.dt) << "*)red_buf);\n";
      o << ind << "    if (threadIdx.x == 0) ((" << T(ac.dt) << "*)P.partials)[" << ac.slot
        << "LL * P.red_stride + gp] = tot; }\n";
      pending.push_back({ac.slot, S.tasks[ac.task].args.back().root, ac.dt, ps});
    }
    o << ind << "}\n";
    i = j;
  }
  o << "      }\n    }\n";
}

bool BatchGen::run(BatchCode& out, std::string& why) {
  // only 0-d and 1-D stores, 1-D launch domains and identity projections
  for (const Task& t : S.tasks) {
    for (const Arg& a : t.args) {
      if (a.imm) continue;
      if (a.nd > 1) return why = "a store of rank 2 or more", false;
      if (a.part.kind == 1 && a.part.proj[0] != 0) return why = "a projected tiling", false;
    }
    if (!t.scalar() && t.dnd != 1) return why = "a multi-dimensional launch domain", false;
  }
  for (const Group& G : S.groups) {
    if (G.scalar) continue;
    for (int i = G.begin; i < G.end; ++i)
      if (S.tasks[i].scalar()) return why = "a group mixes scalar and vector tasks (single-point instances)", false;
  }
  for (const LaunchRoot& r : S.roots) {
    if (r.param >= 0) ptr_of[r.root] = r.param;
    if (r.zero_d) sslot[r.root] = bc.nsval++;
  }
  bc.nptr = 0;
  for (const LaunchRoot& r : S.roots)
    if (r.param >= 0) bc.nptr = std::max(bc.nptr, r.param + 1);
  bc.ptr_roots.assign(bc.nptr, 0);
  for (const LaunchRoot& r : S.roots)
    if (r.param >= 0) bc.ptr_roots[r.param] = r.root;
  for (const LaunchRoot& r : S.roots) produced[r.root] = false;

  // staging x windows needs one-row-per-lane SpMVs (no lanes shared)
  for (const Task& t : S.tasks)
    if (!coop && t.op == DFS_OP_SPMV && t.args.size() == 6) stage = true;
  o << "  __shared__ double red_buf[" << S.block << "];\n";
  o << "  __shared__ i64 s_ticket;\n";
  o << "  Ctl* ctl = P.ctl;\n  const i64 NI = P.ninst;\n";
  if (stage) {
    bc.dyn_smem = DFS_SPMV_STAGE_BYTES;
    o << "  extern __shared__ __align__(128) unsigned char dfs_xs_raw[];\n";
    o << "  __shared__ __align__(8) u64 xs_mbar_;\n  u32 xs_ph_ = 0;\n  bool xs_live_ = true;\n";
    o << "  xstage_init(&xs_mbar_);\n";
  }
  o << "  do {\n";
  bool in_scalar = false, first = true;
  for (int g = 0; g < (int)S.groups.size(); ++g) {
    const Group& G = S.groups[g];
    if (G.scalar) {
      if (!in_scalar) {
        if (!first) barrier();
        open_scalar("    ");
        in_scalar = true;
      }
      scalar_tasks(g, "    ");
    } else {
      bool reads_pending = false;
      for (int i = G.begin; i < G.end; ++i)
        for (const Arg& a : S.tasks[i].args)
          for (const Pending& p : pending)
            if (!a.imm && a.root == p.root) reads_pending = true;
      if (in_scalar) {
        close_scalar("    ");
        in_scalar = false;
        barrier();
      } else if (!first) {
        barrier();
        if (reads_pending) {
          open_scalar("    ");
          close_scalar("    ");
          barrier();
        }
      }
      vector_group(g);
    }
    first = false;
  }
  if (in_scalar) close_scalar("    ");
  o << "  } while (0);\n";
  // the last CTA finishes what remains and publishes the 0-d results
  o << "  if (last_cta(ctl)) {\n";
  o << "    if (ld_relaxed_int(&ctl->err) == 0) {\n";
  o << "      const int lane = threadIdx.x & 31;\n";
  o << "      for (i64 inst = threadIdx.x >> 5; inst < NI; inst += " << S.block / 32 << ") {\n";
  o << "        const Inst& D = P.insts[inst];\n";
  o << "        double* sv = P.sval + inst * " << std::max(1, bc.nsval) << "LL;\n";
  local.clear();
  finals("    ");
  o << "        if (lane == 0) {\n";
  for (const LaunchRoot& r : S.roots) {
    if (!r.zero_d || !r.live_out || r.param < 0) continue;
    o << "          *(" << T(r.dtype) << "*)D.p[" << r.param << "] = " << zero_d_read(r.root, r.dtype, true) << ";\n";
  }
  o << "        }\n      }\n    }\n    ctl_reset(ctl);\n  }\n";
  bc.nbarriers = nbar;
  bc.vec = V;

  std::ostringstream src;
  src << "#include \"dfs_device.cuh\"\nusing namespace dfs;\n";
  src << "struct Inst {\n  void* p[" << std::max(1, bc.nptr) << "];\n  double imm[" << std::max(1, bc.nimm)
      << "];\n  i64 v[" << std::max(1, bc.nv) << "];\n};\n";
  src << "struct BP {\n  const Inst* insts;\n  const i64* prefix;\n  double* sval;\n  void* partials;\n  Ctl* ctl;\n"
         "  u64 timeout_ns;\n  i64 ninst;\n  i64 red_stride;\n};\n";
  src << "__device__ __forceinline__ i64 find_inst(const i64* pf, i64 n, i64 gp) {\n"
         "  i64 lo = 0, hi = n;\n"
         "  while (hi - lo > 1) { const i64 mid = (lo + hi) >> 1; if (pf[mid] <= gp) lo = mid; else hi = mid; }\n"
         "  return lo;\n}\n";
  const std::string body = o.str();
  char nm[64];
  snprintf(nm, sizeof nm, "dfs_b%016zx", std::hash<std::string>{}(body));
  bc.name = nm;
  src << "extern \"C\" __global__ void __launch_bounds__(" << S.block << (S.min_blocks > 0 ? ", " + std::to_string(S.min_blocks) : std::string()) << ") " << bc.name
      << "(const __grid_constant__ BP P) {\n" << body << "}\n";
  bc.source = src.str();
  out = bc;
  return true;
}

}  // namespace

bool generate_batch(const LaunchSpec& spec, int vec, bool coop, BatchCode& out, std::string& why) {
  BatchGen g(spec, vec, coop);
  return g.run(out, why);
}

}  // namespace dfs
