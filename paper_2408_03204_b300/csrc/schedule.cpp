// Graph rules and type schedules (Sec. 2 "Definitions", "Batched processing",
// "Type scheduling").  Host C++; the rest of the plan is built in plan.cpp.
//
// A schedule is a type string t_0..t_N with V_0 = every input and V_N = every output;
// for a chosen type the step takes the maximal ready set (every unscheduled node of
// that type whose predecessors are all scheduled), which keeps the sequence a
// causal, homogeneous partition (conditions (i)-(iii)).
//  - greedy: the type with the most ready nodes; ties go to the smallest type id.
//  - beam(B): expand every candidate by every type with a non-empty ready set, merge
//    equal scheduled sets keeping the smallest type string, stop at the first
//    expansion that completes (smallest complete string), else keep the B best by
//    (most nodes scheduled, smallest string).  beam(1) equals greedy.
//  - optimal: the same search without pruning.
//  - one-by-one: a single processing node per step, smallest original id first.
// Types i and o are never chosen mid-schedule; the o step comes last.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <queue>
#include <thread>
#include <unordered_map>

#include "plan.h"

namespace grafx {

namespace {

struct Bits {
  std::vector<uint64_t> w;
  int32_t count = 0;
  explicit Bits(size_t n = 0) : w((n + 63) / 64, 0) {}
  bool get(int32_t v) const { return (w[v >> 6] >> (v & 63)) & 1u; }
  void set(int32_t v) {
    uint64_t m = uint64_t(1) << (v & 63);
    if (!(w[v >> 6] & m)) { w[v >> 6] |= m; ++count; }
  }
  bool operator==(const Bits& o) const { return w == o.w; }
};

struct BitsHash {
  size_t operator()(const Bits& b) const {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t x : b.w) { h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2); }
    return size_t(h);
  }
};

struct Ctx {
  int32_t n;
  const std::vector<int32_t>* types;
  std::vector<std::vector<int32_t>> preds;
  std::vector<std::vector<int32_t>> of_type;  // nodes of each type, ascending id
  std::vector<int32_t> ptypes;                // processing types present, ascending
  Bits non_out;                               // every non-output node
  Bits inputs;
};

void ready_set(const Ctx& c, const Bits& sched, int32_t t, std::vector<int32_t>* out) {
  out->clear();
  for (int32_t v : c.of_type[t]) {
    if (sched.get(v)) continue;
    bool ok = true;
    for (int32_t p : c.preds[v]) {
      if (!sched.get(p)) { ok = false; break; }
    }
    if (ok) out->push_back(v);
  }
}

bool covers(const Bits& a, const Bits& b) {  // a superset of b
  for (size_t i = 0; i < a.w.size(); ++i)
    if ((a.w[i] & b.w[i]) != b.w[i]) return false;
  return true;
}

Ctx make_ctx(const std::vector<int32_t>& types, const std::vector<std::pair<int32_t, int32_t>>& edges) {
  Ctx c;
  c.n = int32_t(types.size());
  c.types = &types;
  c.preds.assign(c.n, {});
  for (auto& e : edges) c.preds[e.second].push_back(e.first);
  c.of_type.assign(GRAFX_N_TYPES, {});
  for (int32_t v = 0; v < c.n; ++v) c.of_type[types[v]].push_back(v);
  for (int32_t t = 0; t < GRAFX_N_TYPES; ++t)
    if (t != GRAFX_T_IN && t != GRAFX_T_OUT && !c.of_type[t].empty()) c.ptypes.push_back(t);
  c.non_out = Bits(c.n);
  c.inputs = Bits(c.n);
  for (int32_t v = 0; v < c.n; ++v) {
    if (types[v] != GRAFX_T_OUT) c.non_out.set(v);
    if (types[v] == GRAFX_T_IN) c.inputs.set(v);
  }
  return c;
}

template <class F>
void parallel_for(int32_t n, int32_t n_threads, F&& f) {
  if (n_threads <= 1 || n < 4) {
    for (int32_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int32_t> next(0);
  std::vector<std::thread> th;
  int32_t k = std::min(n_threads, n);
  for (int32_t j = 0; j < k; ++j)
    th.emplace_back([&]() {
      for (int32_t i; (i = next.fetch_add(1)) < n;) f(i);
    });
  for (auto& t : th) t.join();
}

int beam(const Ctx& c, int32_t width /* <=0: unlimited */, int32_t n_threads,
         std::vector<int32_t>* out) {
  if (covers(c.inputs, c.non_out)) {
    *out = {GRAFX_T_IN, GRAFX_T_OUT};
    return GRAFX_OK;
  }
  struct Cand { Bits s; std::vector<int32_t> str; };
  std::vector<Cand> cands{{c.inputs, {GRAFX_T_IN}}};
  const size_t kMaxStates = 4u << 20;
  while (true) {
    const int32_t nt = int32_t(c.ptypes.size());
    std::vector<Cand> exp(cands.size() * nt);
    std::vector<char> valid(exp.size(), 0);
    parallel_for(int32_t(exp.size()), c.n > 2000 ? n_threads : 1, [&](int32_t i) {
      const Cand& cd = cands[i / nt];
      int32_t t = c.ptypes[i % nt];
      std::vector<int32_t> r;
      ready_set(c, cd.s, t, &r);
      if (r.empty()) return;
      Cand nc{cd.s, cd.str};
      for (int32_t v : r) nc.s.set(v);
      nc.str.push_back(t);
      exp[i] = std::move(nc);
      valid[i] = 1;
    });
    std::unordered_map<Bits, size_t, BitsHash> where;
    std::vector<Cand> merged;
    for (size_t i = 0; i < exp.size(); ++i) {
      if (!valid[i]) continue;
      auto it = where.find(exp[i].s);
      if (it == where.end()) {
        where.emplace(exp[i].s, merged.size());
        merged.push_back(std::move(exp[i]));
      } else if (exp[i].str < merged[it->second].str) {
        merged[it->second].str = std::move(exp[i].str);
      }
    }
    if (merged.empty()) return fail(GRAFX_EINVAL, "schedule: no computable node (graph not valid)");
    const std::vector<int32_t>* best = nullptr;
    for (auto& m : merged)
      if (covers(m.s, c.non_out) && (!best || m.str < *best)) best = &m.str;
    if (best) {
      *out = *best;
      out->push_back(GRAFX_T_OUT);
      return GRAFX_OK;
    }
    std::sort(merged.begin(), merged.end(), [](const Cand& a, const Cand& b) {
      if (a.s.count != b.s.count) return a.s.count > b.s.count;
      return a.str < b.str;
    });
    if (width > 0 && int32_t(merged.size()) > width) merged.resize(width);
    if (merged.size() > kMaxStates) return fail(GRAFX_EINVAL, "optimal schedule: graph too large for exhaustive search");
    cands = std::move(merged);
  }
}

int greedy(const Ctx& c, std::vector<int32_t>* out) {
  Bits s = c.inputs;
  out->assign(1, GRAFX_T_IN);
  std::vector<int32_t> r, best;
  while (!covers(s, c.non_out)) {
    int32_t bt = -1;
    best.clear();
    for (int32_t t : c.ptypes) {
      ready_set(c, s, t, &r);
      if (r.size() > best.size()) { best = r; bt = t; }
    }
    if (bt < 0) return fail(GRAFX_EINVAL, "schedule: no computable node (graph not valid)");
    for (int32_t v : best) s.set(v);
    out->push_back(bt);
  }
  out->push_back(GRAFX_T_OUT);
  return GRAFX_OK;
}

void steps_from_string(const Ctx& c, const std::vector<int32_t>& str, Schedule* sc) {
  Bits s = c.inputs;
  sc->steps.clear();
  std::vector<int32_t> v0;
  for (int32_t v = 0; v < c.n; ++v)
    if ((*c.types)[v] == GRAFX_T_IN) v0.push_back(v);
  sc->steps.push_back(v0);
  std::vector<int32_t> r;
  for (size_t k = 1; k + 1 < str.size(); ++k) {
    ready_set(c, s, str[k], &r);
    for (int32_t v : r) s.set(v);
    sc->steps.push_back(r);
  }
  std::vector<int32_t> vn;
  for (int32_t v = 0; v < c.n; ++v)
    if ((*c.types)[v] == GRAFX_T_OUT) vn.push_back(v);
  sc->steps.push_back(vn);
  sc->string = str;
}

}  // namespace

int validate(const std::vector<int32_t>& types, const std::vector<std::pair<int32_t, int32_t>>& edges) {
  const int32_t n = int32_t(types.size());
  if (n == 0) return fail(GRAFX_EINVAL, "empty graph");
  for (int32_t t : types)
    if (t < 0 || t >= GRAFX_N_TYPES) return fail(GRAFX_ETYPE, "unknown node type " + std::to_string(t));
  for (auto& e : edges)
    if (e.first < 0 || e.first >= n || e.second < 0 || e.second >= n)
      return fail(GRAFX_EINVAL, "edge out of range");
  std::vector<int32_t> indeg(n, 0), outdeg(n, 0);
  for (auto& e : edges) { ++indeg[e.second]; ++outdeg[e.first]; }
  bool has_out = false;
  for (int32_t v = 0; v < n; ++v) {
    if (types[v] == GRAFX_T_IN && indeg[v]) return fail(GRAFX_EINVAL, "input node " + std::to_string(v) + " has in-edges");
    if (types[v] != GRAFX_T_IN && !indeg[v]) return fail(GRAFX_EINVAL, "node " + std::to_string(v) + " has no input");
    if (types[v] == GRAFX_T_OUT && outdeg[v]) return fail(GRAFX_EINVAL, "output node " + std::to_string(v) + " has out-edges");
    has_out |= types[v] == GRAFX_T_OUT;
  }
  if (!has_out) return fail(GRAFX_EINVAL, "graph has no output node");
  std::vector<std::vector<int32_t>> succ(n);
  for (auto& e : edges) succ[e.first].push_back(e.second);
  std::vector<int32_t> stack;
  for (int32_t v = 0; v < n; ++v)
    if (!indeg[v]) stack.push_back(v);
  int32_t seen = 0;
  while (!stack.empty()) {
    int32_t v = stack.back();
    stack.pop_back();
    ++seen;
    for (int32_t w : succ[v])
      if (--indeg[w] == 0) stack.push_back(w);
  }
  if (seen != n) return fail(GRAFX_ECYCLE, "graph has a cycle");
  return GRAFX_OK;
}

int make_schedule(const std::vector<int32_t>& types, const std::vector<std::pair<int32_t, int32_t>>& edges,
                  int method, int beam_width, int n_threads, Schedule* out) {
  int rc = validate(types, edges);
  if (rc) return rc;
  Ctx c = make_ctx(types, edges);
  std::vector<int32_t> str;
  switch (method) {
    case GRAFX_SCHED_GREEDY: rc = greedy(c, &str); break;
    case GRAFX_SCHED_BEAM:
      if (beam_width < 1) return fail(GRAFX_EINVAL, "beam_width must be >= 1");
      rc = beam(c, beam_width, n_threads, &str);
      break;
    case GRAFX_SCHED_OPTIMAL: {
      int32_t nproc = 0;
      for (int32_t t : types) nproc += (t != GRAFX_T_IN && t != GRAFX_T_OUT);
      if (nproc > 28) return fail(GRAFX_EINVAL, "optimal schedule is limited to 28 processing nodes");
      rc = beam(c, 0, n_threads, &str);
      break;
    }
    case GRAFX_SCHED_ONE_BY_ONE: {
      std::vector<int32_t> indeg(c.n, 0);
      std::vector<std::vector<int32_t>> succ(c.n);
      for (auto& e : edges) { ++indeg[e.second]; succ[e.first].push_back(e.second); }
      std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> heap;
      std::vector<int32_t> ins, outs;
      for (int32_t v = 0; v < c.n; ++v) {
        if (types[v] == GRAFX_T_IN) ins.push_back(v);
        if (types[v] == GRAFX_T_OUT) outs.push_back(v);
      }
      for (int32_t v : ins)
        for (int32_t w : succ[v]) --indeg[w];
      for (int32_t v = 0; v < c.n; ++v)
        if (types[v] != GRAFX_T_IN && types[v] != GRAFX_T_OUT && indeg[v] == 0) heap.push(v);
      out->steps.assign(1, ins);
      out->string.assign(1, GRAFX_T_IN);
      while (!heap.empty()) {
        int32_t v = heap.top();
        heap.pop();
        out->steps.push_back({v});
        out->string.push_back(types[v]);
        for (int32_t w : succ[v])
          if (--indeg[w] == 0 && types[w] != GRAFX_T_IN && types[w] != GRAFX_T_OUT) heap.push(w);
      }
      out->steps.push_back(outs);
      out->string.push_back(GRAFX_T_OUT);
      return GRAFX_OK;
    }
    default: return fail(GRAFX_EINVAL, "unknown schedule method");
  }
  if (rc) return rc;
  steps_from_string(c, str, out);
  return GRAFX_OK;
}

}  // namespace grafx
