// Task graphs of the numeric factorization and of the solves (host), see
// chol_plan.h.  The list order comes from a list schedule of the graph on
// the assumed number of concurrent blocks: tasks whose remaining critical
// path is longest start first, and a task is listed when it starts in the
// simulation, so the list is a topological order in which blocks seldom
// wait for a dependency.
#include "chol_plan.h"

#include <algorithm>
#include <new>
#include <queue>
#include <utility>

#include "symbolic.h"

namespace acopf {
namespace {

constexpr int32_t kSmallRows = 32;  // kCholWarpRows
constexpr int32_t kSmallCols = 8;   // kCholWarpCols

struct Builder {
  std::vector<int32_t> task, dep;
  std::vector<int32_t> dep_ptr{0};
  std::vector<double> dur;
  int32_t add(int32_t kind, int32_t a, int32_t b, int32_t c, double us) {
    task.insert(task.end(), {kind, a, b, c});
    dur.push_back(us);
    return int32_t(dur.size()) - 1;
  }
};

// Reorders the graph (tasks t with dependencies deps[t]) by a list schedule
// on `workers` concurrent workers; fills g and the estimates.
void schedule(const std::vector<int32_t>& task, const std::vector<std::vector<int32_t>>& deps,
              const std::vector<double>& dur, int32_t workers, CholGraph& g, double* makespan,
              double* critical, double* crit_by_kind = nullptr,
              const std::vector<std::vector<int32_t>>* xdeps = nullptr) {
  const int32_t nt = int32_t(dur.size());
  std::vector<std::vector<int32_t>> succ(static_cast<size_t>(nt));
  std::vector<int32_t> indeg(static_cast<size_t>(nt), 0);
  for (int32_t t = 0; t < nt; ++t)
    for (const int32_t d : deps[size_t(t)]) {
      succ[size_t(d)].push_back(t);
      indeg[size_t(t)]++;
    }
  // topological order (Kahn), then the bottom levels in reverse
  std::vector<int32_t> topo;
  topo.reserve(size_t(nt));
  {
    std::vector<int32_t> in = indeg;
    for (int32_t t = 0; t < nt; ++t)
      if (in[size_t(t)] == 0) topo.push_back(t);
    for (size_t q = 0; q < topo.size(); ++q)
      for (const int32_t s : succ[size_t(topo[q])])
        if (--in[size_t(s)] == 0) topo.push_back(s);
  }
  std::vector<double> bl(static_cast<size_t>(nt), 0.0);
  double crit = 0.0;
  for (auto it = topo.rbegin(); it != topo.rend(); ++it) {
    double b = 0.0;
    for (const int32_t s : succ[size_t(*it)]) b = std::max(b, bl[size_t(s)]);
    bl[size_t(*it)] = b + dur[size_t(*it)];
    crit = std::max(crit, bl[size_t(*it)]);
  }
  // list schedule: ready tasks by bottom level (ties: lower index first)
  auto cmp = [&](int32_t a, int32_t b) {
    return bl[size_t(a)] < bl[size_t(b)] || (bl[size_t(a)] == bl[size_t(b)] && a > b);
  };
  std::priority_queue<int32_t, std::vector<int32_t>, decltype(cmp)> ready(cmp);
  using Ev = std::pair<double, int32_t>;  // (finish time, task)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  std::vector<int32_t> in = indeg;
  for (int32_t t = 0; t < nt; ++t)
    if (in[size_t(t)] == 0) ready.push(t);
  std::vector<int32_t> order;
  order.reserve(size_t(nt));
  double now = 0.0;
  int32_t busy = 0;
  while (int32_t(order.size()) < nt) {
    while (busy < workers && !ready.empty()) {
      const int32_t t = ready.top();
      ready.pop();
      order.push_back(t);
      running.push({now + dur[size_t(t)], t});
      ++busy;
    }
    if (running.empty()) break;  // (a cycle: cannot happen for the graphs built here)
    const Ev e = running.top();
    running.pop();
    now = e.first;
    --busy;
    for (const int32_t s : succ[size_t(e.second)])
      if (--in[size_t(s)] == 0) ready.push(s);
  }
  while (!running.empty()) {
    now = std::max(now, running.top().first);
    running.pop();
  }
  std::vector<int32_t> pos(static_cast<size_t>(nt));
  for (int32_t k = 0; k < nt; ++k) pos[size_t(order[size_t(k)])] = k;
  g.task.resize(size_t(nt) * 4);
  g.dep_ptr.assign(size_t(nt) + 1, 0);
  g.dep.clear();
  g.xdep_ptr.assign(size_t(nt) + 1, 0);
  g.xdep.clear();
  for (int32_t k = 0; k < nt; ++k) {
    const int32_t t = order[size_t(k)];
    std::copy(task.begin() + 4 * t, task.begin() + 4 * t + 4, g.task.begin() + 4 * k);
    std::vector<int32_t> ds;
    for (const int32_t d : deps[size_t(t)]) ds.push_back(pos[size_t(d)]);
    std::sort(ds.begin(), ds.end());
    ds.erase(std::unique(ds.begin(), ds.end()), ds.end());
    g.dep.insert(g.dep.end(), ds.begin(), ds.end());
    g.dep_ptr[size_t(k) + 1] = int32_t(g.dep.size());
    if (xdeps) {
      ds = (*xdeps)[size_t(t)];
      std::sort(ds.begin(), ds.end());
      ds.erase(std::unique(ds.begin(), ds.end()), ds.end());
      g.xdep.insert(g.xdep.end(), ds.begin(), ds.end());
    }
    g.xdep_ptr[size_t(k) + 1] = int32_t(g.xdep.size());
  }
  if (makespan) *makespan = now;
  if (critical) *critical = crit;
  if (crit_by_kind) {  // the estimated time of each task kind along the critical path
    int32_t t = -1;
    for (int32_t u = 0; u < nt; ++u)
      if (indeg[size_t(u)] == 0 && (t < 0 || bl[size_t(u)] > bl[size_t(t)])) t = u;
    while (t >= 0) {
      crit_by_kind[task[4 * size_t(t)] & 7] += dur[size_t(t)];
      int32_t nx = -1;
      for (const int32_t s : succ[size_t(t)])
        if (nx < 0 || bl[size_t(s)] > bl[size_t(nx)]) nx = s;
      t = nx;
    }
  }
}

// The list schedule of a forest of tasks of equal duration on `workers`
// workers, in rounds: up to `workers` ready tasks start together and finish
// together; ready tasks with the longest remaining chain start first (ties:
// the most recently released; released tasks wait for the next round).  up[k] is task k's parent (-1: a root; parents
// have larger numbers than their children); `forward`: a task needs its
// children, else its parent.  False if `up` is not such a forest.
bool schedule_forest(const std::vector<int32_t>& task, const std::vector<int32_t>& up,
                     bool forward, int32_t workers, CholGraph& g) {
  const int32_t nt = int32_t(up.size());
  for (int32_t k = 0; k < nt; ++k)
    if (up[size_t(k)] >= nt || (up[size_t(k)] >= 0 && up[size_t(k)] <= k)) return false;
  std::vector<int32_t> kp(size_t(nt) + 1, 0), kids;  // children of each task
  for (int32_t k = 0; k < nt; ++k)
    if (up[size_t(k)] >= 0) kp[size_t(up[size_t(k)]) + 1]++;
  for (int32_t k = 0; k < nt; ++k) kp[size_t(k) + 1] += kp[size_t(k)];
  kids.resize(size_t(kp[size_t(nt)]));
  {
    std::vector<int32_t> nx(kp.begin(), kp.end() - 1);
    for (int32_t k = 0; k < nt; ++k)
      if (up[size_t(k)] >= 0) kids[size_t(nx[size_t(up[size_t(k)])]++)] = k;
  }
  // remaining chain length: forward, the path to the root; backward, the
  // longest path to a leaf
  std::vector<int32_t> bl(static_cast<size_t>(nt), 1);
  int32_t top = 0;
  if (forward) {
    for (int32_t k = nt - 1; k >= 0; --k)
      if (up[size_t(k)] >= 0) bl[size_t(k)] = bl[size_t(up[size_t(k)])] + 1;
  } else {
    for (int32_t k = 0; k < nt; ++k)
      if (up[size_t(k)] >= 0)
        bl[size_t(up[size_t(k)])] = std::max(bl[size_t(up[size_t(k)])], bl[size_t(k)] + 1);
  }
  for (int32_t k = 0; k < nt; ++k) top = std::max(top, bl[size_t(k)]);
  std::vector<std::vector<int32_t>> bucket(size_t(top) + 1);
  std::vector<int32_t> wait(static_cast<size_t>(nt));
  for (int32_t k = 0; k < nt; ++k) {
    wait[size_t(k)] = forward ? kp[size_t(k) + 1] - kp[size_t(k)] : (up[size_t(k)] >= 0 ? 1 : 0);
    if (wait[size_t(k)] == 0) bucket[size_t(bl[size_t(k)])].push_back(k);
  }
  std::vector<int32_t> order, round;
  order.reserve(size_t(nt));
  while (int32_t(order.size()) < nt) {
    round.clear();
    for (int32_t b = top; b >= 1 && int32_t(round.size()) < workers;) {
      if (bucket[size_t(b)].empty()) {
        top = --b;
        continue;
      }
      round.push_back(bucket[size_t(b)].back());
      bucket[size_t(b)].pop_back();
    }
    if (round.empty()) return false;
    order.insert(order.end(), round.begin(), round.end());
    auto release = [&](int32_t t) {
      bucket[size_t(bl[size_t(t)])].push_back(t);
      top = std::max(top, bl[size_t(t)]);
    };
    for (const int32_t k : round) {
      if (forward) {
        const int32_t p = up[size_t(k)];
        if (p >= 0 && --wait[size_t(p)] == 0) release(p);
      } else {
        for (int32_t q = kp[size_t(k)]; q < kp[size_t(k) + 1]; ++q) release(kids[size_t(q)]);
      }
    }
  }
  std::vector<int32_t> pos(static_cast<size_t>(nt));
  for (int32_t k = 0; k < nt; ++k) pos[size_t(order[size_t(k)])] = k;
  g.task.resize(size_t(nt) * 4);
  g.dep_ptr.assign(size_t(nt) + 1, 0);
  g.dep.clear();
  g.dep.reserve(size_t(kp[size_t(nt)]));
  g.xdep_ptr.assign(size_t(nt) + 1, 0);
  g.xdep.clear();
  for (int32_t k = 0; k < nt; ++k) {
    const int32_t t = order[size_t(k)];
    std::copy(task.begin() + 4 * t, task.begin() + 4 * t + 4, g.task.begin() + 4 * k);
    const size_t d0 = g.dep.size();
    if (forward) {
      for (int32_t q = kp[size_t(t)]; q < kp[size_t(t) + 1]; ++q) g.dep.push_back(pos[size_t(kids[size_t(q)])]);
    } else if (up[size_t(t)] >= 0) {
      g.dep.push_back(pos[size_t(up[size_t(t)])]);
    }
    std::sort(g.dep.begin() + d0, g.dep.end());
    g.dep_ptr[size_t(k) + 1] = int32_t(g.dep.size());
  }
  return true;
}

}  // namespace

acopf_status chol_plan(const CholSymbolic& sy, const CholPlanParams& prm, CholPlan& plan,
                       std::string& err) {
  try {
    plan = CholPlan{};
    const int32_t ns = sy.ns;
    const int32_t T = kCholTileEdge;
    std::vector<int32_t> W(static_cast<size_t>(ns)), H(static_cast<size_t>(ns));
    std::vector<double> cost(static_cast<size_t>(ns));
    for (int32_t s = 0; s < ns; ++s) {
      W[size_t(s)] = sy.sn_first[size_t(s) + 1] - sy.sn_first[size_t(s)];
      H[size_t(s)] = sy.sn_rowptr[size_t(s) + 1] - sy.sn_rowptr[size_t(s)];
    }
    for (int32_t s = 0; s < ns; ++s) {
      const double w = W[size_t(s)], m = H[size_t(s)] - w;
      double c = w * w * w / 6.0 + m * w * w / 2.0 + m * m * w / 2.0;
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
        const int32_t k = sy.kid[size_t(q)];
        const double mk = H[size_t(k)] - W[size_t(k)];
        c += mk * (mk + 1.0) / 2.0;
      }
      cost[size_t(s)] = c;
      if (sy.sn_parent[size_t(s)] >= 0 && sy.sn_parent[size_t(s)] <= s) {
        err = "task plan: the supernodes are not in postorder";
        return ACOPF_E_INVALID_ARG;
      }
    }
    // --- classes ------------------------------------------------------------
    plan.sn_class.assign(static_cast<size_t>(ns), kSnBlock);
    for (int32_t s = 0; s < ns; ++s) {
      const int64_t w = W[size_t(s)], h = H[size_t(s)], m = h - w;
      if (h <= kSmallRows && w <= kSmallCols)
        plan.sn_class[size_t(s)] = kSnSmall;
      else if (h * w + m * m > kCholBlockStage || h > kCholBlockMaxRows ||
               cost[size_t(s)] > prm.tile_fma)
        plan.sn_class[size_t(s)] = kSnTiled;
    }
    // --- bottom levels: bottom-closed small supernodes, by height ---------------
    {
      std::vector<int32_t> lv(static_cast<size_t>(ns), -1), cnt;
      for (int32_t s = 0; s < ns; ++s) {
        if (H[size_t(s)] > kCholBottomRows || W[size_t(s)] > kCholBottomCols) continue;
        int32_t l = 0;
        bool ok = true;
        for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1] && ok; ++q) {
          const int32_t k = sy.kid[size_t(q)];
          ok = lv[size_t(k)] >= 0;
          l = std::max(l, lv[size_t(k)] + 1);
        }
        if (!ok) continue;
        lv[size_t(s)] = l;
        if (int32_t(cnt.size()) <= l) cnt.resize(size_t(l) + 1, 0);
        cnt[size_t(l)]++;
      }
      int32_t nbl = 0;
      while (nbl < int32_t(cnt.size()) && cnt[size_t(nbl)] >= kCholBottomMinCount) ++nbl;
      plan.bot_ptr.assign(size_t(nbl) + 1, 0);
      for (int32_t s = 0; s < ns; ++s)
        if (lv[size_t(s)] >= 0 && lv[size_t(s)] < nbl) {
          plan.sn_class[size_t(s)] = kSnBottom;
          plan.bot_ptr[size_t(lv[size_t(s)]) + 1]++;
        }
      for (int32_t v = 0; v < nbl; ++v) plan.bot_ptr[size_t(v) + 1] += plan.bot_ptr[size_t(v)];
      plan.bot_sn.resize(size_t(plan.bot_ptr[size_t(nbl)]));
      std::vector<int32_t> nx(plan.bot_ptr.begin(), plan.bot_ptr.end() - 1);
      for (int32_t s = 0; s < ns; ++s)
        if (plan.sn_class[size_t(s)] == kSnBottom) plan.bot_sn[size_t(nx[size_t(lv[size_t(s)])]++)] = s;
      plan.bot_stage.assign(size_t(nbl), 0);
      for (int32_t v = 0; v < nbl; ++v)
        for (int32_t q = plan.bot_ptr[size_t(v)]; q < plan.bot_ptr[size_t(v) + 1]; ++q) {
          const int32_t t = plan.bot_sn[size_t(q)], m = H[size_t(t)] - W[size_t(t)];
          plan.bot_stage[size_t(v)] =
              std::max(plan.bot_stage[size_t(v)], H[size_t(t)] * W[size_t(t)] + m * (m + 1) / 2);
        }
      for (int32_t v = 0; v < nbl; ++v)  // one shape per warp where possible
        std::stable_sort(plan.bot_sn.begin() + plan.bot_ptr[size_t(v)],
                         plan.bot_sn.begin() + plan.bot_ptr[size_t(v) + 1], [&](int32_t a, int32_t b) {
                           return std::make_pair(W[size_t(a)], H[size_t(a)]) <
                                  std::make_pair(W[size_t(b)], H[size_t(b)]);
                         });
    }
    // --- warp-small supernodes: small ones whose descendants are all small
    // or bottom supernodes; the factorization's warp tasks (before the task
    // kernel) and the solves' warp tasks
    std::vector<char> wsmall(static_cast<size_t>(ns), 0);
    for (int32_t s = 0; s < ns; ++s) {
      if (plan.sn_class[size_t(s)] != kSnSmall) continue;
      bool ok = true;
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1] && ok; ++q) {
        const int32_t k = sy.kid[size_t(q)];
        ok = wsmall[size_t(k)] || plan.sn_class[size_t(k)] == kSnBottom;
      }
      wsmall[size_t(s)] = ok;
    }
    // the other small supernodes go into group tasks
    const auto small = [&](int32_t s) {
      return plan.sn_class[size_t(s)] == kSnSmall && !wsmall[size_t(s)];
    };
    // --- groups: cut the small forest into connected sets of bounded work ---
    std::vector<double> open_cost(static_cast<size_t>(ns), 0.0);
    std::vector<int32_t> open_cnt(static_cast<size_t>(ns), 0);
    std::vector<char> cut(static_cast<size_t>(ns), 0);
    std::vector<std::pair<double, int32_t>> kids;
    for (int32_t s = 0; s < ns; ++s) {
      if (!small(s)) continue;
      double S = cost[size_t(s)];
      int32_t C = 1;
      kids.clear();
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
        const int32_t k = sy.kid[size_t(q)];
        if (!small(k)) continue;
        kids.push_back({open_cost[size_t(k)], k});
        S += open_cost[size_t(k)];
        C += open_cnt[size_t(k)];
      }
      std::sort(kids.begin(), kids.end(), std::greater<>());
      for (const auto& kc : kids) {  // cut the heaviest children's sets first
        if (S <= prm.group_fma && C <= prm.group_members) break;
        cut[size_t(kc.second)] = 1;
        S -= kc.first;
        C -= open_cnt[size_t(kc.second)];
      }
      open_cost[size_t(s)] = S;
      open_cnt[size_t(s)] = C;
    }
    std::vector<int32_t> grp(static_cast<size_t>(ns), -1), top;
    for (int32_t s = ns - 1; s >= 0; --s) {
      if (!small(s)) continue;
      const int32_t p = sy.sn_parent[size_t(s)];
      if (p >= 0 && small(p) && !cut[size_t(s)]) {
        grp[size_t(s)] = grp[size_t(p)];
      } else {
        grp[size_t(s)] = int32_t(top.size());
        top.push_back(s);
      }
    }
    // number the groups by their top supernode (postorder)
    const int32_t ng = int32_t(top.size());
    {
      std::vector<int32_t> ord(static_cast<size_t>(ng)), ren(static_cast<size_t>(ng));
      for (int32_t g = 0; g < ng; ++g) ord[size_t(g)] = g;
      std::sort(ord.begin(), ord.end(),
                [&](int32_t a, int32_t b) { return top[size_t(a)] < top[size_t(b)]; });
      for (int32_t k = 0; k < ng; ++k) ren[size_t(ord[size_t(k)])] = k;
      for (int32_t s = 0; s < ns; ++s)
        if (grp[size_t(s)] >= 0) grp[size_t(s)] = ren[size_t(grp[size_t(s)])];
      std::vector<int32_t> t2(static_cast<size_t>(ng));
      for (int32_t g = 0; g < ng; ++g) t2[size_t(ren[size_t(g)])] = top[size_t(g)];
      top.swap(t2);
    }
    // levels within a group, members by (level, supernode)
    std::vector<int32_t> lvl(static_cast<size_t>(ns), 0);
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t p = sy.sn_parent[size_t(s)];
      if (grp[size_t(s)] >= 0 && p >= 0 && grp[size_t(p)] == grp[size_t(s)])
        lvl[size_t(p)] = std::max(lvl[size_t(p)], lvl[size_t(s)] + 1);
    }
    plan.grp_ptr.assign(size_t(ng) + 1, 0);
    for (int32_t s = 0; s < ns; ++s)
      if (grp[size_t(s)] >= 0) plan.grp_ptr[size_t(grp[size_t(s)]) + 1]++;
    for (int32_t g = 0; g < ng; ++g) plan.grp_ptr[size_t(g) + 1] += plan.grp_ptr[size_t(g)];
    plan.grp_sn.resize(size_t(plan.grp_ptr[size_t(ng)]));
    {
      std::vector<int32_t> nx(plan.grp_ptr.begin(), plan.grp_ptr.end() - 1);
      for (int32_t s = 0; s < ns; ++s)
        if (grp[size_t(s)] >= 0) plan.grp_sn[size_t(nx[size_t(grp[size_t(s)])]++)] = s;
    }
    plan.grp_lptr.assign(size_t(ng) + 1, 0);
    plan.grp_lev.clear();
    std::vector<double> grp_us(static_cast<size_t>(ng), 0.0), grp_solve_us(static_cast<size_t>(ng));
    for (int32_t g = 0; g < ng; ++g) {
      auto* b = plan.grp_sn.data() + plan.grp_ptr[size_t(g)];
      auto* e = plan.grp_sn.data() + plan.grp_ptr[size_t(g) + 1];
      std::stable_sort(b, e, [&](int32_t a, int32_t c) { return lvl[size_t(a)] < lvl[size_t(c)]; });
      const int32_t nlv = lvl[size_t(top[size_t(g)])] + 1;
      int32_t p = plan.grp_ptr[size_t(g)];
      double us = 1.0;
      for (int32_t v = 0; v < nlv; ++v) {
        plan.grp_lev.push_back(p);
        double mx = 0.0;
        int32_t cnt = 0;
        while (p < plan.grp_ptr[size_t(g) + 1] && lvl[size_t(plan.grp_sn[size_t(p)])] == v) {
          mx = std::max(mx, cost[size_t(plan.grp_sn[size_t(p)])]);
          ++p;
          ++cnt;
        }
        us += (1.5 + mx / 500.0) * double((cnt + 7) / 8);
      }
      plan.grp_lev.push_back(p);
      plan.grp_lptr[size_t(g) + 1] = int32_t(plan.grp_lev.size());
      grp_us[size_t(g)] = us;
      grp_solve_us[size_t(g)] = 1.0 + 1.5 * nlv;
    }
    // --- the warp tasks: both directions ordered by a list schedule on the
    // warps; wpos: a warp-small supernode's position in the forward list
    std::vector<int32_t> widx(static_cast<size_t>(ns), -1), wsn;
    for (int32_t s = 0; s < ns; ++s)
      if (wsmall[size_t(s)]) {
        widx[size_t(s)] = int32_t(wsn.size());
        wsn.push_back(s);
      }
    const int32_t nw = int32_t(wsn.size());
    {
      std::vector<int32_t> wtask(size_t(nw) * 4), wup(static_cast<size_t>(nw));
      for (int32_t k = 0; k < nw; ++k) {
        const int32_t s = wsn[size_t(k)], p = sy.sn_parent[size_t(s)];
        wtask[4 * size_t(k)] = kTaskBlock;
        wtask[4 * size_t(k) + 1] = s;
        wtask[4 * size_t(k) + 2] = wtask[4 * size_t(k) + 3] = 0;
        wup[size_t(k)] = p >= 0 ? widx[size_t(p)] : -1;
      }
      if (!schedule_forest(wtask, wup, true, prm.warps, plan.forward_warp) ||
          !schedule_forest(wtask, wup, false, prm.warps, plan.backward_warp)) {
        err = "task plan: the supernodal tree is not a forest in postorder";
        return ACOPF_E_INVALID_ARG;
      }
    }
    std::vector<int32_t> wpos(static_cast<size_t>(ns), -1);
    for (int32_t k = 0; k < nw; ++k) wpos[size_t(plan.forward_warp.task[4 * size_t(k) + 1])] = k;
    // --- the factorization's tasks -------------------------------------------
    Builder B;
    std::vector<std::vector<int32_t>> deps, xdeps;  // xdeps: warp tasks (wpos)
    auto xd = [&](int32_t t) -> std::vector<int32_t>& {  // task t's warp tasks
      if (int32_t(xdeps.size()) <= t) xdeps.resize(size_t(t) + 1);
      return xdeps[size_t(t)];
    };
    std::vector<int32_t> comp(static_cast<size_t>(ns), -1);
    // a tiled supernode's completion: the last writers of its update
    // matrix's tiles (its parent's tasks wait for them directly: no join task)
    std::vector<std::vector<int32_t>> comp_tiles(static_cast<size_t>(ns));
    std::vector<int32_t> grp_task(static_cast<size_t>(ng));
    for (int32_t g = 0; g < ng; ++g) {
      grp_task[size_t(g)] = B.add(kTaskGroup, g, 0, 0, grp_us[size_t(g)]);
      deps.emplace_back();
    }
    for (int32_t s = 0; s < ns; ++s)
      if (grp[size_t(s)] >= 0) comp[size_t(s)] = grp_task[size_t(grp[size_t(s)])];
    auto child_comps = [&](int32_t s, std::vector<int32_t>& out) {  // bottom: done before
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
        const int32_t k = sy.kid[size_t(q)];
        if (comp[size_t(k)] >= 0) out.push_back(comp[size_t(k)]);
        out.insert(out.end(), comp_tiles[size_t(k)].begin(), comp_tiles[size_t(k)].end());
      }
    };
    auto child_warps = [&](int32_t s, std::vector<int32_t>& out) {
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q)
        if (wpos[size_t(sy.kid[size_t(q)])] >= 0) out.push_back(wpos[size_t(sy.kid[size_t(q)])]);
    };
    const double ut = double(T) * T * T;
    plan.brk_off.assign(static_cast<size_t>(ns), 0);
    plan.tile_brk.assign(1, 0);
    for (int32_t s = 0; s < ns; ++s) {
      const int8_t cls = plan.sn_class[size_t(s)];
      if (cls == kSnSmall || cls == kSnBottom) continue;
      if (cls == kSnBlock) {
        comp[size_t(s)] = B.add(kTaskBlock, s, 0, 0, 3.0 + cost[size_t(s)] / 2000.0);
        deps.emplace_back();
        child_comps(s, deps.back());
        child_warps(s, xd(comp[size_t(s)]));
        continue;
      }
      const int32_t w = W[size_t(s)], m = H[size_t(s)] - w;
      const int32_t nbp = (w + T - 1) / T, nb = nbp + (m + T - 1) / T;
      const bool has_kids = sy.kid_ptr[size_t(s) + 1] > sy.kid_ptr[size_t(s)];
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
        const int32_t c = sy.kid[size_t(q)], mc = H[size_t(c)] - W[size_t(c)];
        const int32_t* rel = sy.relmap.data() + sy.rel_off[size_t(c)];
        plan.brk_off[size_t(c)] = int32_t(plan.tile_brk.size());
        for (int32_t I = 0; I <= nb; ++I) {
          const int32_t start = I < nbp ? I * T : (I < nb ? w + (I - nbp) * T : w + m);
          plan.tile_brk.push_back(int32_t(std::lower_bound(rel, rel + mc, start) - rel));
        }
      }
      std::vector<int32_t> last(size_t(nb) * size_t(nb), -1);
      auto L = [&](int32_t i, int32_t j) -> int32_t& { return last[size_t(i) * size_t(nb) + size_t(j)]; };
      std::vector<int32_t> kc, kw;
      child_comps(s, kc);
      child_warps(s, kw);
      if (has_kids)
        for (int32_t i = 0; i < nb; ++i)
          for (int32_t j = 0; j <= i; ++j) {
            L(i, j) = B.add(kTaskAsm, s, i, j, 2.0);
            deps.push_back(kc);
            xd(L(i, j)) = kw;
          }
      std::vector<int32_t> trsm(static_cast<size_t>(nb), -1);
      for (int32_t k = 0; k < nbp; ++k) {
        const int32_t pk = B.add(kTaskPotrf | (k << 8), s, k, k, 3.0 + ut / 6.0 / 1000.0);
        deps.emplace_back();
        if (L(k, k) >= 0) deps.back().push_back(L(k, k));
        L(k, k) = pk;
        for (int32_t i = k + 1; i < nb; ++i) {
          trsm[size_t(i)] = B.add(kTaskTrsm | (k << 8), s, i, k, 2.5 + ut / 2.0 / 2000.0);
          deps.emplace_back();
          deps.back().push_back(pk);
          if (L(i, k) >= 0) deps.back().push_back(L(i, k));
          L(i, k) = trsm[size_t(i)];
        }
        for (int32_t j = k + 1; j < nb; ++j)
          for (int32_t i = j; i < nb; ++i) {
            const int32_t u =
                B.add(kTaskUpd | (k << 8), s, i, j, 2.0 + (i == j ? ut / 2.0 : ut) / 2000.0);
            deps.emplace_back();
            deps.back().push_back(trsm[size_t(i)]);
            if (j != i) deps.back().push_back(trsm[size_t(j)]);
            if (L(i, j) >= 0) deps.back().push_back(L(i, j));
            L(i, j) = u;
          }
      }
      std::vector<int32_t>& ct = comp_tiles[size_t(s)];
      if (nb > nbp) {
        for (int32_t i = nbp; i < nb; ++i)
          for (int32_t j = nbp; j <= i; ++j) ct.push_back(L(i, j));
      } else {
        ct.push_back(L(nbp - 1, nbp - 1));
      }
    }
    for (int32_t g = 0; g < ng; ++g) {
      std::vector<int32_t>& d = deps[size_t(grp_task[size_t(g)])];
      for (int32_t p = plan.grp_ptr[size_t(g)]; p < plan.grp_ptr[size_t(g) + 1]; ++p) {
        const int32_t s = plan.grp_sn[size_t(p)];
        for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
          const int32_t k = sy.kid[size_t(q)];
          if (grp[size_t(k)] != g && comp[size_t(k)] >= 0) d.push_back(comp[size_t(k)]);
          d.insert(d.end(), comp_tiles[size_t(k)].begin(), comp_tiles[size_t(k)].end());
        }
        child_warps(s, xd(grp_task[size_t(g)]));
      }
    }
    xdeps.resize(deps.size());
    schedule(B.task, deps, B.dur, prm.workers, plan.factor, &plan.est_factor_us,
             &plan.est_critical_us, plan.est_critical_by_kind, &xdeps);
    // --- the solves -------------------------------------------------------------
    // Warp tasks: the warp-small supernodes, one task each, in ascending
    // (forward) or descending (backward) order; the rest are block tasks, run
    // after the warp tasks in the forward solve and before them in the
    // backward solve.
    Builder F;
    std::vector<int32_t> fcomp(static_cast<size_t>(ns), -1);
    for (int32_t s = 0; s < ns; ++s)
      if (plan.sn_class[size_t(s)] != kSnBottom && !wsmall[size_t(s)])
        fcomp[size_t(s)] = F.add(kTaskBlock, s, 0, 0,
                                 2.0 + double(H[size_t(s)]) * W[size_t(s)] / 2000.0);
    std::vector<std::vector<int32_t>> fdeps(F.dur.size()), bdeps(F.dur.size()),
        fxdeps(F.dur.size());
    for (int32_t s = 0; s < ns; ++s) {
      if (fcomp[size_t(s)] >= 0) child_warps(s, fxdeps[size_t(fcomp[size_t(s)])]);
      const int32_t p = sy.sn_parent[size_t(s)];
      if (p < 0 || fcomp[size_t(s)] < 0) continue;
      // s's task needs s's children (forward); s's task needs its parent's (backward)
      fdeps[size_t(fcomp[size_t(p)])].push_back(fcomp[size_t(s)]);
      bdeps[size_t(fcomp[size_t(s)])].push_back(fcomp[size_t(p)]);
    }
    // the forward block tasks also wait for their warp-small children's warp
    // tasks (forward_warp positions): the block kernel may start while the
    // warp kernel runs
    schedule(F.task, fdeps, F.dur, prm.workers, plan.forward, nullptr, nullptr, nullptr, &fxdeps);
    schedule(F.task, bdeps, F.dur, prm.workers, plan.backward, nullptr, nullptr);
    // the backward warp tasks whose parent is a block task wait for it
    // (backward positions): the warp kernel may start while the block kernel runs
    {
      std::vector<int32_t> bpos(static_cast<size_t>(ns), -1);
      for (int32_t k = 0; k < plan.backward.n_tasks(); ++k)
        bpos[size_t(plan.backward.task[4 * size_t(k) + 1])] = k;
      CholGraph& bw = plan.backward_warp;
      bw.xdep_ptr.assign(size_t(bw.n_tasks()) + 1, 0);
      bw.xdep.clear();
      for (int32_t k = 0; k < bw.n_tasks(); ++k) {
        const int32_t p = sy.sn_parent[size_t(bw.task[4 * size_t(k) + 1])];
        if (p >= 0 && !wsmall[size_t(p)]) {
          if (bpos[size_t(p)] < 0) {
            err = "task plan: a warp-small supernode's parent has no solve task";
            return ACOPF_E_INVALID_ARG;
          }
          bw.xdep.push_back(bpos[size_t(p)]);
        }
        bw.xdep_ptr[size_t(k) + 1] = int32_t(bw.xdep.size());
      }
    }
    // --- forward-solve gather lists: counts per row slot, then the entries
    // child by child (so each slot's list is in child order) --------------
    if (sy.z_off[size_t(ns)] > int64_t(INT32_MAX)) {
      err = "task plan: the update vectors exceed 2^31 entries";
      return ACOPF_E_INVALID_ARG;
    }
    const size_t slots = sy.rowidx.size();
    plan.fg_ptr.assign(slots + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<int32_t> fill;
      if (pass == 1) {
        for (size_t j = 0; j < slots; ++j) plan.fg_ptr[j + 1] += plan.fg_ptr[j];
        plan.fg_idx.assign(size_t(plan.fg_ptr[slots]), 0);
        fill.assign(plan.fg_ptr.begin(), plan.fg_ptr.end() - 1);
      }
      for (int32_t t = 0; t < ns; ++t) {
        const size_t r0 = size_t(sy.sn_rowptr[size_t(t)]);
        for (int32_t q = sy.kid_ptr[size_t(t)]; q < sy.kid_ptr[size_t(t) + 1]; ++q) {
          const int32_t c = sy.kid[size_t(q)];
          const int32_t mc = H[size_t(c)] - W[size_t(c)];
          const int32_t* rel = sy.relmap.data() + sy.rel_off[size_t(c)];
          for (int32_t i = 0; i < mc; ++i) {
            const size_t j = r0 + size_t(rel[i]);
            if (pass == 0)
              ++plan.fg_ptr[j + 1];
            else
              plan.fg_idx[size_t(fill[j]++)] = int32_t(sy.z_off[size_t(c)] + i);
          }
        }
      }
    }
  } catch (const std::bad_alloc&) {
    err = "host allocation failed";
    return ACOPF_E_OOM;
  }
  return ACOPF_OK;
}

}  // namespace acopf
