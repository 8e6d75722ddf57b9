// Sparse Cholesky factorization of M_cond (acopf_chol_*): the consumer of
// the condensed KKT matrix.  Sec. IV.C: M_aug has the inertia (n + m, 0, m)
// exactly when M_cond is positive definite, so a Cholesky factorization that
// meets a non-positive pivot is the inertia test, and the regularization
// (delta_w, delta_c) is raised until it succeeds.  Sec. V factorizes with a
// fill-reducing order fixed once per pattern and refactors numerically every
// iteration.
//
// Here: the symbolic phase (symbolic.cpp) and the task graphs (chol_plan.cpp)
// are built on the host once per chol object; the numeric factorization
// (multifrontal), its pivot test and the solves are the persistent task
// kernels of chol.cu: one launch for the factorization, one per direction of
// a solve.
#include <algorithm>
#include <climits>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "chol_internal.h"
#include "chol_plan.h"
#include "host_internal.h"
#include "symbolic.h"

static_assert(acopf::kMaxSupernodeWidth == acopf::kCholMaxWidth,
              "the solves stage a supernode's diagonal block in shared memory");
static_assert(acopf::kCholBottomRows * acopf::kCholBottomCols +
                      (acopf::kCholBottomRows - acopf::kCholBottomCols) *
                          (acopf::kCholBottomRows - acopf::kCholBottomCols + 1) / 2 <=
                  acopf::kCholBottomStage,
              "a bottom supernode's staging fits the kernel's bound");
static_assert(acopf::kMaxRowsBelow == acopf::kCholMaxRelRows &&
                  acopf::kCholBlockStage == acopf::kCholBlockDoubles &&
                  acopf::kCholBlockMaxRows == acopf::kCholBlockRows &&
                  acopf::kCholTileEdge == acopf::kCholTile,
              "the plan and the kernels agree on what a task stages");

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

struct acopf_chol {
  acopf_model* model = nullptr;
  int32_t n = 0;
  int64_t nnz_low = 0;
  acopf_chol_stats stats{};
  std::vector<int32_t> perm_host, bot_ptr, bot_stage;  // the bottom levels (chol_plan.h)
  const int32_t* bot_sn = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  acopf::CholDev dev{};
  // the task graphs: factorization (block tasks), forward warp tasks,
  // forward block tasks, backward block tasks, backward warp tasks, the
  // factorization's warp tasks (the forward warp list with flags of its
  // own); flags and counters in the order 0, 5, 1, 2, 3, 4, the four of the
  // solves adjacent
  acopf::CholTasks tg[6] = {};
  int32_t* flags = nullptr;             // the graphs' done flags and counters
  size_t flag_ints = 0;
  // persistent blocks of the task kernels
  int blocks = 0, warp_blocks = 0;
  int fwd_blocks = 0, fwd_warp_blocks = 0, bwd_blocks = 0, bwd_warp_blocks = 0;  // the solves
  const int64_t* amap = nullptr;
  const int32_t* perm = nullptr;
  double* work = nullptr;       // n: the permuted right-hand side / solution
  size_t u_doubles = 0, z_doubles = 0;  // update matrices / vectors
  int32_t* status_host = nullptr;       // page-locked copy of {bad, abort}
  long long* trace = nullptr;           // task trace of the graphs (NULL: off)
  bool factored = false;
  // the factorization's and the solve's launch sequences, captured as CUDA
  // graphs for the last arguments they ran with
  cudaGraphExec_t factor_exec = nullptr, solve_exec = nullptr;
  const void* factor_key = nullptr;
  double factor_tol = -1.0;
  const void *solve_b = nullptr, *solve_x = nullptr;
};

namespace {

// Blocks per SM of the solves' block-task and warp-task kernels.  Backward,
// the warp kernel starts under the block kernel and they run side by side
// (one block-task block and three warp-task blocks fit an SM's registers
// together); forward, the warp kernel fills the GPU (the block tasks' first
// inputs come late in the warp phase, so sharing SMs measured slower).
constexpr int kFwdBlocksPerSm = 2, kFwdWarpBlocksPerSm = 4;
constexpr int kBwdBlocksPerSm = 1, kBwdWarpBlocksPerSm = 3;

void release(acopf_chol* c) {
  if (c->factor_exec) cudaGraphExecDestroy(c->factor_exec);
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  if (c->arena) cudaFree(c->arena);
  if (c->trace) cudaFree(c->trace);
  if (c->status_host) cudaFreeHost(c->status_host);
  delete c;
}

acopf_status check_model(const acopf_model* model, const char* where) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": null model");
  const acopf::HostModel& hm = model->hm;
  const int32_t n = hm.L.n;
  for (int32_t i = 0; i < n; ++i) {
    const int32_t a = hm.krowptr[size_t(i)], b = hm.krowptr[size_t(i) + 1];
    if (a == b || hm.kcolind[size_t(b) - 1] != i)
      return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": M_cond pattern lacks a diagonal");
  }
  return ACOPF_OK;
}

// The plan's counts: tasks of the factorization, and the launches of one
// factorization (assembly, the bottom levels, the task kernel) and of one
// solve (permutation, bottom levels, warp and block tasks per direction,
// bottom levels, permutation back).
void plan_stats(const acopf::CholPlan& plan, acopf_chol_stats& st) {
  const int64_t nbl = int64_t(plan.bot_ptr.size()) - 1;
  st.factor_tasks = plan.factor.n_tasks() + plan.forward_warp.n_tasks();
  st.factor_launches = 3 + nbl;
  st.solve_launches = 6 + 2 * nbl;
}

acopf_status run_symbolic(const acopf_model* model, acopf::CholSymbolic& sy, const char* where) {
  std::string err;
  const acopf_status st =
      acopf::chol_symbolic(model->hm.L.n, model->hm.krowptr, model->hm.kcolind, sy, err);
  if (st != ACOPF_OK) return fail(st, std::string(where) + ": " + err);
  return ACOPF_OK;
}

// The factorization's device work: zeroed blocks, update matrices, flags
// and counters, the pivot marker, the assembly of M_cond's values, the
// bottom levels, the warp tasks, then the block-task kernel.
cudaError_t record_factor(const acopf_chol* chol, const double* kvals, double tol,
                          cudaStream_t s) {
  const acopf::CholDev& d = chol->dev;
  cudaError_t e = cudaMemsetAsync(d.Lx, 0, size_t(chol->stats.storage) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.Ux, 0, chol->u_doubles * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.bad, 0x7f, sizeof(int32_t), s);  // 0x7f7f7f7f: none
  if (e == cudaSuccess)  // graphs 0 and 5: adjacent
    e = cudaMemsetAsync(chol->tg[0].done, 0,
                        (size_t(chol->tg[0].n) + size_t(chol->tg[5].n) + 2) * sizeof(int32_t), s);
  if (e == cudaSuccess) e = acopf::launch_chol_assemble(d.Lx, chol->amap, kvals, chol->nnz_low, s);
  const std::vector<int32_t>& bp = chol->bot_ptr;
  for (size_t v = 0; e == cudaSuccess && v + 1 < bp.size(); ++v)
    e = acopf::launch_chol_bottom(d, chol->bot_sn + bp[v], bp[v + 1] - bp[v], chol->bot_stage[v],
                                  tol, s);
  if (e == cudaSuccess)
    e = acopf::launch_chol_factor_warps(d, chol->tg[5], tol, chol->warp_blocks, s);
  if (e == cudaSuccess)
    e = acopf::launch_chol_factor_tasks(d, chol->tg[0], tol, chol->blocks, chol->tg[5].n > 0, s);
  return e;
}

// The solve's device work: permutation, forward tasks, backward tasks,
// permutation back.
cudaError_t record_solve(const acopf_chol* chol, const double* b, double* x, cudaStream_t s) {
  const acopf::CholDev& d = chol->dev;
  cudaError_t e = acopf::launch_gather(chol->work, b, chol->perm, chol->n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.Zx, 0, chol->z_doubles * sizeof(double), s);
  if (e == cudaSuccess) {  // the solve graphs' flags and counters are adjacent
    size_t words = 0;
    for (int k = 1; k < 5; ++k) words += size_t(chol->tg[k].n) + 1;
    e = cudaMemsetAsync(chol->tg[1].done, 0, words * sizeof(int32_t), s);
  }
  const std::vector<int32_t>& bp = chol->bot_ptr;
  for (size_t v = 0; e == cudaSuccess && v + 1 < bp.size(); ++v)
    e = acopf::launch_chol_bottom_fwd(d, chol->bot_sn + bp[v], bp[v + 1] - bp[v], chol->work, s);
  if (e == cudaSuccess)
    e = acopf::launch_chol_solve_warps(d, chol->tg[1], chol->work, true, chol->fwd_warp_blocks,
                                       false, s);
  if (e == cudaSuccess)  // under the warp tasks, waiting for their flags
    e = acopf::launch_chol_forward_tasks(d, chol->tg[2], chol->work, chol->fwd_blocks,
                                         chol->tg[1].n > 0, s);
  if (e == cudaSuccess)
    e = acopf::launch_chol_backward_tasks(d, chol->tg[3], chol->work, chol->bwd_blocks, s);
  if (e == cudaSuccess)  // under the block tasks, waiting for their flags
    e = acopf::launch_chol_solve_warps(d, chol->tg[4], chol->work, false, chol->bwd_warp_blocks,
                                       chol->tg[3].n > 0, s);
  for (size_t v = bp.size() - 1; e == cudaSuccess && v > 0; --v)
    e = acopf::launch_chol_bottom_bwd(d, chol->bot_sn + bp[v - 1], bp[v] - bp[v - 1], chol->work, s);
  if (e == cudaSuccess) e = acopf::launch_scatter(x, chol->work, chol->perm, chol->n, s);
  return e;
}

// Runs `record` on `s`: through a CUDA graph captured for the current
// arguments (re-captured when they change), or directly on the legacy
// default stream, which cannot be captured, and on a stream the caller is
// capturing (the launches then become part of the caller's graph).
template <typename Record>
cudaError_t run_recorded(cudaGraphExec_t& exec, bool reuse, cudaStream_t s, Record record) {
  if (s == nullptr || s == cudaStreamLegacy) return record(s);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t qe = cudaStreamIsCapturing(s, &cap);
  if (qe != cudaSuccess) return qe;
  if (cap != cudaStreamCaptureStatusNone) return record(s);
  if (!(reuse && exec)) {
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t er = record(s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (er != cudaSuccess) e = er;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      exec = nullptr;
      return e;
    }
  }
  return cudaGraphLaunch(exec, s);
}

}  // namespace

namespace acopf {
acopf_model* chol_model(const acopf_chol* c) { return c->model; }
}  // namespace acopf

extern "C" {

acopf_status acopf_chol_analyze(acopf_model* model, acopf_chol_stats* stats,
                                int32_t* perm) {
  if (!stats) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_analyze: null output pointer");
  acopf_status st = check_model(model, "acopf_chol_analyze");
  if (st != ACOPF_OK) return st;
  acopf::CholSymbolic sy;
  st = run_symbolic(model, sy, "acopf_chol_analyze");
  if (st != ACOPF_OK) return st;
  acopf::CholPlan plan;
  {
    std::string err;
    st = acopf::chol_plan(sy, acopf::CholPlanParams{}, plan, err);
    if (st != ACOPF_OK) return fail(st, "acopf_chol_analyze: " + err);
  }
  plan_stats(plan, sy.stats);
  *stats = sy.stats;
  if (perm) std::copy(sy.perm.begin(), sy.perm.end(), perm);
  return ACOPF_OK;
}

acopf_status acopf_chol_create(acopf_model* model, acopf_chol** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_create: null output pointer");
  *out = nullptr;
  acopf_status st = check_model(model, "acopf_chol_create");
  if (st != ACOPF_OK) return st;
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "acopf_chol_create: host-only model");
  acopf::CholSymbolic sy;
  st = run_symbolic(model, sy, "acopf_chol_create");
  if (st != ACOPF_OK) return st;
  acopf::CholPlan plan;
  {
    std::string err;
    st = acopf::chol_plan(sy, acopf::CholPlanParams{}, plan, err);
    if (st != ACOPF_OK) return fail(st, "acopf_chol_create: " + err);
  }
  acopf_chol* c = new (std::nothrow) acopf_chol;
  if (!c) return fail(ACOPF_E_OOM, "host allocation failed");
  c->model = model;
  c->n = sy.n;
  c->nnz_low = int64_t(sy.amap.size());
  c->stats = sy.stats;
  plan_stats(plan, c->stats);
  try {
    c->perm_host = sy.perm;
    c->bot_ptr = plan.bot_ptr;
    c->bot_stage = plan.bot_stage;
  } catch (const std::bad_alloc&) {
    release(c);
    return fail(ACOPF_E_OOM, "host allocation failed");
  }
  const size_t ns = size_t(sy.ns), n = size_t(sy.n), ng = plan.grp_ptr.size() - 1;
  const acopf::CholGraph* graphs[5] = {&plan.factor, &plan.forward_warp, &plan.forward,
                                       &plan.backward, &plan.backward_warp};
  acopf::ArenaPlan p;
  const size_t o_first = p.take<int32_t>(ns + 1), o_rowptr = p.take<int32_t>(ns + 1);
  const size_t o_rowidx = p.take<int32_t>(sy.rowidx.size()), o_off = p.take<int64_t>(ns + 1);
  const size_t o_kptr = p.take<int32_t>(ns + 1), o_kid = p.take<int32_t>(sy.kid.size());
  const size_t o_roff = p.take<int32_t>(ns), o_rel = p.take<int32_t>(sy.relmap.size());
  const size_t o_uoff = p.take<int64_t>(ns + 1), o_zoff = p.take<int64_t>(ns + 1);
  const size_t o_gptr = p.take<int32_t>(ng + 1), o_gsn = p.take<int32_t>(plan.grp_sn.size());
  const size_t o_glp = p.take<int32_t>(ng + 1), o_glev = p.take<int32_t>(plan.grp_lev.size());
  const size_t o_bot = p.take<int32_t>(plan.bot_sn.size() + 1);
  const size_t o_boff = p.take<int32_t>(ns), o_brk = p.take<int32_t>(plan.tile_brk.size());
  const size_t o_fgp = p.take<int32_t>(plan.fg_ptr.size()), o_fgi = p.take<int32_t>(plan.fg_idx.size());
  const size_t o_kd = p.take<int32_t>(4 * sy.kid.size()), o_kb = p.take<int32_t>(sy.kid.size());
  size_t o_task[5], o_dptr[5], o_dep[5], o_xptr[5], o_xdep[5];
  for (int k = 0; k < 5; ++k) {
    o_task[k] = p.take<int32_t>(graphs[k]->task.size());
    o_dptr[k] = p.take<int32_t>(graphs[k]->dep_ptr.size());
    o_dep[k] = p.take<int32_t>(graphs[k]->dep.size() + 1);
    o_xptr[k] = p.take<int32_t>(graphs[k]->xdep_ptr.size());
    o_xdep[k] = p.take<int32_t>(graphs[k]->xdep.size() + 1);
  }
  // done flags and counters: per graph [its n flags, its counter]
  c->flag_ints = size_t(plan.forward_warp.n_tasks()) + 1;  // graph 5
  for (int k = 0; k < 5; ++k) c->flag_ints += size_t(graphs[k]->n_tasks()) + 1;
  const size_t o_flags = p.take<int32_t>(c->flag_ints);
  const size_t o_amap = p.take<int64_t>(sy.amap.size()), o_perm = p.take<int32_t>(n);
  const size_t o_work = p.take<double>(n), o_status = p.take<int32_t>(2);
  const size_t o_dinv = p.take<double>(n);
  const size_t o_lx = p.take<double>(size_t(sy.stats.storage));
  const size_t o_ux = p.take<double>(size_t(sy.u_off[ns]) + 1);
  const size_t o_zx = p.take<double>(size_t(sy.z_off[ns]) + 1);
  c->u_doubles = size_t(sy.u_off[ns]);
  c->z_doubles = size_t(sy.z_off[ns]);
  DeviceScope ds(model->device);
  cudaError_t e = ds.error();
  if (e == cudaSuccess) e = cudaMalloc(&c->arena, p.off);
  if (e != cudaSuccess) {
    c->arena = nullptr;
    release(c);
    return cuda_fail(e, "acopf_chol_create");
  }
  c->arena_bytes = p.off;
  char* base = static_cast<char*>(c->arena);
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice);
  };
  up(o_first, sy.sn_first.data(), (ns + 1) * 4);
  up(o_rowptr, sy.sn_rowptr.data(), (ns + 1) * 4);
  up(o_rowidx, sy.rowidx.data(), sy.rowidx.size() * 4);
  up(o_off, sy.sn_off.data(), (ns + 1) * 8);
  up(o_kptr, sy.kid_ptr.data(), (ns + 1) * 4);
  up(o_kid, sy.kid.data(), sy.kid.size() * 4);
  up(o_roff, sy.rel_off.data(), ns * 4);
  up(o_rel, sy.relmap.data(), sy.relmap.size() * 4);
  up(o_uoff, sy.u_off.data(), (ns + 1) * 8);
  up(o_zoff, sy.z_off.data(), (ns + 1) * 8);
  up(o_gptr, plan.grp_ptr.data(), (ng + 1) * 4);
  up(o_gsn, plan.grp_sn.data(), plan.grp_sn.size() * 4);
  up(o_glp, plan.grp_lptr.data(), (ng + 1) * 4);
  up(o_glev, plan.grp_lev.data(), plan.grp_lev.size() * 4);
  up(o_bot, plan.bot_sn.data(), plan.bot_sn.size() * 4);
  up(o_boff, plan.brk_off.data(), ns * 4);
  up(o_brk, plan.tile_brk.data(), plan.tile_brk.size() * 4);
  up(o_fgp, plan.fg_ptr.data(), plan.fg_ptr.size() * 4);
  up(o_fgi, plan.fg_idx.data(), plan.fg_idx.size() * 4);
  {  // children's descriptors for the extend-add
    std::vector<int32_t> kd;
    try {
      kd.resize(4 * sy.kid.size());
    } catch (const std::bad_alloc&) {
      release(c);
      return fail(ACOPF_E_OOM, "host allocation failed");
    }
    for (size_t q = 0; q < sy.kid.size(); ++q) {
      const size_t k = size_t(sy.kid[q]);
      const int64_t uo = sy.u_off[k];
      kd[4 * q] = (sy.sn_rowptr[k + 1] - sy.sn_rowptr[k]) - (sy.sn_first[k + 1] - sy.sn_first[k]);
      kd[4 * q + 1] = sy.rel_off[k];
      kd[4 * q + 2] = int32_t(uint32_t(uint64_t(uo) & 0xffffffffu));
      kd[4 * q + 3] = int32_t(uint32_t(uint64_t(uo) >> 32));
    }
    up(o_kd, kd.data(), kd.size() * 4);
    for (size_t q = 0; q < sy.kid.size(); ++q) kd[q] = plan.brk_off[size_t(sy.kid[q])];
    up(o_kb, kd.data(), sy.kid.size() * 4);
  }
  for (int k = 0; k < 5; ++k) {
    up(o_task[k], graphs[k]->task.data(), graphs[k]->task.size() * 4);
    up(o_dptr[k], graphs[k]->dep_ptr.data(), graphs[k]->dep_ptr.size() * 4);
    up(o_dep[k], graphs[k]->dep.data(), graphs[k]->dep.size() * 4);
    up(o_xptr[k], graphs[k]->xdep_ptr.data(), graphs[k]->xdep_ptr.size() * 4);
    up(o_xdep[k], graphs[k]->xdep.data(), graphs[k]->xdep.size() * 4);
  }
  up(o_amap, sy.amap.data(), sy.amap.size() * 8);
  up(o_perm, sy.perm.data(), n * 4);
  if (e == cudaSuccess) e = cudaMemset(base + o_status, 0, 2 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&c->status_host, 2 * sizeof(int32_t));
  int per_sm = 0, warp_per_sm = 0, sms = 0;
  if (e == cudaSuccess) e = acopf::chol_task_setup(&per_sm, &warp_per_sm);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, model->device);
  if (e != cudaSuccess) {
    release(c);
    return cuda_fail(e, "acopf_chol_create: upload");
  }
  c->blocks = per_sm * sms;
  c->warp_blocks = warp_per_sm * sms;
  c->fwd_blocks = kFwdBlocksPerSm * sms;
  c->fwd_warp_blocks = kFwdWarpBlocksPerSm * sms;
  c->bwd_blocks = kBwdBlocksPerSm * sms;
  c->bwd_warp_blocks = kBwdWarpBlocksPerSm * sms;
  acopf::CholDev& d = c->dev;
  d.n = sy.n;
  d.sn_first = reinterpret_cast<const int32_t*>(base + o_first);
  d.sn_rowptr = reinterpret_cast<const int32_t*>(base + o_rowptr);
  d.rowidx = reinterpret_cast<const int32_t*>(base + o_rowidx);
  d.sn_off = reinterpret_cast<const int64_t*>(base + o_off);
  d.kid_ptr = reinterpret_cast<const int32_t*>(base + o_kptr);
  d.kid = reinterpret_cast<const int32_t*>(base + o_kid);
  d.rel_off = reinterpret_cast<const int32_t*>(base + o_roff);
  d.relmap = reinterpret_cast<const int32_t*>(base + o_rel);
  d.u_off = reinterpret_cast<const int64_t*>(base + o_uoff);
  d.z_off = reinterpret_cast<const int64_t*>(base + o_zoff);
  d.grp_ptr = reinterpret_cast<const int32_t*>(base + o_gptr);
  d.grp_sn = reinterpret_cast<const int32_t*>(base + o_gsn);
  d.grp_lptr = reinterpret_cast<const int32_t*>(base + o_glp);
  d.grp_lev = reinterpret_cast<const int32_t*>(base + o_glev);
  d.brk_off = reinterpret_cast<const int32_t*>(base + o_boff);
  d.tile_brk = reinterpret_cast<const int32_t*>(base + o_brk);
  d.kid_desc = reinterpret_cast<const int4*>(base + o_kd);
  d.kid_brk = reinterpret_cast<const int32_t*>(base + o_kb);
  d.fg_ptr = reinterpret_cast<const int32_t*>(base + o_fgp);
  d.fg_idx = reinterpret_cast<const int32_t*>(base + o_fgi);
  d.Lx = reinterpret_cast<double*>(base + o_lx);
  d.Ux = reinterpret_cast<double*>(base + o_ux);
  d.Zx = reinterpret_cast<double*>(base + o_zx);
  d.Dinv = reinterpret_cast<double*>(base + o_dinv);
  d.bad = reinterpret_cast<int32_t*>(base + o_status);
  d.abort = d.bad + 1;
  c->flags = reinterpret_cast<int32_t*>(base + o_flags);
  int32_t* fl = c->flags;
  for (const int k : {0, 5, 1, 2, 3, 4}) {
    acopf::CholTasks& t = c->tg[k];
    const int src = k == 5 ? 1 : k;  // graph 5 runs graph 1's list
    t.task = reinterpret_cast<const int4*>(base + o_task[src]);
    t.dep_ptr = reinterpret_cast<const int32_t*>(base + o_dptr[src]);
    t.dep = reinterpret_cast<const int32_t*>(base + o_dep[src]);
    t.n = graphs[src]->n_tasks();
    t.done = fl;
    t.next = fl + t.n;
    fl += t.n + 1;
  }
  // tasks that wait for the graph launched before theirs: the
  // factorization's block tasks for its warp tasks, the forward solve's
  // block tasks for its warp tasks, the backward solve's warp tasks for its
  // block tasks
  const int xsrc[3][3] = {{0, 0, 5}, {2, 2, 1}, {4, 4, 3}};  // {tg, graph, tg waited for}
  for (const auto& x : xsrc) {
    if (graphs[x[1]]->xdep_ptr.empty()) continue;
    c->tg[x[0]].xdep_ptr = reinterpret_cast<const int32_t*>(base + o_xptr[x[1]]);
    c->tg[x[0]].xdep = reinterpret_cast<const int32_t*>(base + o_xdep[x[1]]);
    c->tg[x[0]].xdone = c->tg[x[2]].done;
  }
  c->bot_sn = reinterpret_cast<const int32_t*>(base + o_bot);
  c->amap = reinterpret_cast<const int64_t*>(base + o_amap);
  c->perm = reinterpret_cast<const int32_t*>(base + o_perm);
  c->work = reinterpret_cast<double*>(base + o_work);
  *out = c;
  return ACOPF_OK;
}

acopf_status acopf_chol_destroy(acopf_chol* chol) {
  if (!chol) return ACOPF_OK;
  DeviceScope ds(chol->model->device);
  cudaDeviceSynchronize();
  release(chol);
  return ACOPF_OK;
}

acopf_status acopf_chol_factor(acopf_chol* chol, const double* kvals, double pivot_tol,
                               int32_t* first_bad_pivot, acopf_stream stream) {
  if (!chol || !kvals || !first_bad_pivot)
    return fail(ACOPF_E_INVALID_ARG, "acopf_chol_factor: null pointer");
  if (!(pivot_tol >= 0.0) || !std::isfinite(pivot_tol))
    return fail(ACOPF_E_INVALID_ARG, "acopf_chol_factor: pivot_tol must be finite and >= 0");
  DeviceScope ds(chol->model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_chol_factor");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  chol->factored = false;
  const acopf::CholDev& d = chol->dev;
  const bool reuse = chol->factor_key == kvals && chol->factor_tol == pivot_tol;
  cudaError_t e = run_recorded(chol->factor_exec, reuse, s, [&](cudaStream_t st) {
    return record_factor(chol, kvals, pivot_tol, st);
  });
  chol->factor_key = chol->factor_exec ? kvals : nullptr;
  chol->factor_tol = pivot_tol;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(chol->status_host, d.bad, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_factor");
  if (chol->status_host[1] != 0)
    return fail(ACOPF_E_TIMEOUT,
                "acopf_chol_factor: a task of the factorization or of an earlier solve waited "
                "past its limit; the object is unusable");
  const int32_t bad = chol->status_host[0];
  *first_bad_pivot = bad < chol->n ? bad : -1;
  chol->factored = bad >= chol->n;
  return ACOPF_OK;
}

acopf_status acopf_chol_solve(acopf_chol* chol, const double* b, double* x, acopf_stream stream) {
  if (!chol || !b || !x) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_solve: null pointer");
  if (!chol->factored)
    return fail(ACOPF_E_INVALID_ARG,
                "acopf_chol_solve: no positive definite factorization to solve with");
  DeviceScope ds(chol->model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_chol_solve");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool reuse = chol->solve_b == b && chol->solve_x == x;
  const cudaError_t e = run_recorded(chol->solve_exec, reuse, s, [&](cudaStream_t st) {
    return record_solve(chol, b, x, st);
  });
  chol->solve_b = chol->solve_exec ? b : nullptr;
  chol->solve_x = chol->solve_exec ? x : nullptr;
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_solve");
  return ACOPF_OK;
}

acopf_status acopf_chol_info(const acopf_chol* chol, acopf_chol_stats* stats,
                             int64_t* device_bytes) {
  if (!chol) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_info: null pointer");
  if (stats) *stats = chol->stats;
  if (device_bytes) *device_bytes = int64_t(chol->arena_bytes);
  return ACOPF_OK;
}

acopf_status acopf_chol_set_trace(acopf_chol* chol, int32_t enable) {
  if (!chol) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_set_trace: null pointer");
  DeviceScope ds(chol->model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_chol_set_trace");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_set_trace");
  acopf::CholTasks* tk[6] = {&chol->tg[0], &chol->tg[1], &chol->tg[2],
                             &chol->tg[3], &chol->tg[4], &chol->tg[5]};
  if (chol->trace) {
    cudaFree(chol->trace);
    chol->trace = nullptr;
  }
  if (enable) {
    size_t words = 0;
    for (auto* t : tk) words += 6 * size_t(t->n);
    e = cudaMalloc(&chol->trace, words * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(chol->trace, 0, words * sizeof(long long));
    if (e != cudaSuccess) {
      if (chol->trace) cudaFree(chol->trace);
      chol->trace = nullptr;
      for (auto* t : tk) t->trace = nullptr;
      return fail(ACOPF_E_OOM, "acopf_chol_set_trace: trace buffer");
    }
  }
  long long* p = chol->trace;
  for (auto* t : tk) {
    t->trace = p;
    if (p) p += 6 * size_t(t->n);
  }
  // the captured graphs hold the old kernel arguments
  if (chol->factor_exec) cudaGraphExecDestroy(chol->factor_exec);
  if (chol->solve_exec) cudaGraphExecDestroy(chol->solve_exec);
  chol->factor_exec = chol->solve_exec = nullptr;
  chol->factor_key = chol->solve_b = chol->solve_x = nullptr;
  return ACOPF_OK;
}

acopf_status acopf_chol_get_trace(acopf_chol* chol, int32_t which, int64_t* out, int64_t capacity,
                                  int64_t* n_tasks) {
  if (!chol || !n_tasks || which < 0 || which > 5 || capacity < 0 || (!out && capacity > 0))
    return fail(ACOPF_E_INVALID_ARG, "acopf_chol_get_trace: bad argument");
  const acopf::CholTasks* tk[6] = {&chol->tg[0], &chol->tg[2], &chol->tg[3],
                                   &chol->tg[1], &chol->tg[4], &chol->tg[5]};
  *n_tasks = tk[which]->n;
  if (!tk[which]->trace) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_get_trace: trace is off");
  DeviceScope ds(chol->model->device);
  cudaError_t e = ds.error();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  const size_t cnt = size_t(std::min<int64_t>(capacity, tk[which]->n));
  if (e == cudaSuccess && cnt)
    e = cudaMemcpy(out, tk[which]->trace, 6 * cnt * sizeof(long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_get_trace");
  return ACOPF_OK;
}

acopf_status acopf_chol_permutation(const acopf_chol* chol, int32_t* perm) {
  if (!chol || !perm) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_permutation: null pointer");
  std::copy(chol->perm_host.begin(), chol->perm_host.end(), perm);
  return ACOPF_OK;
}

}  // extern "C"
