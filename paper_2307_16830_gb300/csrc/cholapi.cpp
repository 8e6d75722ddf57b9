// Sparse Cholesky factorization of M_cond (acopf_chol_*): the consumer of
// the condensed KKT matrix.  Sec. IV.C: M_aug has the inertia (n + m, 0, m)
// exactly when M_cond is positive definite, so a Cholesky factorization that
// meets a non-positive pivot is the inertia test, and the regularization
// (delta_w, delta_c) is raised until it succeeds.  Sec. V factorizes with a
// fill-reducing order fixed once per pattern and refactors numerically every
// iteration.
//
// Here: the symbolic phase (symbolic.cpp) runs on the host once per chol
// object; the numeric factorization (multifrontal), its pivot test and the
// solves are the supernodal kernels of chol.cu, one launch per level of the
// supernodal elimination tree.
#include <algorithm>
#include <climits>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "chol_internal.h"
#include "host_internal.h"
#include "symbolic.h"

static_assert(acopf::kMaxSupernodeWidth == acopf::kCholMaxWidth,
              "the syrk tiles and solve staging hold a supernode's full width");
static_assert(acopf::kPanelSmemDoubles == acopf::kCholPanelDoubles &&
                  acopf::kWarpMaxRows == acopf::kCholWarpRows &&
                  acopf::kWarpMaxCols == acopf::kCholWarpCols &&
                  acopf::kMaxRowsBelow == acopf::kCholMaxRelRows,
              "host and kernels agree on what is staged in shared memory");

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

struct acopf_chol {
  acopf_model* model = nullptr;
  int32_t n = 0;
  int64_t nnz_low = 0;
  acopf_chol_stats stats{};
  std::vector<int32_t> perm_host, level_ptr, level_large, level_smem, tile_ptr;
  std::vector<int32_t> level_big, level_smem_big, level_small_stage;
  const int4* tiles = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  acopf::CholDev dev{};
  const int64_t* amap = nullptr;
  const int32_t* perm = nullptr;
  double* work = nullptr;       // n: the permuted right-hand side / solution
  size_t u_doubles = 0, z_doubles = 0;  // update matrices / vectors
  int32_t* bad_host = nullptr;  // page-locked copy of dev.bad
  bool factored = false;
  // the groups of a level (big, other block-handled, small supernodes) are
  // independent: two side streams run them beside the caller's stream
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  // the factorization's and the solve's launch sequences, captured as CUDA
  // graphs for the last arguments they ran with
  cudaGraphExec_t factor_exec = nullptr, solve_exec = nullptr;
  const void* factor_key = nullptr;
  double factor_tol = -1.0;
  const void *solve_b = nullptr, *solve_x = nullptr;
};

namespace {

void release(acopf_chol* c) {
  for (cudaStream_t st : c->side)
    if (st) cudaStreamDestroy(st);
  if (c->fork) cudaEventDestroy(c->fork);
  for (cudaEvent_t ev : c->join)
    if (ev) cudaEventDestroy(ev);
  if (c->factor_exec) cudaGraphExecDestroy(c->factor_exec);
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  if (c->arena) cudaFree(c->arena);
  if (c->bad_host) cudaFreeHost(c->bad_host);
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

acopf_status run_symbolic(const acopf_model* model, acopf::CholSymbolic& sy, const char* where) {
  std::string err;
  const acopf_status st =
      acopf::chol_symbolic(model->hm.L.n, model->hm.krowptr, model->hm.kcolind, sy, err);
  if (st != ACOPF_OK) return fail(st, std::string(where) + ": " + err);
  return ACOPF_OK;
}

// The factorization's device work: zeroed blocks, the assembly of M_cond's
// values, and per level the big, the other block-handled and the small
// supernodes (independent: on the caller's stream and two side streams that
// fork from it and join back), then the update-matrix tiles.
cudaError_t record_factor(const acopf_chol* chol, const double* kvals, double tol,
                          cudaStream_t s) {
  const acopf::CholDev& d = chol->dev;
  cudaError_t e = cudaMemsetAsync(d.Lx, 0, size_t(chol->stats.storage) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.Ux, 0, chol->u_doubles * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.bad, 0x7f, sizeof(int32_t), s);  // 0x7f7f7f7f: none
  if (e == cudaSuccess) e = acopf::launch_chol_assemble(d.Lx, chol->amap, kvals, chol->nnz_low, s);
  const std::vector<int32_t>&lp = chol->level_ptr, &ll = chol->level_large, &tp = chol->tile_ptr;
  for (size_t v = 0; e == cudaSuccess && v + 1 < lp.size(); ++v) {
    const int32_t nb = chol->level_big[v], nl = ll[v], cnt = lp[v + 1] - lp[v];
    // the level's groups, each on its own stream when more than one is present
    const bool groups[3] = {nb > 0, nl > nb, cnt > nl};
    const int ngroups = int(groups[0]) + int(groups[1]) + int(groups[2]);
    cudaStream_t gs[3] = {s, s, s};
    if (ngroups > 1) {
      e = cudaEventRecord(chol->fork, s);
      int k = 0;
      for (int g = 0; g < 3 && e == cudaSuccess; ++g) {
        if (!groups[g]) continue;
        if (k > 0) {
          gs[g] = chol->side[k - 1];
          e = cudaStreamWaitEvent(gs[g], chol->fork, 0);
        }
        ++k;
      }
    }
    if (e == cudaSuccess && groups[0])
      e = acopf::launch_chol_factor_level(d, lp[v], nb, nb, tol, chol->level_smem_big[v],
                                          chol->tiles, 0, 0, gs[0]);
    if (e == cudaSuccess && groups[1])
      e = acopf::launch_chol_factor_level(d, lp[v] + nb, nl - nb, nl - nb, tol,
                                          chol->level_smem[v], chol->tiles, 0, 0, gs[1]);
    if (e == cudaSuccess && groups[2])
      e = acopf::launch_chol_factor_level(d, lp[v] + nl, cnt - nl, 0, tol,
                                          chol->level_small_stage[v], chol->tiles, 0, 0, gs[2]);
    if (ngroups > 1) {  // join the side streams back
      int k = 0;
      for (int g = 0; g < 3 && e == cudaSuccess; ++g) {
        if (!groups[g] || gs[g] == s) continue;
        e = cudaEventRecord(chol->join[k], gs[g]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, chol->join[k], 0);
        ++k;
      }
    }
    if (e == cudaSuccess && tp[v + 1] > tp[v])
      e = acopf::launch_chol_factor_level(d, lp[v], 0, 0, tol, 0, chol->tiles, tp[v],
                                          tp[v + 1] - tp[v], s);
  }
  return e;
}

// The solve's device work: permutation, forward levels, backward levels,
// permutation back.
cudaError_t record_solve(const acopf_chol* chol, const double* b, double* x, cudaStream_t s) {
  const acopf::CholDev& d = chol->dev;
  const std::vector<int32_t>&lp = chol->level_ptr, &ll = chol->level_large;
  cudaError_t e = acopf::launch_gather(chol->work, b, chol->perm, chol->n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.Zx, 0, chol->z_doubles * sizeof(double), s);
  for (size_t v = 0; e == cudaSuccess && v + 1 < lp.size(); ++v)
    e = acopf::launch_chol_fwd_level(d, lp[v], lp[v + 1] - lp[v], ll[v], chol->work, s);
  for (size_t v = lp.size() - 1; e == cudaSuccess && v > 0; --v)
    e = acopf::launch_chol_bwd_level(d, lp[v - 1], lp[v] - lp[v - 1], ll[v - 1], chol->work, s);
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

extern "C" {

acopf_status acopf_chol_analyze(acopf_model* model, acopf_chol_stats* stats,
                                int32_t* perm) {
  if (!stats) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_analyze: null output pointer");
  acopf_status st = check_model(model, "acopf_chol_analyze");
  if (st != ACOPF_OK) return st;
  acopf::CholSymbolic sy;
  st = run_symbolic(model, sy, "acopf_chol_analyze");
  if (st != ACOPF_OK) return st;
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
  acopf_chol* c = new (std::nothrow) acopf_chol;
  if (!c) return fail(ACOPF_E_OOM, "host allocation failed");
  c->model = model;
  c->n = sy.n;
  c->nnz_low = int64_t(sy.amap.size());
  c->stats = sy.stats;
  try {
    c->perm_host = sy.perm;
    c->level_ptr = sy.level_ptr;
    c->level_large = sy.level_large;
    c->level_smem = sy.level_smem;
    c->level_big = sy.level_big;
    c->level_smem_big = sy.level_smem_big;
    c->level_small_stage = sy.level_small_stage;
    c->tile_ptr = sy.tile_ptr;
  } catch (const std::bad_alloc&) {
    release(c);
    return fail(ACOPF_E_OOM, "host allocation failed");
  }
  const size_t ns = size_t(sy.ns), n = size_t(sy.n);
  acopf::ArenaPlan p;
  const size_t o_first = p.take<int32_t>(ns + 1), o_rowptr = p.take<int32_t>(ns + 1);
  const size_t o_rowidx = p.take<int32_t>(sy.rowidx.size()), o_off = p.take<int64_t>(ns + 1);
  const size_t o_kptr = p.take<int32_t>(ns + 1), o_kid = p.take<int32_t>(sy.kid.size());
  const size_t o_roff = p.take<int32_t>(ns), o_rel = p.take<int32_t>(sy.relmap.size());
  const size_t o_uoff = p.take<int64_t>(ns + 1), o_zoff = p.take<int64_t>(ns + 1);
  const size_t o_lev = p.take<int32_t>(ns), o_tiles = p.take<int32_t>(sy.tiles.size());
  const size_t o_amap = p.take<int64_t>(sy.amap.size()), o_perm = p.take<int32_t>(n);
  const size_t o_work = p.take<double>(n), o_bad = p.take<int32_t>(1);
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
  up(o_lev, sy.level_sn.data(), ns * 4);
  up(o_tiles, sy.tiles.data(), sy.tiles.size() * 4);
  up(o_amap, sy.amap.data(), sy.amap.size() * 8);
  up(o_perm, sy.perm.data(), n * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&c->bad_host, sizeof(int32_t));
  for (cudaStream_t& st : c->side)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
  for (cudaEvent_t& ev : c->join)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  size_t smem = 0;
  for (size_t v = 0; v + 1 < sy.level_ptr.size(); ++v) {
    const int32_t nb = sy.level_big[v], nl = sy.level_large[v];
    const int32_t cnt = sy.level_ptr[v + 1] - sy.level_ptr[v];
    smem = std::max({smem, acopf::chol_factor_smem_bytes(nb, nb, sy.level_smem_big[v]),
                     acopf::chol_factor_smem_bytes(nl - nb, nl - nb, sy.level_smem[v]),
                     acopf::chol_factor_smem_bytes(cnt - nl, 0, sy.level_small_stage[v])});
  }
  if (e == cudaSuccess) e = acopf::chol_allow_smem(smem);
  if (e != cudaSuccess) {
    release(c);
    return cuda_fail(e, "acopf_chol_create: upload");
  }
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
  d.level_sn = reinterpret_cast<const int32_t*>(base + o_lev);
  d.Lx = reinterpret_cast<double*>(base + o_lx);
  d.Ux = reinterpret_cast<double*>(base + o_ux);
  d.Zx = reinterpret_cast<double*>(base + o_zx);
  d.bad = reinterpret_cast<int32_t*>(base + o_bad);
  c->amap = reinterpret_cast<const int64_t*>(base + o_amap);
  c->perm = reinterpret_cast<const int32_t*>(base + o_perm);
  c->work = reinterpret_cast<double*>(base + o_work);
  c->tiles = reinterpret_cast<const int4*>(base + o_tiles);
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
    e = cudaMemcpyAsync(chol->bad_host, d.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_factor");
  const int32_t bad = *chol->bad_host;
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

acopf_status acopf_chol_permutation(const acopf_chol* chol, int32_t* perm) {
  if (!chol || !perm) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_permutation: null pointer");
  std::copy(chol->perm_host.begin(), chol->perm_host.end(), perm);
  return ACOPF_OK;
}

}  // extern "C"
