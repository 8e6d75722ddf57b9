// Sparse Cholesky factorization of M_cond (acopf_chol_*): the consumer of
// the condensed KKT matrix.  Sec. IV.C: M_aug has the inertia (n + m, 0, m)
// exactly when M_cond is positive definite, so a Cholesky factorization that
// meets a non-positive pivot is the inertia test, and the regularization
// (delta_w, delta_c) is raised until it succeeds.  Sec. V factorizes with a
// fill-reducing AMD order fixed once per pattern and a numeric
// refactorization per iteration.
//
// Here: the symbolic part (the full symmetric pattern of M_cond, its AMD
// order, the permuted pattern and a map from each of its entries to the
// lower-CSR values the assembler writes) is built on the host once per
// chol object; the numeric factorization and the triangular solves are
// cuSOLVER's sparse Cholesky (a library call, as in the paper), whose
// zero-pivot test is the positive-definiteness test; the value gather and
// the permutation of right-hand sides and solutions are kernels of chol.cu.
#include <cusolverSp.h>
#include <cusolverSp_LOWLEVEL_PREVIEW.h>
#include <cusparse.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "host_internal.h"

#if defined(__GNUC__)
#pragma GCC diagnostic ignored "-Wdeprecated-declarations"
#endif

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

struct acopf_chol {
  acopf_model* model = nullptr;
  int32_t n = 0;
  int32_t nnz = 0;             // of the full symmetric pattern
  acopf_chol_stats stats{};    // symbolic counts in the AMD order
  void* arena = nullptr;
  int32_t* rowptr = nullptr;   // n + 1: permuted full pattern (device)
  int32_t* colind = nullptr;   // nnz
  int32_t* src = nullptr;      // nnz: lower-CSR value index of each entry
  int32_t* perm = nullptr;     // n: row i of the permuted matrix is row perm[i] of M_cond
  double* vals = nullptr;      // nnz: values of the last factorization
  double* bp = nullptr;        // n: permuted right-hand side
  double* xp = nullptr;        // n: permuted solution
  void* buffer = nullptr;
  size_t internal_bytes = 0, work_bytes = 0;
  cusolverSpHandle_t handle = nullptr;
  cusparseMatDescr_t descr = nullptr;
  csrcholInfo_t info = nullptr;
  bool factored = false;
  std::vector<int32_t> perm_host;  // the fill-reducing order
};

namespace {

acopf_status solver_fail(cusolverStatus_t s, const char* where) {
  return fail(ACOPF_E_CUDA, std::string(where) + ": cuSOLVER status " + std::to_string(int(s)));
}

void release(acopf_chol* c) {
  if (c->info) cusolverSpDestroyCsrcholInfo(c->info);
  if (c->descr) cusparseDestroyMatDescr(c->descr);
  if (c->handle) cusolverSpDestroy(c->handle);
  if (c->buffer) cudaFree(c->buffer);
  if (c->arena) cudaFree(c->arena);
  delete c;
}

// Full symmetric CSR of the lower pattern (rp, ci): every strictly lower
// entry (i, j) also appears as (j, i).  src gives, per full entry, the index
// of its value in the lower CSR.  Columns ascend within each row when they
// ascend within each lower row.
void full_pattern(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                  std::vector<int32_t>& frp, std::vector<int32_t>& fci,
                  std::vector<int32_t>& fsrc) {
  frp.assign(size_t(n) + 1, 0);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
      frp[size_t(i) + 1]++;
      if (ci[size_t(k)] != i) frp[size_t(ci[size_t(k)]) + 1]++;
    }
  for (int32_t i = 0; i < n; ++i) frp[size_t(i) + 1] += frp[size_t(i)];
  fci.resize(size_t(frp[size_t(n)]));
  fsrc.resize(fci.size());
  std::vector<int32_t> next(frp.begin(), frp.end() - 1);
  // lower part of each row (columns <= i) first, then the mirrored entries
  // (i, j > i), which arrive in ascending j because rows are visited in order
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
      const int32_t p = next[size_t(i)]++;
      fci[size_t(p)] = ci[size_t(k)];
      fsrc[size_t(p)] = k;
    }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
      const int32_t j = ci[size_t(k)];
      if (j == i) continue;
      const int32_t p = next[size_t(j)]++;
      fci[size_t(p)] = i;
      fsrc[size_t(p)] = k;
    }
}

// Symbolic counts of the Cholesky factor of the permuted pattern (rp, ci,
// full symmetric, columns ascending): the elimination tree (Liu's algorithm
// with path compression), then the column counts of L by walking, for each
// row i, from every k < i in row i up the tree until a node already
// visited for row i (each visited node is a nonzero L(i, j)).  Returns
// nnz(L) including the diagonal and the flops of a column Cholesky:
// per column j with c_j off-diagonal entries, one square root, c_j
// divisions and c_j (c_j + 1) / 2 multiply-adds for the update.
void symbolic_counts(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     int64_t& nnz_l, double& flops, int64_t& max_col) {
  std::vector<int32_t> parent(size_t(n), -1), anc(size_t(n), -1), mark(size_t(n), -1);
  std::vector<int64_t> cnt(size_t(n), 0);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1] && ci[size_t(k)] < i; ++k) {
      int32_t r = ci[size_t(k)];
      while (anc[size_t(r)] != -1 && anc[size_t(r)] != i) {
        const int32_t t = anc[size_t(r)];
        anc[size_t(r)] = i;
        r = t;
      }
      if (anc[size_t(r)] == -1) {
        anc[size_t(r)] = i;
        parent[size_t(r)] = i;
      }
    }
  for (int32_t i = 0; i < n; ++i) {
    mark[size_t(i)] = i;
    for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1] && ci[size_t(k)] < i; ++k)
      for (int32_t j = ci[size_t(k)]; j != -1 && mark[size_t(j)] != i; j = parent[size_t(j)]) {
        mark[size_t(j)] = i;
        cnt[size_t(j)]++;
      }
  }
  nnz_l = n;
  flops = 0.0;
  max_col = 0;
  for (int32_t j = 0; j < n; ++j) {
    const double c = double(cnt[size_t(j)]);
    max_col = std::max<int64_t>(max_col, cnt[size_t(j)] + 1);
    nnz_l += cnt[size_t(j)];
    flops += 1.0 + c + c * (c + 1.0);
  }
}

// The symbolic phase: the AMD order P of M_cond's full symmetric pattern,
// the pattern of P M_cond P' (rows sorted by column) with, per entry, the
// index of its value in the lower CSR, and the factor's counts.
struct Symbolic {
  std::vector<int32_t> perm, prp, pci, psrc;
  acopf_chol_stats stats{};
};

acopf_status check_model(const acopf_model* model, const char* where) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": null model");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, std::string(where) + ": host-only model");
  const acopf::HostModel& hm = model->hm;
  const int32_t n = hm.L.n;
  for (int32_t i = 0; i < n; ++i) {
    const int32_t a = hm.krowptr[size_t(i)], b = hm.krowptr[size_t(i) + 1];
    if (a == b || hm.kcolind[size_t(b) - 1] != i)
      return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": M_cond pattern lacks a diagonal");
  }
  if (2 * int64_t(hm.krowptr[size_t(n)]) - n > INT32_MAX)
    return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": pattern too large");
  return ACOPF_OK;
}

cusolverStatus_t make_handle(cusolverSpHandle_t& h, cusparseMatDescr_t& d) {
  cusolverStatus_t cs = cusolverSpCreate(&h);
  if (cs == CUSOLVER_STATUS_SUCCESS && cusparseCreateMatDescr(&d) != CUSPARSE_STATUS_SUCCESS)
    cs = CUSOLVER_STATUS_INTERNAL_ERROR;
  if (cs == CUSOLVER_STATUS_SUCCESS) {
    cusparseSetMatType(d, CUSPARSE_MATRIX_TYPE_GENERAL);
    cusparseSetMatIndexBase(d, CUSPARSE_INDEX_BASE_ZERO);
  }
  return cs;
}

acopf_status symbolic(const acopf::HostModel& hm, cusolverSpHandle_t h, cusparseMatDescr_t d,
                      Symbolic& sy) {
  const int32_t n = hm.L.n;
  try {
    std::vector<int32_t> frp, fci, fsrc, iperm(static_cast<size_t>(n), -1);
    full_pattern(n, hm.krowptr, hm.kcolind, frp, fci, fsrc);
    const int32_t nnz = int32_t(fci.size());
    // Fill-reducing order of the symmetric pattern (approximate minimum degree).
    sy.perm.assign(size_t(n), 0);
    cusolverStatus_t cs =
        cusolverSpXcsrsymamdHost(h, n, nnz, d, frp.data(), fci.data(), sy.perm.data());
    if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "M_cond ordering");
    for (int32_t i = 0; i < n; ++i) {
      const int32_t r = sy.perm[size_t(i)];
      if (r < 0 || r >= n || iperm[size_t(r)] >= 0)
        return fail(ACOPF_E_CUDA, "M_cond ordering: not a permutation");
      iperm[size_t(r)] = i;
    }
    // Permuted pattern: row i holds row perm[i] of the full matrix, with each
    // column j renumbered iperm[j] and the rows sorted by column.
    sy.prp.assign(size_t(n) + 1, 0);
    sy.pci.resize(fci.size());
    sy.psrc.resize(fci.size());
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int32_t i = 0; i < n; ++i) {
      const int32_t r = sy.perm[size_t(i)];
      row.clear();
      for (int32_t k = frp[size_t(r)]; k < frp[size_t(r) + 1]; ++k)
        row.emplace_back(iperm[size_t(fci[size_t(k)])], fsrc[size_t(k)]);
      std::sort(row.begin(), row.end());
      const int32_t base = sy.prp[size_t(i)];
      for (size_t t = 0; t < row.size(); ++t) {
        sy.pci[size_t(base) + t] = row[t].first;
        sy.psrc[size_t(base) + t] = row[t].second;
      }
      sy.prp[size_t(i) + 1] = base + int32_t(row.size());
    }
    sy.stats.n = n;
    sy.stats.nnz_full = nnz;
    symbolic_counts(n, sy.prp, sy.pci, sy.stats.nnz_factor, sy.stats.factor_flops,
                    sy.stats.max_col);
  } catch (const std::bad_alloc&) {
    return fail(ACOPF_E_OOM, "host allocation failed");
  }
  return ACOPF_OK;
}

}  // namespace

extern "C" {

acopf_status acopf_chol_create(acopf_model* model, acopf_chol** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_create: null output pointer");
  *out = nullptr;
  acopf_status st = check_model(model, "acopf_chol_create");
  if (st != ACOPF_OK) return st;
  const int32_t n = model->hm.L.n;
  acopf_chol* c = new (std::nothrow) acopf_chol;
  if (!c) return fail(ACOPF_E_OOM, "host allocation failed");
  c->model = model;
  c->n = n;
  DeviceScope ds(model->device);
  cudaError_t e = ds.error();
  if (e != cudaSuccess) {
    release(c);
    return cuda_fail(e, "acopf_chol_create");
  }
  cusolverStatus_t cs = make_handle(c->handle, c->descr);
  if (cs != CUSOLVER_STATUS_SUCCESS) {
    release(c);
    return solver_fail(cs, "acopf_chol_create: handle");
  }
  Symbolic sy;
  st = symbolic(model->hm, c->handle, c->descr, sy);
  if (st != ACOPF_OK) {
    release(c);
    return st;
  }
  c->nnz = int32_t(sy.pci.size());
  c->stats = sy.stats;
  c->perm_host = sy.perm;
  const std::vector<int32_t>&prp = sy.prp, &pci = sy.pci, &psrc = sy.psrc, &perm = sy.perm;

  acopf::ArenaPlan p;
  const size_t o_rp = p.take<int32_t>(size_t(n) + 1), o_ci = p.take<int32_t>(size_t(c->nnz));
  const size_t o_src = p.take<int32_t>(size_t(c->nnz)), o_perm = p.take<int32_t>(size_t(n));
  const size_t o_v = p.take<double>(size_t(c->nnz));
  const size_t o_bp = p.take<double>(size_t(n)), o_xp = p.take<double>(size_t(n));
  e = cudaMalloc(&c->arena, p.off);
  if (e != cudaSuccess) {
    c->arena = nullptr;
    release(c);
    return cuda_fail(e, "acopf_chol_create");
  }
  char* base = static_cast<char*>(c->arena);
  c->rowptr = reinterpret_cast<int32_t*>(base + o_rp);
  c->colind = reinterpret_cast<int32_t*>(base + o_ci);
  c->src = reinterpret_cast<int32_t*>(base + o_src);
  c->perm = reinterpret_cast<int32_t*>(base + o_perm);
  c->vals = reinterpret_cast<double*>(base + o_v);
  c->bp = reinterpret_cast<double*>(base + o_bp);
  c->xp = reinterpret_cast<double*>(base + o_xp);
  e = cudaMemcpy(c->rowptr, prp.data(), prp.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->colind, pci.data(), pci.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->src, psrc.data(), psrc.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->vals, 0, size_t(c->nnz) * sizeof(double));
  if (e != cudaSuccess) {
    release(c);
    return cuda_fail(e, "acopf_chol_create: upload");
  }
  cs = cusolverSpCreateCsrcholInfo(&c->info);
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpXcsrcholAnalysis(c->handle, n, c->nnz, c->descr, c->rowptr, c->colind, c->info);
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpDcsrcholBufferInfo(c->handle, n, c->nnz, c->descr, c->vals, c->rowptr,
                                      c->colind, c->info, &c->internal_bytes, &c->work_bytes);
  if (cs != CUSOLVER_STATUS_SUCCESS) {
    const std::string what = "acopf_chol_create: analysis of a factor of " +
                             std::to_string(c->stats.nnz_factor) + " entries (" +
                             std::to_string(c->stats.factor_flops * 1e-9) +
                             " GFLOP, largest column " + std::to_string(c->stats.max_col) +
                             ") in the AMD order";
    release(c);
    return solver_fail(cs, what.c_str());
  }
  e = cudaMalloc(&c->buffer, std::max<size_t>(c->work_bytes, 256));
  if (e != cudaSuccess) {
    c->buffer = nullptr;
    release(c);
    return cuda_fail(e, "acopf_chol_create: workspace");
  }
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
  cudaError_t e = acopf::launch_gather(chol->vals, kvals, chol->src, chol->nnz, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_factor: gather");
  cusolverStatus_t cs = cusolverSpSetStream(chol->handle, s);
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpDcsrcholFactor(chol->handle, chol->n, chol->nnz, chol->descr, chol->vals,
                                  chol->rowptr, chol->colind, chol->info, chol->buffer);
  // The library's zero-pivot test: the first pivot that is negative or at
  // most pivot_tol (a factorization of an indefinite matrix runs to the end
  // but records it); this returns to the host.
  int pos = -1;
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpDcsrcholZeroPivot(chol->handle, chol->info, pivot_tol, &pos);
  if (cs != CUSOLVER_STATUS_SUCCESS && cs != CUSOLVER_STATUS_ZERO_PIVOT)
    return solver_fail(cs, "acopf_chol_factor");
  if (cs == CUSOLVER_STATUS_ZERO_PIVOT && pos < 0) pos = 0;
  *first_bad_pivot = pos < 0 ? -1 : pos;
  chol->factored = pos < 0;
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
  cudaError_t e = acopf::launch_gather(chol->bp, b, chol->perm, chol->n, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_solve: permute");
  cusolverStatus_t cs = cusolverSpSetStream(chol->handle, s);
  if (cs == CUSOLVER_STATUS_SUCCESS)
    cs = cusolverSpDcsrcholSolve(chol->handle, chol->n, chol->bp, chol->xp, chol->info,
                                 chol->buffer);
  if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "acopf_chol_solve");
  e = acopf::launch_scatter(x, chol->xp, chol->perm, chol->n, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_chol_solve: permute back");
  return ACOPF_OK;
}

acopf_status acopf_chol_info(const acopf_chol* chol, acopf_chol_stats* stats,
                             int64_t* device_bytes) {
  if (!chol) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_info: null pointer");
  if (stats) *stats = chol->stats;
  if (device_bytes)
    *device_bytes = int64_t(chol->internal_bytes + std::max<size_t>(chol->work_bytes, 256));
  return ACOPF_OK;
}

acopf_status acopf_chol_analyze(acopf_model* model, acopf_chol_stats* stats) {
  if (!stats) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_analyze: null output pointer");
  acopf_status st = check_model(model, "acopf_chol_analyze");
  if (st != ACOPF_OK) return st;
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_chol_analyze");
  cusolverSpHandle_t h = nullptr;
  cusparseMatDescr_t d = nullptr;
  cusolverStatus_t cs = make_handle(h, d);
  Symbolic sy;
  if (cs == CUSOLVER_STATUS_SUCCESS) st = symbolic(model->hm, h, d, sy);
  if (d) cusparseDestroyMatDescr(d);
  if (h) cusolverSpDestroy(h);
  if (cs != CUSOLVER_STATUS_SUCCESS) return solver_fail(cs, "acopf_chol_analyze: handle");
  if (st != ACOPF_OK) return st;
  *stats = sy.stats;
  return ACOPF_OK;
}

acopf_status acopf_chol_permutation(const acopf_chol* chol, int32_t* perm) {
  if (!chol || !perm) return fail(ACOPF_E_INVALID_ARG, "acopf_chol_permutation: null pointer");
  std::copy(chol->perm_host.begin(), chol->perm_host.end(), perm);
  return ACOPF_OK;
}

}  // extern "C"
