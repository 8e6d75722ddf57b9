// The condensed-space interior-point method (Algorithm 1), driven from the
// host over the library's device kernels (acopf_ipm_solve).
//
// Per iteration: the scaled residual of Eq. first (convergence test), the
// monotone barrier update, the Newton right-hand side, the Hessian, the
// condensation and the assembly of M_cond, its factorization with the
// inertia correction on delta_w, the solve and the step recovery, the step
// bounds, the filter line search over trial points (objective, constraints
// and barrier terms evaluated on the device), the update of the iterate and
// of the multipliers.  The scalar decisions (filter, step sizes, barrier
// parameter, regularization) are taken on the host from a few reduced values
// per step; every vector stays on the device.  The rules and constants are
// those of the interior-point reference the paper cites for its line
// search, with its second-order correction (reading d11); a failed line search enters a
// feasibility restoration (reading d10) that returns to the iteration or
// ends the solve as infeasible.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "host_internal.h"
#include "ipm_internal.h"

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

namespace {

// The reference's default constants (see the oracle for their roles).
constexpr double kKappaEps = 10.0, kKappaMu = 0.2, kThetaMu = 1.5, kTauMin = 0.99;
constexpr double kBoundPush = 1e-2, kBoundFrac = 1e-2;
constexpr double kGammaTheta = 1e-5, kGammaPhi = 1e-8, kDelta = 1.0, kSTheta = 1.1, kSPhi = 2.3;
constexpr double kEtaPhi = 1e-4, kAlphaMinFrac = 0.05, kKappaSigma = 1e10;
constexpr int kSocMax = 4;          // second-order corrections per line search at most
constexpr double kKappaSoc = 0.99;  // ... each cutting the violation below this fraction
constexpr double kDeltaW0 = 1e-4, kDeltaWMin = 1e-20, kDeltaWMax = 1e40;
constexpr double kKappaWMinus = 1.0 / 3.0, kKappaWPlus = 8.0, kKappaWPlusBar = 100.0;
constexpr int kMaxBacktracks = 60, kMaxInertiaTries = 200;
// feasibility restoration (reading d10): iterations at most, stall window,
// smallest barrier parameter, required reduction of the violation
constexpr int kRestoMaxIter = 200, kRestoStall = 10;
constexpr double kRestoMuMin = 1e-9, kRestoReduction = 0.9, kRestoReductionRepeat = 1e-3;

// The reference's initial-point rule: at least min(k1 max(1,|b|), k2 (hi - lo))
// inside each finite bound.
double push_interior(double v, double lo, double hi) {
  const bool fl = std::isfinite(lo), fh = std::isfinite(hi);
  const double width = fl && fh ? hi - lo : std::numeric_limits<double>::infinity();
  if (fl) v = std::max(v, lo + std::min(kBoundPush * std::max(1.0, std::fabs(lo)), kBoundFrac * width));
  if (fh) v = std::min(v, hi - std::min(kBoundPush * std::max(1.0, std::fabs(hi)), kBoundFrac * width));
  return v;
}

struct Buffers {
  void* arena = nullptr;
  acopf::IpmVec v{};
  double *xl, *xu, *sl, *su, *sigma_x, *sigma_s, *q_s, *rhs, *hvals, *kvals;
  double *xr, *lo_s, *hi_s, *r;  // restoration: proximal centre, pushed slack box, violation
  // second-order correction: its direction (dx, ds, dy and the bound
  // multipliers' steps; the rest of an IpmVec is the iterate's), c_soc, -c_soc
  double *dx2, *ds2, *dy2, *dzl_x2, *dzu_x2, *dzl_s2, *dzu_s2, *c_soc, *py_soc;
  double *f, *ft, *out, *part;  // out: 16 reduced scalars, part: per-block partials
  ~Buffers() {
    if (arena) cudaFree(arena);
  }
};

}  // namespace

extern "C" {

// The solve; `given`: a Cholesky object of this model to use (the caller's),
// or NULL to create one for this solve.
static acopf_status ipm_solve_impl(acopf_model* model, acopf_chol* given,
                                   const acopf_ipm_options* options, double* x_out,
                                   double* history, acopf_ipm_result* result,
                                   acopf_stream stream) {
  if (!model || !options || !result)
    return fail(ACOPF_E_INVALID_ARG, "acopf_ipm_solve: null pointer");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "acopf_ipm_solve: host-only model");
  const double tol = options->tol, mu_init = options->mu_init;
  const int32_t max_iter = options->max_iter;
  if (!(tol > 0.0) || !std::isfinite(tol) || !(mu_init > 0.0) || !std::isfinite(mu_init) ||
      max_iter < 0)
    return fail(ACOPF_E_INVALID_ARG,
                "acopf_ipm_solve: tol and mu_init must be finite and > 0, max_iter >= 0");
  const auto t_start = std::chrono::steady_clock::now();
  *result = acopf_ipm_result{};
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_ipm_solve");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  acopf_stream as = stream;
  const acopf::HostModel& hm = model->hm;
  const acopf::Layout& L = hm.L;
  const int32_t n = L.n, m = L.m;
  acopf_status st = acopf::step_lists(model);
  if (st != ACOPF_OK) return st;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, model->device);
  const int blocks = acopf::ipm_blocks(std::max(sms, 1));

  // ---- device buffers ------------------------------------------------------
  Buffers B;
  acopf::ArenaPlan p;
  const size_t N = size_t(n), M = size_t(m);
  enum { kVecN = 20, kVecM = 29 };
  const size_t o_n = p.take<double>(kVecN * N), o_m = p.take<double>(kVecM * M);
  const size_t o_j = p.take<double>(size_t(L.nnzj)), o_h = p.take<double>(size_t(L.nnzh));
  const size_t o_k = p.take<double>(size_t(L.nnzk)), o_s = p.take<double>(32);
  const size_t o_p = p.take<double>(4 * size_t(blocks));
  cudaError_t e = cudaMalloc(&B.arena, p.off);
  if (e != cudaSuccess) {
    B.arena = nullptr;
    return cuda_fail(e, "acopf_ipm_solve: allocation");
  }
  char* base = static_cast<char*>(B.arena);
  double* vn = reinterpret_cast<double*>(base + o_n);
  double* vm = reinterpret_cast<double*>(base + o_m);
  auto nv = [&](int k) { return vn + size_t(k) * N; };
  auto mv = [&](int k) { return vm + size_t(k) * M; };
  acopf::IpmVec& v = B.v;
  v.x = nv(0); v.xt = nv(1); B.xl = nv(2); B.xu = nv(3); v.zl_x = nv(4); v.zu_x = nv(5);
  v.grad = nv(6); v.p_x = nv(7); v.p_zl_x = nv(8); v.p_zu_x = nv(9); B.sigma_x = nv(10);
  B.rhs = nv(11); v.dx = nv(12); v.dzl_x = nv(13); v.dzu_x = nv(14);
  v.s = mv(0); v.st = mv(1); B.sl = mv(2); B.su = mv(3); v.zl_s = mv(4); v.zu_s = mv(5);
  v.y = mv(6); v.ym = mv(7); v.cons = mv(8); v.cons_t = mv(9); v.p_s = mv(10); v.p_y = mv(11);
  v.p_zl_s = mv(12); v.p_zu_s = mv(13); B.sigma_s = mv(14); B.q_s = mv(15); v.ds = mv(16);
  v.dy = mv(17); v.dzl_s = mv(18); v.dzu_s = mv(19);
  B.xr = nv(15); B.lo_s = mv(20); B.hi_s = mv(21); B.r = mv(22);
  B.dx2 = nv(16); B.dzl_x2 = nv(17); B.dzu_x2 = nv(18);
  B.ds2 = mv(23); B.dy2 = mv(24); B.dzl_s2 = mv(25); B.dzu_s2 = mv(26); B.c_soc = mv(27);
  B.py_soc = mv(28);
  v.xl = B.xl; v.xu = B.xu; v.sl = B.sl; v.su = B.su;
  v.jvals = reinterpret_cast<double*>(base + o_j);
  B.hvals = reinterpret_cast<double*>(base + o_h);
  B.kvals = reinterpret_cast<double*>(base + o_k);
  double* scal = reinterpret_cast<double*>(base + o_s);
  B.f = scal; B.ft = scal + 1; B.out = scal + 8;
  B.part = reinterpret_cast<double*>(base + o_p);

  // ---- initial point (reading d8) -------------------------------------------
  std::vector<double> hx(N, 0.0), hs(M), hsl(M), hsu(M), hzlx(N), hzux(N), hzls(M), hzus(M);
  std::vector<double> hlos(M), hhis(M);
  for (int32_t j = 0; j < n; ++j) {
    const double lo = hm.xl[size_t(j)], hi = hm.xu[size_t(j)];
    hx[size_t(j)] = std::isfinite(lo) && std::isfinite(hi) ? 0.5 * (lo + hi) : 0.0;
  }
  for (int32_t b = 0; b < L.nb; ++b) {
    hx[size_t(b)] = 0.0;          // va
    hx[size_t(L.nb + b)] = 1.0;   // vm
  }
  for (int32_t j = 0; j < n; ++j) {
    hx[size_t(j)] = push_interior(hx[size_t(j)], hm.xl[size_t(j)], hm.xu[size_t(j)]);
    hzlx[size_t(j)] = std::isfinite(hm.xl[size_t(j)]) ? 1.0 : 0.0;
    hzux[size_t(j)] = std::isfinite(hm.xu[size_t(j)]) ? 1.0 : 0.0;
  }
  for (int32_t r = 0; r < m; ++r) {  // Eq. relax: bounds widened by tol max(1, |b|)
    const double lo = hm.gl[size_t(r)], hi = hm.gu[size_t(r)];
    hsl[size_t(r)] = std::isfinite(lo) ? lo - tol * std::max(1.0, std::fabs(lo)) : -INFINITY;
    hsu[size_t(r)] = std::isfinite(hi) ? hi + tol * std::max(1.0, std::fabs(hi)) : INFINITY;
    hzls[size_t(r)] = std::isfinite(hsl[size_t(r)]) ? 1.0 : 0.0;
    hzus[size_t(r)] = std::isfinite(hsu[size_t(r)]) ? 1.0 : 0.0;
    // the restoration's slack box: the slack bounds pushed inside as for the initial point
    hlos[size_t(r)] = std::isfinite(hsl[size_t(r)]) ? push_interior(-INFINITY, hsl[size_t(r)], hsu[size_t(r)])
                                                    : -INFINITY;
    hhis[size_t(r)] = std::isfinite(hsu[size_t(r)]) ? push_interior(INFINITY, hsl[size_t(r)], hsu[size_t(r)])
                                                    : INFINITY;
  }
  auto up = [&](double* d, const std::vector<double>& h) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s);
  };
  up(v.x, hx); up(B.xl, hm.xl); up(B.xu, hm.xu); up(B.sl, hsl); up(B.su, hsu);
  up(v.zl_x, hzlx); up(v.zu_x, hzux); up(v.zl_s, hzls); up(v.zu_s, hzus);
  up(B.lo_s, hlos); up(B.hi_s, hhis);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.y, 0, M * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.ym, 0, M * 8, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: upload");
  st = acopf_eval_cons(model, v.x, v.cons, as);
  if (st != ACOPF_OK) return st;
  e = cudaMemcpyAsync(hs.data(), v.cons, M * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: initial constraints");
  for (int32_t r = 0; r < m; ++r) {
    const double lo = hsl[size_t(r)], hi = hsu[size_t(r)];
    double sr = std::min(std::max(hs[size_t(r)], lo), hi);
    hs[size_t(r)] = push_interior(sr, lo, hi);
  }
  up(v.s, hs);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: slacks");

  acopf_chol* chol = given;
  if (!chol) {
    st = acopf_chol_create(model, &chol);
    if (st != ACOPF_OK) return st;
  }
  struct CholGuard {
    acopf_chol* c;
    ~CholGuard() {
      if (c) acopf_chol_destroy(c);
    }
  } guard{given ? nullptr : chol};

  // ---- helpers ---------------------------------------------------------------
  acopf_iterate it{};
  auto set_iterate = [&]() {
    it = acopf_iterate{v.x,    v.s,    B.xl,     B.xu,     B.sl,     B.su,     v.zl_x,
                       v.zu_x, v.zl_s, v.zu_s,   v.p_x,    v.p_s,    v.p_y,    v.p_zl_x,
                       v.p_zu_x, v.p_zl_s, v.p_zu_s};
  };
  double hout[16];
  auto fetch = [&](int count) -> cudaError_t {  // B.out[0..count) -> hout
    cudaError_t err = cudaMemcpyAsync(hout, B.out, size_t(count) * 8, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    return err;
  };
  auto residual = [&](double mu, double& out_e) -> acopf_status {
    acopf_status r = acopf_kkt_residual(model, &it, v.y, v.grad, v.cons, v.jvals, mu, B.out, as);
    if (r != ACOPF_OK) return r;
    const cudaError_t err = fetch(1);
    if (err != cudaSuccess) return cuda_fail(err, "acopf_ipm_solve: residual");
    out_e = hout[0];
    return ACOPF_OK;
  };
  // E at 0 (the convergence test) and at mu (the barrier test) from one pass.
  auto residual_pair = [&](double mu2, double& e0, double& e_mu) -> acopf_status {
    acopf::StepIterate si{};
    si.x = it.x;
    si.s = it.s;
    si.xl = it.xl;
    si.xu = it.xu;
    si.sl = it.sl;
    si.su = it.su;
    si.zl_x = it.zl_x;
    si.zu_x = it.zu_x;
    si.zl_s = it.zl_s;
    si.zu_s = it.zu_s;
    cudaError_t err = acopf::launch_kkt_residual2(model->step, si, v.y, v.grad, v.cons, v.jvals,
                                                  0.0, mu2, B.out, s);
    if (err == cudaSuccess) err = fetch(10);
    if (err != cudaSuccess) return cuda_fail(err, "acopf_ipm_solve: residual");
    e0 = hout[0];
    e_mu = hout[9];
    return ACOPF_OK;
  };
  auto record = [&](int32_t k, int field, double value) {
    if (history && k <= max_iter) history[size_t(k) * ACOPF_IPM_HISTORY_FIELDS + size_t(field)] = value;
  };
  if (history)
    std::fill(history, history + size_t(max_iter + 1) * ACOPF_IPM_HISTORY_FIELDS,
              std::numeric_limits<double>::quiet_NaN());

  // ---- evaluation at the initial point ----------------------------------------
  double f = 0.0;
  st = acopf_eval_obj(model, v.x, B.f, as);
  if (st == ACOPF_OK) st = acopf_eval_grad(model, v.x, v.grad, as);
  if (st == ACOPF_OK) st = acopf_eval_jac_coo(model, v.x, v.jvals, as);
  if (st != ACOPF_OK) return st;
  e = acopf::launch_ipm_measure(v, v.x, v.s, v.cons, n, m, blocks, B.part, B.out + 2, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B.out, B.f, 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = fetch(4);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: initial point");
  f = hout[0];
  double theta = hout[2];
  const double theta_max = 1e4 * std::max(1.0, theta), theta_min = 1e-4 * std::max(1.0, theta);
  std::vector<std::pair<double, double>> filter{{theta_max, -INFINITY}};
  double mu = mu_init, dw_last = 0.0, res0 = INFINITY;
  double resto_exit = -1.0;  // the violation where the last restoration ended (-1: none yet)
  result->setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  int32_t status = ACOPF_IPM_MAX_ITER, k = 0;

  // Feasibility restoration (reading d10, the oracle's `restoration`): from
  // x, minimise 1/2 ||r||^2 - mu_R sum log gaps(x) + zeta/2 ||x - x_R||^2,
  // r = g(x) - clip(g(x)), by Gauss-Newton steps on M_cond's pattern (no
  // Hessian, D the 0/1 rows outside the box), until the filter accepts a
  // point with at most `reduction` times theta_k (returns 1) or the
  // violation stalls at the smallest barrier (returns 0: infeasible).  On
  // return x, s, cons, f and theta are those of the last point.
  auto restoration = [&](double mu, double theta_k, double reduction, int& code) -> acopf_status {
    double mu_r = mu;
    code = 0;
    auto slack = [&](const double* cons, double* sv, double* rv, double* wv) -> cudaError_t {
      cudaError_t err = acopf::launch_resto_slack(cons, B.lo_s, B.hi_s, m, sv, rv, wv, blocks,
                                                  B.part, B.out, s);
      if (err == cudaSuccess) err = fetch(2);
      return err;
    };
    e = slack(v.cons, v.s, B.r, B.sigma_s);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration");
    double th = hout[0], rr = hout[1];
    double best = th;
    int since = 0;
    e = cudaMemcpyAsync(B.xr, v.x, N * 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration");
    auto accepted = [&](bool& ok) -> acopf_status {  // the main filter's test at (x, s)
      acopf_status r = acopf_eval_obj(model, v.x, B.f, as);
      if (r != ACOPF_OK) return r;
      cudaError_t err =
          acopf::launch_ipm_measure(v, v.x, v.s, v.cons, n, m, blocks, B.part, B.out + 2, s);
      if (err == cudaSuccess) err = cudaMemcpyAsync(B.out, B.f, 8, cudaMemcpyDeviceToDevice, s);
      if (err == cudaSuccess) err = fetch(4);
      if (err != cudaSuccess) return cuda_fail(err, "acopf_ipm_solve: restoration");
      f = hout[0];
      theta = hout[2];
      const double pv = f - mu * hout[3];
      bool dominated = false;
      for (const auto& fe : filter)
        if (theta >= fe.first && pv >= fe.second) dominated = true;
      ok = theta <= reduction * theta_k && !dominated;
      return ACOPF_OK;
    };
    for (int it_r = 0; it_r < kRestoMaxIter; ++it_r) {
      bool ok = false;
      acopf_status r = accepted(ok);
      if (r != ACOPF_OK) return r;
      if (ok) {
        code = 1;
        return ACOPF_OK;
      }
      // Gauss-Newton step
      r = acopf_eval_jac_coo(model, v.x, v.jvals, as);
      if (r != ACOPF_OK) return r;
      const double zeta = std::sqrt(mu_r);
      e = acopf::launch_resto_grad(model->step, v.jvals, B.r, v.x, B.xr, B.xl, B.xu, mu_r, zeta,
                                   B.rhs, B.sigma_x, blocks, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(B.hvals, 0, size_t(L.nnzh) * 8, s);
      if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration step");
      r = acopf_assemble_condensed_kkt_csr(model, B.hvals, v.jvals, B.sigma_x, B.sigma_s, 0.0,
                                           0.0, B.kvals, as);
      int32_t bad = -1;
      if (r == ACOPF_OK) r = acopf_chol_factor(chol, B.kvals, 0.0, &bad, as);
      if (r != ACOPF_OK) return r;
      result->factorizations++;
      if (bad >= 0) break;  // (positive definite by construction; a failure ends as infeasible)
      r = acopf_chol_solve(chol, B.rhs, v.dx, as);
      if (r != ACOPF_OK) return r;
      e = acopf::launch_resto_dir(v.x, v.dx, B.rhs, B.xr, B.xl, B.xu, n, 0.99, blocks, B.part,
                                  B.out, s);
      if (e == cudaSuccess) e = fetch(4);
      if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration step");
      double alpha = hout[0];
      const double slope = hout[1];
      const double psi0 = 0.5 * rr - mu_r * hout[2] + 0.5 * zeta * hout[3];
      double rt = 0.0, tht = 0.0;
      bool step_ok = false;
      while (true) {
        e = acopf::launch_resto_trial(v.x, v.dx, B.xr, B.xl, B.xu, n, alpha, v.xt, blocks, B.part,
                                      B.out, s);
        if (e == cudaSuccess) e = fetch(2);
        if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration trial");
        const double lg = hout[0], pr = hout[1];
        r = acopf_eval_cons(model, v.xt, v.cons_t, as);
        if (r != ACOPF_OK) return r;
        e = slack(v.cons_t, v.st, nullptr, nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration trial");
        result->trial_points++;
        tht = hout[0];
        rt = hout[1];
        if (0.5 * rt - mu_r * lg + 0.5 * zeta * pr <= psi0 + 1e-4 * alpha * slope) {
          step_ok = true;
          break;
        }
        alpha *= 0.5;
        if (alpha < 1e-12) break;
      }
      if (!step_ok) {  // no decrease along the step: a smaller barrier, else infeasible
        if (mu_r <= kRestoMuMin) return ACOPF_OK;
        mu_r *= 0.1;
        since = 0;
        continue;
      }
      std::swap(v.x, v.xt);
      std::swap(v.s, v.st);
      std::swap(v.cons, v.cons_t);
      rr = rt;
      e = slack(v.cons, v.s, B.r, B.sigma_s);  // the violation and its rows at the new point
      if (e == cudaSuccess) e = cudaMemcpyAsync(B.xr, v.x, N * 8, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration update");
      if (tht < 0.99 * best) {
        best = tht;
        since = 0;
      } else if (++since >= kRestoStall) {  // stalled: a smaller barrier, else infeasible
        if (mu_r <= kRestoMuMin) return ACOPF_OK;
        mu_r *= 0.1;
        since = 0;
      }
    }
    bool ok = false;
    const acopf_status r = accepted(ok);
    if (r != ACOPF_OK) return r;
    code = ok ? 1 : 0;
    return ACOPF_OK;
  };

  for (k = 0; k <= max_iter; ++k) {
    set_iterate();
    double emu = 0.0;
    st = residual_pair(mu, res0, emu);
    if (st != ACOPF_OK) return st;
    record(k, 0, f);
    record(k, 1, res0);
    record(k, 2, mu);
    record(k, 3, theta);
    if (res0 <= tol) {
      status = ACOPF_IPM_CONVERGED;
      break;
    }
    if (k == max_iter) break;
    // monotone barrier update, possibly several times (the first test uses
    // E at mu from the pass above)
    for (bool first = true; mu > tol / 10.0; first = false) {
      if (!first) {
        st = residual(mu, emu);
        if (st != ACOPF_OK) return st;
      }
      if (emu > kKappaEps * mu) break;
      mu = std::max(tol / 10.0, std::min(kKappaMu * mu, std::pow(mu, kThetaMu)));
      filter.assign(1, {theta_max, -INFINITY});
    }
    const double tau = std::max(kTauMin, 1.0 - mu);
    // Newton right-hand side, Hessian of f - y'g
    e = acopf::launch_ipm_rhs(model->step, v, mu, blocks, s);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: right-hand side");
    st = acopf_eval_hess_coo(model, v.x, v.ym, 1.0, B.hvals, as);
    if (st != ACOPF_OK) return st;
    // inertia correction on delta_w
    double dw = 0.0;
    bool ok = false;
    for (int tries = 0; tries < kMaxInertiaTries; ++tries) {
      st = acopf_condense(model, &it, v.jvals, dw, 0.0, B.sigma_x, B.sigma_s, B.q_s, B.rhs, as);
      if (st == ACOPF_OK)
        st = acopf_assemble_condensed_kkt_csr(model, B.hvals, v.jvals, B.sigma_x, B.sigma_s, dw,
                                              0.0, B.kvals, as);
      int32_t bad = -1;
      if (st == ACOPF_OK) st = acopf_chol_factor(chol, B.kvals, 0.0, &bad, as);
      if (st != ACOPF_OK) return st;
      result->factorizations++;
      if (bad < 0) {
        ok = true;
        break;
      }
      if (dw == 0.0)
        dw = dw_last == 0.0 ? kDeltaW0 : std::max(kDeltaWMin, kKappaWMinus * dw_last);
      else
        dw *= dw_last == 0.0 ? kKappaWPlusBar : kKappaWPlus;
      if (dw > kDeltaWMax) break;
    }
    if (!ok) {
      status = ACOPF_IPM_INERTIA_FAILED;
      break;
    }
    if (dw > 0.0) dw_last = dw;
    st = acopf_chol_solve(chol, B.rhs, v.dx, as);
    if (st == ACOPF_OK)
      st = acopf_recover_step(model, &it, v.jvals, dw, 0.0, B.sigma_s, B.q_s, v.dx, v.ds, v.dy,
                              v.dzl_x, v.dzu_x, v.dzl_s, v.dzu_s, as);
    if (st != ACOPF_OK) return st;
    e = acopf::launch_ipm_dir(v, n, m, tau, mu, blocks, B.part, B.out, s);
    if (e == cudaSuccess) e = fetch(4);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: step bounds");
    const double a_max = hout[0], a_z = hout[1], gphi = hout[2];
    const double phi = f - mu * hout[3];
    double alpha_min = kGammaTheta;
    if (gphi < 0.0)
      alpha_min = std::min({alpha_min, kGammaPhi * theta / (-gphi),
                            kDelta * std::pow(theta, kSTheta) / std::pow(-gphi, kSPhi)});
    alpha_min *= kAlphaMinFrac;
    // filter line search: 1 (f-type), 2 (h-type) or 0 for a trial point of
    // violation tht_ and barrier objective pht_ at step a
    auto acceptable = [&](double tht_, double pht_, double a) -> int {
      for (const auto& fe : filter)
        if (tht_ >= fe.first && pht_ >= fe.second) return 0;
      const bool switching =
          gphi < 0.0 && a * std::pow(-gphi, kSPhi) > kDelta * std::pow(theta, kSTheta);
      if (switching && theta <= theta_min) return pht_ <= phi + kEtaPhi * a * gphi ? 1 : 0;
      if (tht_ <= (1.0 - kGammaTheta) * theta || pht_ <= phi - kGammaPhi * theta) return 2;
      return 0;
    };
    // the trial point x + a d, s + a d (direction of w): objective, constraints, measures
    auto trial = [&](const acopf::IpmVec& w, double a) -> acopf_status {
      cudaError_t err = acopf::launch_ipm_trial(w, n, m, a, blocks, s);
      if (err != cudaSuccess) return cuda_fail(err, "acopf_ipm_solve: trial point");
      acopf_status r = acopf_eval_obj(model, v.xt, B.ft, as);
      if (r == ACOPF_OK) r = acopf_eval_cons(model, v.xt, v.cons_t, as);
      if (r != ACOPF_OK) return r;
      err = acopf::launch_ipm_measure(v, v.xt, v.st, v.cons_t, n, m, blocks, B.part, B.out + 2, s);
      if (err == cudaSuccess) err = cudaMemcpyAsync(B.out, B.ft, 8, cudaMemcpyDeviceToDevice, s);
      if (err == cudaSuccess) err = fetch(4);
      if (err != cudaSuccess) return cuda_fail(err, "acopf_ipm_solve: trial measures");
      result->trial_points++;
      return ACOPF_OK;
    };
    // the second-order correction's direction in w (the iterate's vectors,
    // the correction's step buffers)
    acopf::IpmVec w = v;
    w.dx = B.dx2; w.ds = B.ds2; w.dy = B.dy2; w.dzl_x = B.dzl_x2; w.dzu_x = B.dzu_x2;
    w.dzl_s = B.dzl_s2; w.dzu_s = B.dzu_s2;
    acopf_iterate it_soc = it;
    it_soc.p_y = B.py_soc;
    double alpha = a_max, alpha_z = a_z, ft = 0.0, tht = 0.0, pht = 0.0;
    int accepted = 0;  // 1: f-type, 2: h-type
    bool soc_step = false;
    for (int b = 0; b < kMaxBacktracks; ++b) {
      st = trial(v, alpha);
      if (st != ACOPF_OK) return st;
      ft = hout[0];
      tht = hout[2];
      pht = ft - mu * hout[3];
      accepted = acceptable(tht, pht, alpha);
      if (accepted) break;
      if (b == 0 && tht >= theta) {
        // second-order correction: c_soc = alpha c(x_k) + c(x_trial), then
        // alpha_soc c_soc + c(x_soc) while the violation keeps falling; the
        // corrected point's tests use the first trial step alpha_{k,0}
        double th_old = theta, a_c = alpha;
        const double *c0 = v.cons, *s0 = v.s;
        for (int q = 0; q < kSocMax && !accepted; ++q) {
          e = acopf::launch_soc_rhs(B.c_soc, B.py_soc, c0, s0, v.cons_t, v.st, a_c, m, blocks, s);
          if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: second-order correction");
          c0 = s0 = nullptr;
          st = acopf_condense(model, &it_soc, v.jvals, dw, 0.0, B.sigma_x, B.sigma_s, B.q_s, B.rhs,
                              as);
          if (st == ACOPF_OK) st = acopf_chol_solve(chol, B.rhs, w.dx, as);
          if (st == ACOPF_OK)
            st = acopf_recover_step(model, &it_soc, v.jvals, dw, 0.0, B.sigma_s, B.q_s, w.dx,
                                    w.ds, w.dy, w.dzl_x, w.dzu_x, w.dzl_s, w.dzu_s, as);
          if (st != ACOPF_OK) return st;
          e = acopf::launch_ipm_dir(w, n, m, tau, mu, blocks, B.part, B.out, s);
          if (e == cudaSuccess) e = fetch(2);
          if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: second-order correction");
          const double a_soc = hout[0], az_soc = hout[1];
          st = trial(w, a_soc);
          if (st != ACOPF_OK) return st;
          const double fs = hout[0], ths = hout[2], phs = fs - mu * hout[3];
          accepted = acceptable(ths, phs, a_max);
          if (accepted) {
            soc_step = true;
            alpha = a_soc;
            alpha_z = az_soc;
            ft = fs;
            tht = ths;
            break;
          }
          if (ths > kKappaSoc * th_old) break;
          th_old = ths;
          a_c = a_soc;
        }
        if (accepted) break;
      }
      alpha *= 0.5;
      if (alpha < alpha_min) break;
    }
    if (!accepted) {  // feasibility restoration from the current point
      filter.push_back({(1.0 - kGammaTheta) * theta, phi - kGammaPhi * theta});
      // back without getting below the last restoration's exit: demand
      // (nearly) feasibility this time, which an infeasible network cannot give
      const double red =
          resto_exit >= 0.0 && theta >= resto_exit ? kRestoReductionRepeat : kRestoReduction;
      int code = 0;
      st = restoration(mu, theta, red, code);
      if (st != ACOPF_OK) return st;
      resto_exit = theta;
      record(k, 4, 0.0);
      record(k, 5, 0.0);
      record(k, 6, dw);
      if (code == 0) {
        status = ACOPF_IPM_INFEASIBLE;
        break;
      }
      // multipliers restart: y = 0, bound duals on the central path
      e = acopf::launch_resto_duals(v, n, m, mu, blocks, s);
      if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: restoration duals");
      st = acopf_eval_grad(model, v.x, v.grad, as);
      if (st == ACOPF_OK) st = acopf_eval_jac_coo(model, v.x, v.jvals, as);
      if (st != ACOPF_OK) return st;
      continue;
    }
    if (accepted == 2)
      filter.push_back({(1.0 - kGammaTheta) * theta, phi - kGammaPhi * theta});
    std::swap(v.x, v.xt);
    std::swap(v.s, v.st);
    std::swap(v.cons, v.cons_t);
    f = ft;
    theta = tht;
    {
      acopf::IpmVec va = v;  // the step taken: the correction's when it was accepted
      if (soc_step) {
        va.dx = B.dx2; va.ds = B.ds2; va.dy = B.dy2; va.dzl_x = B.dzl_x2; va.dzu_x = B.dzu_x2;
        va.dzl_s = B.dzl_s2; va.dzu_s = B.dzu_s2;
      }
      e = acopf::launch_ipm_accept(va, n, m, alpha, alpha_z, mu, kKappaSigma, blocks, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: update");
    st = acopf_eval_grad(model, v.x, v.grad, as);
    if (st == ACOPF_OK) st = acopf_eval_jac_coo(model, v.x, v.jvals, as);
    if (st != ACOPF_OK) return st;
    record(k, 4, alpha);
    record(k, 5, alpha_z);
    record(k, 6, dw);
  }
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && x_out) e = cudaMemcpy(x_out, v.x, N * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_ipm_solve: result");
  result->status = status;
  result->iterations = std::min(k, max_iter);
  result->objective = f;
  result->residual = res0;
  result->mu = mu;
  result->seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return ACOPF_OK;
}

acopf_status acopf_ipm_solve(acopf_model* model, const acopf_ipm_options* options, double* x_out,
                             double* history, acopf_ipm_result* result, acopf_stream stream) {
  return ipm_solve_impl(model, nullptr, options, x_out, history, result, stream);
}

acopf_status acopf_ipm_solve_chol(acopf_model* model, acopf_chol* chol,
                                  const acopf_ipm_options* options, double* x_out,
                                  double* history, acopf_ipm_result* result,
                                  acopf_stream stream) {
  if (!model || !chol) return fail(ACOPF_E_INVALID_ARG, "acopf_ipm_solve_chol: null pointer");
  if (acopf::chol_model(chol) != model)
    return fail(ACOPF_E_INVALID_ARG,
                "acopf_ipm_solve_chol: the Cholesky object was made for another model");
  return ipm_solve_impl(model, chol, options, x_out, history, result, stream);
}

}  // extern "C"
