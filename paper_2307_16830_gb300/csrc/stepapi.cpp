// Entry points of the condensation around M_cond and the step recovery
// (acopf_condense, acopf_recover_step).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "host_internal.h"

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

namespace {

// Builds the Jacobian's row and column lists (ascending slot in each) and
// the row scratch on the model's device, once.
acopf_status ensure_step(acopf_model* m) {
  if (m->step_arena) return ACOPF_OK;
  const acopf::HostModel& hm = m->hm;
  const int32_t n = hm.L.n, mm = hm.L.m;
  const size_t nnz = hm.jrows.size();
  std::vector<int32_t> rp(size_t(mm) + 1, 0), cp(size_t(n) + 1, 0);
  std::vector<int32_t> rslot(nnz), rcol(nnz), cslot(nnz), crow(nnz);
  for (size_t k = 0; k < nnz; ++k) {
    rp[size_t(hm.jrows[k]) + 1]++;
    cp[size_t(hm.jcols[k]) + 1]++;
  }
  for (int32_t r = 0; r < mm; ++r) rp[size_t(r) + 1] += rp[size_t(r)];
  for (int32_t c = 0; c < n; ++c) cp[size_t(c) + 1] += cp[size_t(c)];
  std::vector<int32_t> rnext(rp.begin(), rp.end() - 1), cnext(cp.begin(), cp.end() - 1);
  for (size_t k = 0; k < nnz; ++k) {
    const int32_t r = hm.jrows[k], c = hm.jcols[k];
    const int32_t a = rnext[size_t(r)]++, b = cnext[size_t(c)]++;
    rslot[size_t(a)] = int32_t(k);
    rcol[size_t(a)] = c;
    cslot[size_t(b)] = int32_t(k);
    crow[size_t(b)] = r;
  }
  acopf::ArenaPlan p;
  const size_t o_rp = p.take<int32_t>(rp.size()), o_rs = p.take<int32_t>(nnz);
  const size_t o_rc = p.take<int32_t>(nnz), o_cp = p.take<int32_t>(cp.size());
  const size_t o_cs = p.take<int32_t>(nnz), o_cr = p.take<int32_t>(nnz);
  const size_t o_w = p.take<double>(size_t(mm));
  int sms = 0;
  cudaError_t ae = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  if (ae != cudaSuccess) return cuda_fail(ae, "acopf_condense: device attribute");
  const int res_blocks = acopf::residual_blocks(sms > 0 ? sms : 1);
  const size_t o_rp2 = p.take<double>(acopf::kResPart * size_t(res_blocks));
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, p.off);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_condense: cudaMalloc");
  char* base = static_cast<char*>(arena);
  auto up = [&](size_t off, const std::vector<int32_t>& v) {
    if (e == cudaSuccess && !v.empty())
      e = cudaMemcpy(base + off, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
  };
  up(o_rp, rp);
  up(o_rs, rslot);
  up(o_rc, rcol);
  up(o_cp, cp);
  up(o_cs, cslot);
  up(o_cr, crow);
  if (e != cudaSuccess) {
    cudaFree(arena);
    return cuda_fail(e, "acopf_condense: upload");
  }
  acopf::DevStep& st = m->step;
  st.n = n;
  st.m = mm;
  st.jr_ptr = reinterpret_cast<const int32_t*>(base + o_rp);
  st.jr_slot = reinterpret_cast<const int32_t*>(base + o_rs);
  st.jr_col = reinterpret_cast<const int32_t*>(base + o_rc);
  st.jt_ptr = reinterpret_cast<const int32_t*>(base + o_cp);
  st.jt_slot = reinterpret_cast<const int32_t*>(base + o_cs);
  st.jt_row = reinterpret_cast<const int32_t*>(base + o_cr);
  st.w = reinterpret_cast<double*>(base + o_w);
  st.res_part = reinterpret_cast<double*>(base + o_rp2);
  st.res_blocks = res_blocks;
  m->step_arena = arena;
  return ACOPF_OK;
}

acopf_status check_iterate(const acopf_iterate* it, acopf::StepIterate& out, const char* where) {
  if (!it) return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": null iterate");
  const double* f[] = {it->x,    it->s,      it->xl,     it->xu,     it->sl,     it->su,
                       it->zl_x, it->zu_x,   it->zl_s,   it->zu_s,   it->p_x,    it->p_s,
                       it->p_y,  it->p_zl_x, it->p_zu_x, it->p_zl_s, it->p_zu_s};
  for (const double* q : f)
    if (!q) return fail(ACOPF_E_INVALID_ARG, std::string(where) + ": null iterate array");
  out = acopf::StepIterate{it->x,    it->s,    it->xl,   it->xu,     it->sl,     it->su,
                           it->zl_x, it->zu_x, it->zl_s, it->zu_s,   it->p_x,    it->p_s,
                           it->p_y,  it->p_zl_x, it->p_zu_x, it->p_zl_s, it->p_zu_s};
  return ACOPF_OK;
}

}  // namespace

namespace acopf {

acopf_status step_lists(acopf_model* m) { return ensure_step(m); }
void free_step(acopf_model* m) {
  if (m->step_arena) cudaFree(m->step_arena);
  m->step_arena = nullptr;
}
}  // namespace acopf

extern "C" {

acopf_status acopf_condense(acopf_model* model, const acopf_iterate* it, const double* jvals,
                            double delta_w, double delta_c, double* sigma_x, double* sigma_s,
                            double* q_s, double* rhs, acopf_stream stream) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "acopf_condense: null model");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "model was created host-only (device = -1)");
  acopf::StepIterate si;
  acopf_status st = check_iterate(it, si, "acopf_condense");
  if (st != ACOPF_OK) return st;
  if (!jvals || !sigma_x || !sigma_s || !q_s || !rhs)
    return fail(ACOPF_E_INVALID_ARG, "acopf_condense: null pointer");
  st = acopf::check_eval_scalars(1.0, delta_w, delta_c);
  if (st != ACOPF_OK) return st;
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_condense");
  st = ensure_step(model);
  if (st != ACOPF_OK) return st;
  cudaError_t e = acopf::launch_condense(model->step, si, jvals, delta_w, delta_c, sigma_x,
                                         sigma_s, q_s, rhs, model->dm.pdl != 0,
                                         reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "acopf_condense");
  return ACOPF_OK;
}

acopf_status acopf_recover_step(acopf_model* model, const acopf_iterate* it, const double* jvals,
                                double delta_w, double delta_c, const double* sigma_s,
                                const double* q_s, const double* dx, double* ds, double* dy,
                                double* dzl_x, double* dzu_x, double* dzl_s, double* dzu_s,
                                acopf_stream stream) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "acopf_recover_step: null model");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "model was created host-only (device = -1)");
  acopf::StepIterate si;
  acopf_status st = check_iterate(it, si, "acopf_recover_step");
  if (st != ACOPF_OK) return st;
  if (!jvals || !sigma_s || !q_s || !dx || !ds || !dy || !dzl_x || !dzu_x || !dzl_s || !dzu_s)
    return fail(ACOPF_E_INVALID_ARG, "acopf_recover_step: null pointer");
  st = acopf::check_eval_scalars(1.0, delta_w, delta_c);
  if (st != ACOPF_OK) return st;
  DeviceScope dsc(model->device);
  if (dsc.error() != cudaSuccess) return cuda_fail(dsc.error(), "acopf_recover_step");
  st = ensure_step(model);
  if (st != ACOPF_OK) return st;
  cudaError_t e = acopf::launch_recover(model->step, si, jvals, delta_w, delta_c, sigma_s, q_s,
                                        dx, ds, dy, dzl_x, dzu_x, dzl_s, dzu_s,
                                        reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "acopf_recover_step");
  return ACOPF_OK;
}

acopf_status acopf_kkt_residual(acopf_model* model, const acopf_iterate* it, const double* y,
                                const double* grad, const double* cons, const double* jvals,
                                double mu, double* out, acopf_stream stream) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "acopf_kkt_residual: null model");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "model was created host-only (device = -1)");
  if (!it || !it->x || !it->s || !it->xl || !it->xu || !it->sl || !it->su || !it->zl_x ||
      !it->zu_x || !it->zl_s || !it->zu_s)
    return fail(ACOPF_E_INVALID_ARG, "acopf_kkt_residual: null iterate array");
  if (!y || !grad || !cons || !jvals || !out)
    return fail(ACOPF_E_INVALID_ARG, "acopf_kkt_residual: null pointer");
  if (!std::isfinite(mu) || mu < 0.0)
    return fail(ACOPF_E_INVALID_ARG, "acopf_kkt_residual: mu must be finite and >= 0");
  DeviceScope dsc(model->device);
  if (dsc.error() != cudaSuccess) return cuda_fail(dsc.error(), "acopf_kkt_residual");
  acopf_status st = ensure_step(model);
  if (st != ACOPF_OK) return st;
  acopf::StepIterate si{};
  si.x = it->x;
  si.s = it->s;
  si.xl = it->xl;
  si.xu = it->xu;
  si.sl = it->sl;
  si.su = it->su;
  si.zl_x = it->zl_x;
  si.zu_x = it->zu_x;
  si.zl_s = it->zl_s;
  si.zu_s = it->zu_s;
  cudaError_t e = acopf::launch_kkt_residual(model->step, si, y, grad, cons, jvals, mu, out,
                                             reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "acopf_kkt_residual");
  return ACOPF_OK;
}

}  // extern "C"
