// extern "C" entry points of libacopf (declared in include/acopf.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "host_internal.h"

namespace acopf {

thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

acopf_status fail(acopf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

acopf_status cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(e == cudaErrorMemoryAllocation ? ACOPF_E_OOM : ACOPF_E_CUDA, m);
}

acopf_status check_eval_scalars(double obj_weight, double delta_w, double delta_c) {
  if (!(delta_w >= 0.0) || !(delta_c >= 0.0) || !std::isfinite(delta_w) || !std::isfinite(delta_c))
    return fail(ACOPF_E_INVALID_ARG, "delta_w and delta_c must be finite and >= 0");
  if (!std::isfinite(obj_weight)) return fail(ACOPF_E_INVALID_ARG, "obj_weight must be finite");
  return ACOPF_OK;
}

void append_items(const Layout& L, int32_t inst, std::vector<int4>& p1, std::vector<int4>& p2) {
  const int nbb = ceil_div(L.nl, kBranchThreads);
  const int nbi = ceil_div(L.nb, kBusThreads);
  const int ngb = std::max(1, ceil_div(L.ng, kGenThreads));
  for (int k = 0; k < nbb; ++k) p1.push_back(make_int4(inst, 0, k, nbb));
  for (int k = 0; k < nbi; ++k) p1.push_back(make_int4(inst, 1, k, nbi));
  for (int k = 0; k < ngb; ++k) p1.push_back(make_int4(inst, 2, k, ngb));
  const int nbr = ceil_div(L.nrc, kBusThreads);  // bus-row blocks (row chunks)
  for (int k = 0; k < nbr; ++k) p2.push_back(make_int4(inst, 3, k, nbr));
}

}  // namespace acopf

namespace {

using acopf::ArenaPlan;
using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;
using acopf::g_last_error;

acopf_status check_device_model(const acopf_model* m) {
  if (!m) return fail(ACOPF_E_INVALID_ARG, "null model");
  if (m->device < 0) return fail(ACOPF_E_NO_DEVICE, "model was created host-only (device = -1)");
  return ACOPF_OK;
}

acopf_status run_eval(const acopf_model* m, unsigned what, const acopf::EvalArgs& a,
                      acopf_stream stream, const char* name) {
  acopf_status st = check_device_model(m);
  if (st != ACOPF_OK) return st;
  DeviceScope ds(m->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), name);
  cudaError_t e = acopf::launch_eval(m->dm, what, a, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, name);
  return ACOPF_OK;
}

acopf::EvalArgs empty_args() {
  acopf::EvalArgs a;
  std::memset(&a, 0, sizeof(a));
  a.obj_weight = 1.0;
  return a;
}

}  // namespace

extern "C" {

const char* acopf_status_string(acopf_status s) {
  switch (s) {
    case ACOPF_OK:
      return "ACOPF_OK";
    case ACOPF_E_INVALID_ARG:
      return "ACOPF_E_INVALID_ARG";
    case ACOPF_E_BAD_MODEL:
      return "ACOPF_E_BAD_MODEL";
    case ACOPF_E_CUDA:
      return "ACOPF_E_CUDA";
    case ACOPF_E_OOM:
      return "ACOPF_E_OOM";
    case ACOPF_E_BUDGET:
      return "ACOPF_E_BUDGET";
    case ACOPF_E_TIMEOUT:
      return "ACOPF_E_TIMEOUT";
    case ACOPF_E_BUSY:
      return "ACOPF_E_BUSY";
    case ACOPF_E_NO_DEVICE:
      return "ACOPF_E_NO_DEVICE";
    default:
      return "ACOPF_E_UNKNOWN";
  }
}

const char* acopf_last_error(void) { return g_last_error.c_str(); }

acopf_status acopf_model_create(const acopf_buses* buses, const acopf_branches* branches,
                                const acopf_gens* gens, int device, acopf_model** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (device < -1) return fail(ACOPF_E_INVALID_ARG, "device must be >= -1");
  acopf_model* m = new (std::nothrow) acopf_model;
  if (!m) return fail(ACOPF_E_OOM, "host allocation failed");
  std::string err;
  acopf_status st;
  try {
    st = acopf::build_host_model(buses, branches, gens, m->hm, err);
  } catch (const std::bad_alloc&) {
    st = ACOPF_E_OOM;
    err = "host allocation failed";
  }
  if (st != ACOPF_OK) {
    delete m;
    return fail(st, err);
  }
  m->device = device;
  const acopf::HostModel& hm = m->hm;
  const acopf::Layout& L = hm.L;
  acopf::DevModel& dm = m->dm;
  dm.L = L;
  dm.has_shunt = 0;
  for (int32_t i = 0; i < L.nb; ++i)
    if (hm.Gs[i] != 0.0 || hm.Bs[i] != 0.0) dm.has_shunt = 1;
  dm.pdl = 1;
  if (device < 0) {
    *out = m;
    return ACOPF_OK;
  }

  DeviceScope ds(device);
  if (ds.error() != cudaSuccess) {
    delete m;
    return cuda_fail(ds.error(), "acopf_model_create: cudaSetDevice");
  }
  const size_t nl = L.nl, nb = L.nb, ng = L.ng, n = L.n;
  ArenaPlan p;
  const size_t o_f = p.take<int32_t>(nl), o_t = p.take<int32_t>(nl);
  const size_t o_coef = p.take<double>(acopf::NCOEF * nl);
  const size_t o_Pd = p.take<double>(nb), o_Qd = p.take<double>(nb);
  const size_t o_Gs = p.take<double>(nb), o_Bs = p.take<double>(nb);
  const size_t o_ref = p.take<int32_t>(nb);
  const size_t o_aptr = p.take<int32_t>(nb + 1);
  const size_t o_aidx = p.take<int32_t>(2 * nl);
  const size_t o_snbr = p.take<int32_t>(2 * nl), o_soa = p.take<int32_t>(2 * nl);
  const size_t o_pord = p.take<int32_t>(nb), o_psp = p.take<int32_t>(nb + 1);
  const size_t o_gptr = p.take<int32_t>(nb + 1), o_gat = p.take<int32_t>(ng);
  const size_t o_gbus = p.take<int32_t>(ng);
  const size_t o_bptr = p.take<int32_t>(nb + 1), o_bidx = p.take<int32_t>(ng + 2 * nl);
  const size_t o_c2 = p.take<double>(ng), o_c1 = p.take<double>(ng), o_c0 = p.take<double>(ng);
  const size_t o_krp = p.take<int32_t>(n + 1);
  const size_t o_brow = p.take<int4>(nl), o_bcnt = p.take<uint32_t>(nl);
  const size_t o_rch = p.take<int4>(2 * size_t(L.nrc));
  const acopf::WorkspacePlan wsp = acopf::workspace_plan(L);
  const size_t o_ws = p.take<char>(wsp.bytes);
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, p.off);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "acopf_model_create: cudaMalloc");
  }
  m->arena = arena;
  m->arena_bytes = p.off;
  char* base = static_cast<char*>(arena);
  auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice);
  };
  e = cudaSuccess;
  if (e == cudaSuccess) e = up(o_f, hm.f.data(), nl * 4);
  if (e == cudaSuccess) e = up(o_t, hm.t.data(), nl * 4);
  if (e == cudaSuccess) e = up(o_coef, hm.coef.data(), acopf::NCOEF * nl * 8);
  if (e == cudaSuccess) e = up(o_Pd, hm.Pd.data(), nb * 8);
  if (e == cudaSuccess) e = up(o_Qd, hm.Qd.data(), nb * 8);
  if (e == cudaSuccess) e = up(o_Gs, hm.Gs.data(), nb * 8);
  if (e == cudaSuccess) e = up(o_Bs, hm.Bs.data(), nb * 8);
  if (e == cudaSuccess) e = up(o_ref, hm.ref_row.data(), nb * 4);
  if (e == cudaSuccess) e = up(o_aptr, hm.arc_ptr.data(), (nb + 1) * 4);
  if (e == cudaSuccess) e = up(o_aidx, hm.arcs_by_idx.data(), 2 * nl * 4);
  if (e == cudaSuccess) e = up(o_snbr, hm.slot_nbr.data(), 2 * nl * 4);
  if (e == cudaSuccess) e = up(o_soa, hm.slot_of_arc.data(), 2 * nl * 4);
  if (e == cudaSuccess) e = up(o_gptr, hm.gen_ptr.data(), (nb + 1) * 4);
  if (e == cudaSuccess) e = up(o_gat, hm.gens_at.data(), ng * 4);
  if (e == cudaSuccess) e = up(o_gbus, hm.gbus.data(), ng * 4);
  if (e == cudaSuccess) e = up(o_c2, hm.c2.data(), ng * 8);
  if (e == cudaSuccess) e = up(o_c1, hm.c1.data(), ng * 8);
  if (e == cudaSuccess) e = up(o_c0, hm.c0.data(), ng * 8);
  if (e == cudaSuccess) e = up(o_krp, hm.krowptr.data(), (n + 1) * 4);
  if (e == cudaSuccess) e = up(o_brow, hm.brow.data(), nl * 16);
  if (e == cudaSuccess) e = up(o_bcnt, hm.bcnt.data(), nl * 4);
  if (e == cudaSuccess) e = up(o_rch, hm.rchunk.data(), hm.rchunk.size() * 4);
  if (e == cudaSuccess) e = up(o_bptr, hm.pbal_ptr.data(), (nb + 1) * 4);
  if (e == cudaSuccess) e = up(o_pord, hm.porder.data(), nb * 4);
  if (e == cudaSuccess) e = up(o_psp, hm.pslot_ptr.data(), (nb + 1) * 4);
  if (e == cudaSuccess) e = up(o_bidx, hm.bal_idx.data(), (ng + 2 * nl) * 4);
  if (e == cudaSuccess) e = cudaMemset(base + o_ws, 0, wsp.bytes);  // counters start at zero
  if (e != cudaSuccess) {
    cudaFree(arena);
    delete m;
    return cuda_fail(e, "acopf_model_create: upload");
  }
  dm.f = reinterpret_cast<const int32_t*>(base + o_f);
  dm.t = reinterpret_cast<const int32_t*>(base + o_t);
  dm.coef = reinterpret_cast<const double*>(base + o_coef);
  dm.Pd = reinterpret_cast<const double*>(base + o_Pd);
  dm.Qd = reinterpret_cast<const double*>(base + o_Qd);
  dm.Gs = reinterpret_cast<const double*>(base + o_Gs);
  dm.Bs = reinterpret_cast<const double*>(base + o_Bs);
  dm.ref_row = reinterpret_cast<const int32_t*>(base + o_ref);
  dm.arc_ptr = reinterpret_cast<const int32_t*>(base + o_aptr);
  dm.arcs_by_idx = reinterpret_cast<const int32_t*>(base + o_aidx);
  dm.porder = reinterpret_cast<const int32_t*>(base + o_pord);
  dm.pslot_ptr = reinterpret_cast<const int32_t*>(base + o_psp);
  dm.slot_nbr = reinterpret_cast<const int32_t*>(base + o_snbr);
  dm.slot_of_arc = reinterpret_cast<const int32_t*>(base + o_soa);
  dm.gen_ptr = reinterpret_cast<const int32_t*>(base + o_gptr);
  dm.gens_at = reinterpret_cast<const int32_t*>(base + o_gat);
  dm.gbus = reinterpret_cast<const int32_t*>(base + o_gbus);
  dm.c2 = reinterpret_cast<const double*>(base + o_c2);
  dm.c1 = reinterpret_cast<const double*>(base + o_c1);
  dm.c0 = reinterpret_cast<const double*>(base + o_c0);
  dm.krowptr = reinterpret_cast<const int32_t*>(base + o_krp);
  dm.brow = reinterpret_cast<const int4*>(base + o_brow);
  dm.bcnt = reinterpret_cast<const uint32_t*>(base + o_bcnt);
  dm.rchunk = reinterpret_cast<const int4*>(base + o_rch);
  dm.pbal_ptr = reinterpret_cast<const int32_t*>(base + o_bptr);
  dm.bal_idx = reinterpret_cast<const int32_t*>(base + o_bidx);
  acopf::bind_workspace(dm, base + o_ws, wsp);
  *out = m;
  return ACOPF_OK;
}

static void destroy_profile_events(acopf_model* m);

acopf_status acopf_model_destroy(acopf_model* model) {
  if (!model) return ACOPF_OK;
  if (model->device >= 0) {
    DeviceScope ds(model->device);
    destroy_profile_events(model);
    acopf::free_step(model);
    if (model->arena) cudaFree(model->arena);
    if (model->stage) cudaFree(model->stage);
  }
  delete model;
  return ACOPF_OK;
}

acopf_status acopf_model_dims(const acopf_model* model, int64_t* n, int64_t* m, int64_t* nnz_jac,
                              int64_t* nnz_hess, int64_t* nnz_kkt, int64_t* device_bytes) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "null model");
  const acopf::Layout& L = model->hm.L;
  if (n) *n = L.n;
  if (m) *m = L.m;
  if (nnz_jac) *nnz_jac = L.nnzj;
  if (nnz_hess) *nnz_hess = L.nnzh;
  if (nnz_kkt) *nnz_kkt = L.nnzk;
  if (device_bytes) *device_bytes = int64_t(model->arena_bytes + model->stage_bytes);
  return ACOPF_OK;
}

acopf_status acopf_model_counts(const acopf_model* model, int32_t* n_bus, int32_t* n_branch,
                                int32_t* n_gen, int32_t* n_ref) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "null model");
  const acopf::Layout& L = model->hm.L;
  if (n_bus) *n_bus = L.nb;
  if (n_branch) *n_branch = L.nl;
  if (n_gen) *n_gen = L.ng;
  if (n_ref) *n_ref = L.nref;
  return ACOPF_OK;
}

acopf_status acopf_bounds(const acopf_model* model, double* xl, double* xu, double* gl,
                          double* gu) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "null model");
  const acopf::HostModel& hm = model->hm;
  if (xl) std::memcpy(xl, hm.xl.data(), hm.xl.size() * 8);
  if (xu) std::memcpy(xu, hm.xu.data(), hm.xu.size() * 8);
  if (gl) std::memcpy(gl, hm.gl.data(), hm.gl.size() * 8);
  if (gu) std::memcpy(gu, hm.gu.data(), hm.gu.size() * 8);
  return ACOPF_OK;
}

acopf_status acopf_jac_structure(const acopf_model* model, int32_t* rows, int32_t* cols) {
  if (!model || !rows || !cols) return fail(ACOPF_E_INVALID_ARG, "null argument");
  std::memcpy(rows, model->hm.jrows.data(), model->hm.jrows.size() * 4);
  std::memcpy(cols, model->hm.jcols.data(), model->hm.jcols.size() * 4);
  return ACOPF_OK;
}

acopf_status acopf_hess_structure(const acopf_model* model, int32_t* rows, int32_t* cols) {
  if (!model || !rows || !cols) return fail(ACOPF_E_INVALID_ARG, "null argument");
  std::memcpy(rows, model->hm.hrows.data(), model->hm.hrows.size() * 4);
  std::memcpy(cols, model->hm.hcols.data(), model->hm.hcols.size() * 4);
  return ACOPF_OK;
}

acopf_status acopf_kkt_structure(const acopf_model* model, int32_t* rowptr, int32_t* colind) {
  if (!model || !rowptr || !colind) return fail(ACOPF_E_INVALID_ARG, "null argument");
  std::memcpy(rowptr, model->hm.krowptr.data(), model->hm.krowptr.size() * 4);
  std::memcpy(colind, model->hm.kcolind.data(), model->hm.kcolind.size() * 4);
  return ACOPF_OK;
}

acopf_status acopf_eval_obj(const acopf_model* model, const double* x, double* f_dev,
                            acopf_stream stream) {
  if (!x || !f_dev) return fail(ACOPF_E_INVALID_ARG, "acopf_eval_obj: null pointer");
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.f = f_dev;
  return run_eval(model, acopf::OUT_OBJ, a, stream, "acopf_eval_obj");
}

acopf_status acopf_eval_grad(const acopf_model* model, const double* x, double* grad,
                             acopf_stream stream) {
  if (!x || !grad) return fail(ACOPF_E_INVALID_ARG, "acopf_eval_grad: null pointer");
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.grad = grad;
  return run_eval(model, acopf::OUT_GRAD, a, stream, "acopf_eval_grad");
}

acopf_status acopf_eval_cons(const acopf_model* model, const double* x, double* cons,
                             acopf_stream stream) {
  if (!x || !cons) return fail(ACOPF_E_INVALID_ARG, "acopf_eval_cons: null pointer");
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.cons = cons;
  return run_eval(model, acopf::OUT_CONS, a, stream, "acopf_eval_cons");
}

acopf_status acopf_eval_jac_coo(const acopf_model* model, const double* x, double* jvals,
                                acopf_stream stream) {
  if (!x || !jvals) return fail(ACOPF_E_INVALID_ARG, "acopf_eval_jac_coo: null pointer");
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.jvals = jvals;
  return run_eval(model, acopf::OUT_JAC, a, stream, "acopf_eval_jac_coo");
}

acopf_status acopf_eval_hess_coo(const acopf_model* model, const double* x, const double* y,
                                 double obj_weight, double* hvals, acopf_stream stream) {
  if (!x || !y || !hvals) return fail(ACOPF_E_INVALID_ARG, "acopf_eval_hess_coo: null pointer");
  if (!std::isfinite(obj_weight)) return fail(ACOPF_E_INVALID_ARG, "obj_weight must be finite");
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.y = y;
  a.obj_weight = obj_weight;
  a.hvals = hvals;
  return run_eval(model, acopf::OUT_HESS, a, stream, "acopf_eval_hess_coo");
}

acopf_status acopf_assemble_condensed_kkt_csr(const acopf_model* model, const double* hvals,
                                              const double* jvals, const double* sigma_x,
                                              const double* sigma_s, double delta_w,
                                              double delta_c, double* kvals,
                                              acopf_stream stream) {
  if (!hvals || !jvals || !sigma_x || !sigma_s || !kvals)
    return fail(ACOPF_E_INVALID_ARG, "acopf_assemble_condensed_kkt_csr: null pointer");
  if (!(delta_w >= 0.0) || !(delta_c >= 0.0) || !std::isfinite(delta_w) || !std::isfinite(delta_c))
    return fail(ACOPF_E_INVALID_ARG, "delta_w and delta_c must be finite and >= 0");
  acopf_status st = check_device_model(model);
  if (st != ACOPF_OK) return st;
  acopf::EvalArgs a = empty_args();
  a.hvals_in = hvals;
  a.jvals_in = jvals;
  a.sigma_x = sigma_x;
  a.sigma_s = sigma_s;
  a.delta_w = delta_w;
  a.delta_c = delta_c;
  a.kvals = kvals;
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_assemble_condensed_kkt_csr");
  cudaError_t e = acopf::launch_assemble(model->dm, a, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "acopf_assemble_condensed_kkt_csr");
  return ACOPF_OK;
}

acopf_status acopf_eval_assemble(const acopf_model* model, const double* x, const double* y,
                                 double obj_weight, const double* sigma_x, const double* sigma_s,
                                 double delta_w, double delta_c, double* f_dev, double* grad,
                                 double* cons, double* jvals, double* hvals, double* kvals,
                                 acopf_stream stream) {
  if (!x || !y || !sigma_x || !sigma_s || !f_dev || !grad || !cons || !jvals || !hvals || !kvals)
    return fail(ACOPF_E_INVALID_ARG, "acopf_eval_assemble: null pointer");
  acopf_status st0 = acopf::check_eval_scalars(obj_weight, delta_w, delta_c);
  if (st0 != ACOPF_OK) return st0;
  acopf::EvalArgs a = empty_args();
  a.x = x;
  a.y = y;
  a.obj_weight = obj_weight;
  a.sigma_x = sigma_x;
  a.sigma_s = sigma_s;
  a.delta_w = delta_w;
  a.delta_c = delta_c;
  a.f = f_dev;
  a.grad = grad;
  a.cons = cons;
  a.jvals = jvals;
  a.hvals = hvals;
  a.kvals = kvals;
  acopf_model* mm = const_cast<acopf_model*>(model);
  if (mm && mm->prof_calls < mm->prof_capacity) {
    acopf_status st = check_device_model(mm);
    if (st != ACOPF_OK) return st;
    DeviceScope ds(mm->device);
    if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_eval_assemble");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t* ev = mm->prof_events.data() + 3 * mm->prof_calls;
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = acopf::launch_eval(mm->dm, acopf::OUT_ALL, a, s, ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_eval_assemble (profiled)");
    mm->prof_calls++;
    return ACOPF_OK;
  }
  return run_eval(model, acopf::OUT_ALL, a, stream, "acopf_eval_assemble");
}

static void destroy_profile_events(acopf_model* m) {
  for (cudaEvent_t e : m->prof_events) cudaEventDestroy(e);
  m->prof_events.clear();
  m->prof_capacity = 0;
  m->prof_calls = 0;
}

acopf_status acopf_profile_begin(acopf_model* model, int32_t capacity) {
  acopf_status st = check_device_model(model);
  if (st != ACOPF_OK) return st;
  if (capacity < 0) return fail(ACOPF_E_INVALID_ARG, "capacity must be >= 0");
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_profile_begin");
  destroy_profile_events(model);
  model->prof_events.resize(size_t(capacity) * 3, nullptr);
  for (auto& e : model->prof_events) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      e = nullptr;
      destroy_profile_events(model);
      return cuda_fail(err, "acopf_profile_begin: cudaEventCreate");
    }
  }
  model->prof_capacity = capacity;
  model->prof_calls = 0;
  return ACOPF_OK;
}

acopf_status acopf_profile_end(acopf_model* model, int32_t* calls, double* phase1_ms,
                               double* phase2_ms, double* total_ms) {
  acopf_status st = check_device_model(model);
  if (st != ACOPF_OK) return st;
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_profile_end");
  double t1 = 0, t2 = 0, tt = 0;
  cudaError_t e = cudaSuccess;
  const int32_t nc = model->prof_calls;
  if (nc > 0) e = cudaEventSynchronize(model->prof_events[3 * (nc - 1) + 2]);
  for (int32_t k = 0; k < nc && e == cudaSuccess; ++k) {
    cudaEvent_t* ev = model->prof_events.data() + 3 * k;
    float a = 0, b = 0, c = 0;
    e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&c, ev[0], ev[2]);
    t1 += a;
    t2 += b;
    tt += c;
  }
  destroy_profile_events(model);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_profile_end");
  if (calls) *calls = nc;
  if (phase1_ms) *phase1_ms = t1;
  if (phase2_ms) *phase2_ms = t2;
  if (total_ms) *total_ms = tt;
  return ACOPF_OK;
}

acopf_status acopf_eval_assemble_host(acopf_model* model, const double* x, const double* y,
                                      double obj_weight, const double* sigma_x,
                                      const double* sigma_s, double delta_w, double delta_c,
                                      double* f, double* grad, double* cons, double* jvals,
                                      double* hvals, double* kvals, acopf_stream stream) {
  acopf_status st = check_device_model(model);
  if (st != ACOPF_OK) return st;
  if (!x || !y || !sigma_x || !sigma_s || !f || !grad || !cons || !jvals || !hvals || !kvals)
    return fail(ACOPF_E_INVALID_ARG, "acopf_eval_assemble_host: null pointer");
  const acopf::Layout& L = model->hm.L;
  const size_t n = L.n, m = L.m, nj = L.nnzj, nh = L.nnzh, nk = L.nnzk;
  // staging: inputs x, Sx (n) y, Ss (m); outputs f (1) grad (n) cons (m) J H K
  const size_t doubles = 2 * n + 2 * m + 1 + n + m + nj + nh + nk;
  DeviceScope ds(model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_eval_assemble_host");
  if (model->stage_bytes < doubles * 8) {
    if (model->stage) cudaFree(model->stage);
    model->stage = nullptr;
    model->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&model->stage, doubles * 8);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_eval_assemble_host: cudaMalloc");
    model->stage_bytes = doubles * 8;
  }
  double* d = model->stage;
  double *dx = d, *dsx = dx + n, *dy = dsx + n, *dss = dy + m;
  double *df = dss + m, *dg = df + 1, *dc = dg + n, *dj = dc + m, *dh = dj + nj, *dk = dh + nh;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(dx, x, n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dsx, sigma_x, n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, m * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dss, sigma_s, m * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_eval_assemble_host: upload");
  st = acopf_eval_assemble(model, dx, dy, obj_weight, dsx, dss, delta_w, delta_c, df, dg, dc, dj,
                           dh, dk, stream);
  if (st != ACOPF_OK) return st;
  e = cudaMemcpyAsync(f, df, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dg, n * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cons, dc, m * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(jvals, dj, nj * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hvals, dh, nh * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kvals, dk, nk * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_eval_assemble_host: download");
  return ACOPF_OK;
}

acopf_status acopf_model_set_option(acopf_model* model, int32_t option, int64_t value) {
  if (!model) return fail(ACOPF_E_INVALID_ARG, "null model");
  switch (option) {
    case ACOPF_OPT_PDL:
      if (value != 0 && value != 1) return fail(ACOPF_E_INVALID_ARG, "ACOPF_OPT_PDL takes 0 or 1");
      model->dm.pdl = int32_t(value);
      return ACOPF_OK;
    default:
      return fail(ACOPF_E_INVALID_ARG, "unknown option");
  }
}

int32_t acopf_launches_per_call(int32_t kind) {
  switch (kind) {
    case 0:
      return acopf::launches_for(acopf::OUT_ALL);
    case 1:
      return acopf::launches_for(acopf::OUT_KKT);
    case 2:
      return acopf::launches_for(acopf::OUT_OBJ);
    case 3:
      return acopf::launches_for(acopf::OUT_GRAD);
    case 4:
      return acopf::launches_for(acopf::OUT_CONS);
    case 5:
      return acopf::launches_for(acopf::OUT_JAC);
    case 6:
      return acopf::launches_for(acopf::OUT_HESS);
    default:
      return -1;
  }
}

}  // extern "C"

namespace {

// Best-of-5 rate (G operations / s) of the FP64 probe for `op`.
acopf_status measure_fp64_op(int device, int op, double* ginst) {
  DeviceScope ds(device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_measure_fp64");
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_measure_fp64");
  const int blocks = prop.multiProcessorCount * 8, iters = 16384;
  double* buf = nullptr;
  e = cudaMalloc(&buf, size_t(blocks) * 256 * 8);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_measure_fp64: cudaMalloc");
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 1e30f;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = acopf::launch_fp64_probe(op, buf, blocks, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_measure_fp64");
  const double ops = double(blocks) * 256 * 8 * iters;
  *ginst = ops / (double(best) * 1e-3) / 1e9;
  return ACOPF_OK;
}

}  // namespace

extern "C" {

acopf_status acopf_measure_fp64_gflops(int device, double* gflops) {
  if (!gflops || device < 0) return fail(ACOPF_E_INVALID_ARG, "bad argument");
  double r = 0.0;
  acopf_status st = measure_fp64_op(device, 0, &r);
  if (st == ACOPF_OK) *gflops = 2.0 * r;
  return st;
}

acopf_status acopf_measure_fp64_rates(int device, double* dfma, double* dadd, double* dmul) {
  if (device < 0) return fail(ACOPF_E_INVALID_ARG, "bad argument");
  double* out[3] = {dfma, dadd, dmul};
  for (int op = 0; op < 3; ++op) {
    if (!out[op]) continue;
    acopf_status st = measure_fp64_op(device, op, out[op]);
    if (st != ACOPF_OK) return st;
  }
  return ACOPF_OK;
}

}  // extern "C"
