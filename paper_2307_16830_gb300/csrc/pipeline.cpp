// Host-buffer pipeline (acopf_pipeline_*): consecutive fused evaluations of
// one model whose host-to-device copies, kernels and device-to-host copies
// overlap: one upload stream, one compute stream and one download stream per
// device staging slot (so the copies back of consecutive calls can use
// several copy engines).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "host_internal.h"

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

namespace {

// One staging slot: device inputs and outputs of one call, and the events
// that order its three stages.
struct PipeSlot {
  double* mem = nullptr;
  cudaStream_t d2h = nullptr;  // each slot's copies back run on their own stream
  cudaEvent_t uploaded = nullptr, computed = nullptr, downloaded = nullptr;
  bool used = false;
};

}  // namespace

struct acopf_pipeline {
  acopf_model* model = nullptr;
  std::vector<PipeSlot> slots;
  cudaStream_t h2d = nullptr, compute = nullptr;
  int64_t submitted = 0;
};

namespace {

void release(acopf_pipeline* p) {
  if (p->h2d) cudaStreamSynchronize(p->h2d);
  if (p->compute) cudaStreamSynchronize(p->compute);
  for (PipeSlot& s : p->slots) {
    if (s.d2h) {
      cudaStreamSynchronize(s.d2h);
      cudaStreamDestroy(s.d2h);
    }
    if (s.uploaded) cudaEventDestroy(s.uploaded);
    if (s.computed) cudaEventDestroy(s.computed);
    if (s.downloaded) cudaEventDestroy(s.downloaded);
    if (s.mem) cudaFree(s.mem);
  }
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->compute) cudaStreamDestroy(p->compute);
  delete p;
}

}  // namespace

extern "C" {

acopf_status acopf_pipeline_create(acopf_model* model, int32_t depth, acopf_pipeline** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_create: null output pointer");
  *out = nullptr;
  if (!model) return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_create: null model");
  if (model->device < 0) return fail(ACOPF_E_NO_DEVICE, "acopf_pipeline_create: host-only model");
  if (depth < 2 || depth > 8)
    return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_create: depth must be in [2, 8]");
  acopf_pipeline* p = new (std::nothrow) acopf_pipeline;
  if (!p) return fail(ACOPF_E_OOM, "host allocation failed");
  p->model = model;
  DeviceScope ds(model->device);
  cudaError_t e = ds.error();
  const acopf::Layout& L = model->hm.L;
  const size_t n = L.n, m = L.m;
  const size_t doubles = 2 * n + 2 * m + 1 + n + m + size_t(L.nnzj) + L.nnzh + L.nnzk;
  try {
    p->slots.resize(depth);
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(ACOPF_E_OOM, "host allocation failed");
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->compute, cudaStreamNonBlocking);
  for (PipeSlot& s : p->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s.mem, doubles * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.computed, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.downloaded, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release(p);
    return cuda_fail(e, "acopf_pipeline_create");
  }
  *out = p;
  return ACOPF_OK;
}

acopf_status acopf_pipeline_destroy(acopf_pipeline* pipeline) {
  if (!pipeline) return ACOPF_OK;
  DeviceScope ds(pipeline->model->device);
  release(pipeline);
  return ACOPF_OK;
}

acopf_status acopf_pipeline_submit(acopf_pipeline* pipeline, const double* x, const double* y,
                                   double obj_weight, const double* sigma_x,
                                   const double* sigma_s, double delta_w, double delta_c,
                                   double* f, double* grad, double* cons, double* jvals,
                                   double* hvals, double* kvals) {
  if (!pipeline) return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_submit: null pipeline");
  if (!x || !y || !sigma_x || !sigma_s || !f || !grad || !cons || !jvals || !hvals || !kvals)
    return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_submit: null pointer");
  acopf_status st = acopf::check_eval_scalars(obj_weight, delta_w, delta_c);
  if (st != ACOPF_OK) return st;
  acopf_pipeline* p = pipeline;
  const acopf::Layout& L = p->model->hm.L;
  const size_t n = L.n, m = L.m, nj = L.nnzj, nh = L.nnzh, nk = L.nnzk;
  DeviceScope ds(p->model->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_pipeline_submit");
  PipeSlot& s = p->slots[size_t(p->submitted % int64_t(p->slots.size()))];
  double *dx = s.mem, *dsx = dx + n, *dy = dsx + n, *dss = dy + m;
  double *df = dss + m, *dg = df + 1, *dc = dg + n, *dj = dc + m, *dh = dj + nj, *dk = dh + nh;
  cudaError_t e = cudaSuccess;
  // Stage 1: the slot's previous call must have been copied out.
  if (s.used) e = cudaStreamWaitEvent(p->h2d, s.downloaded, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, n * 8, cudaMemcpyHostToDevice, p->h2d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dsx, sigma_x, n * 8, cudaMemcpyHostToDevice, p->h2d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, m * 8, cudaMemcpyHostToDevice, p->h2d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dss, sigma_s, m * 8, cudaMemcpyHostToDevice, p->h2d);
  if (e == cudaSuccess) e = cudaEventRecord(s.uploaded, p->h2d);
  // Stage 2: the kernels, in call order on one stream (the model's scratch).
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->compute, s.uploaded, 0);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_pipeline_submit: upload");
  st = acopf_eval_assemble(p->model, dx, dy, obj_weight, dsx, dss, delta_w, delta_c, df, dg, dc,
                           dj, dh, dk, reinterpret_cast<acopf_stream>(p->compute));
  if (st != ACOPF_OK) return st;
  e = cudaEventRecord(s.computed, p->compute);
  // Stage 3: the outputs back to the host.
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s.d2h, s.computed, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, df, 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dg, n * 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cons, dc, m * 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(jvals, dj, nj * 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hvals, dh, nh * 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kvals, dk, nk * 8, cudaMemcpyDeviceToHost, s.d2h);
  if (e == cudaSuccess) e = cudaEventRecord(s.downloaded, s.d2h);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_pipeline_submit: download");
  s.used = true;
  p->submitted++;
  return ACOPF_OK;
}

acopf_status acopf_pipeline_wait(acopf_pipeline* pipeline) {
  if (!pipeline) return fail(ACOPF_E_INVALID_ARG, "acopf_pipeline_wait: null pipeline");
  DeviceScope ds(pipeline->model->device);
  cudaError_t e = cudaStreamSynchronize(pipeline->compute);
  for (PipeSlot& s : pipeline->slots)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pipeline->h2d);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_pipeline_wait");
  return ACOPF_OK;
}

}  // extern "C"
