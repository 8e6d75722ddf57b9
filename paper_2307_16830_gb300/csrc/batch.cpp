// Batched evaluation entry points (acopf_batch_*): many instances of the
// fused evaluation in one pair of launches over flattened work-item lists.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "host_internal.h"

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

struct acopf_batch {
  int device = 0;
  int32_t count = 0;
  std::vector<const acopf_model*> models;
  std::vector<acopf::DevModel> inst;  // per instance: model view with own scratch
  std::vector<acopf::EvalArgs> args;
  void* scratch = nullptr;            // instances' workspaces
  size_t scratch_bytes = 0;
  acopf::DevModel* d_models = nullptr;
  acopf::EvalArgs* d_args = nullptr;
  int4* d_items = nullptr;            // phase-1 items, then phase-2 items
  int64_t n1 = 0, n2 = 0;
  int64_t seg1[5] = {0, 0, 0, 0, 0};  // phase-1 items of code variant c: [seg1[c], seg1[c + 1])
  std::vector<uint8_t> variant;       // per instance: 2 * regularised + has shunt
  std::vector<int4> items_host;       // the uploaded lists (kept for asynchronous copies)
  int occ1 = 0, occ2 = 0, sms = 0;
  int32_t schedule = -1;
  bool io_set = false;
  // CUDA graph of the current schedule's launches
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

bool schedule_valid(int32_t s) { return s >= 0 && s < ACOPF_BATCH_SCHEDULES && (s & 3) < 3; }

void destroy_graph(acopf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

// Builds the item lists of schedule `s` for the current code variants into
// b->items_host and b->seg1.
void build_items(acopf_batch* b, int32_t s) {
  const int order = s & 3;
  std::vector<int32_t> perm(b->count);
  std::iota(perm.begin(), perm.end(), 0);
  if (order == ACOPF_SCHED_ORDER_SIZE) {
    // Largest first; ties keep the given order.
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t i, int32_t j) {
      const acopf::Layout &A = b->inst[i].L, &B = b->inst[j].L;
      return int64_t(A.nl) + A.nb + A.ng > int64_t(B.nl) + B.nb + B.ng;
    });
  }
  std::vector<int4> p1, p2, all;
  all.reserve(size_t(b->n1 + b->n2));
  for (int c = 0; c < 4; ++c) {
    b->seg1[c] = int64_t(all.size());
    p1.clear();
    for (int32_t i : perm)
      if (b->variant[i] == c) acopf::append_items(b->inst[i].L, i, p1, p2);
    if (order == ACOPF_SCHED_ORDER_GROUP)
      std::stable_sort(p1.begin(), p1.end(), [](const int4& u, const int4& v) { return u.y < v.y; });
    all.insert(all.end(), p1.begin(), p1.end());
  }
  b->seg1[4] = int64_t(all.size());
  p2.clear();
  p1.clear();
  for (int32_t i : perm) acopf::append_items(b->inst[i].L, i, p1, p2);
  all.insert(all.end(), p2.begin(), p2.end());
  b->items_host.swap(all);
}

cudaError_t launch(acopf_batch* b, cudaStream_t s) {
  const bool persistent = (b->schedule & ACOPF_SCHED_PERSISTENT) != 0;
  const int64_t cap1 = persistent ? int64_t(std::max(1, b->occ1)) * b->sms : INT32_MAX;
  const int64_t cap2 = persistent ? int64_t(std::max(1, b->occ2)) * b->sms : INT32_MAX;
  const int g2 = int(std::min(b->n2, cap2));
  return acopf::launch_batch(b->d_models, b->d_args, b->d_items, b->seg1, cap1, b->d_items + b->n1,
                             int(b->n2), g2, (b->schedule & ACOPF_SCHED_PDL) != 0, s);
}

acopf_status run(acopf_batch* b, cudaStream_t s) {
  if ((b->schedule & ACOPF_SCHED_GRAPH) == 0) {
    cudaError_t e = launch(b, s);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_batch_eval_assemble");
    return ACOPF_OK;
  }
  if (!b->exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_batch: cudaStreamBeginCapture");
    cudaError_t le = launch(b, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le, "acopf_batch: launch under capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "acopf_batch: cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return cuda_fail(e, "acopf_batch: cudaGraphInstantiate");
    }
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_batch: cudaGraphLaunch");
  return ACOPF_OK;
}

acopf_status set_schedule(acopf_batch* b, int32_t s) {
  if (!schedule_valid(s)) return fail(ACOPF_E_INVALID_ARG, "acopf_batch: invalid schedule");
  if (s == b->schedule) return ACOPF_OK;
  // The item lists and the graph are re-made; nothing of the batch may be in flight.
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "acopf_batch_set_schedule");
  if (b->schedule < 0 || (b->schedule & 3) != (s & 3)) {
    build_items(b, s);
    e = cudaMemcpy(b->d_items, b->items_host.data(), b->items_host.size() * sizeof(int4),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "acopf_batch: item upload");
  }
  destroy_graph(b);
  b->schedule = s;
  return ACOPF_OK;
}

void release(acopf_batch* b) {
  destroy_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->scratch) cudaFree(b->scratch);
  delete b;
}

}  // namespace

extern "C" {

acopf_status acopf_batch_create(acopf_model* const* models, int32_t count, acopf_batch** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_create: null output pointer");
  *out = nullptr;
  if (!models || count < 1) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_create: need count >= 1");
  for (int32_t i = 0; i < count; ++i) {
    if (!models[i]) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_create: null model");
    if (models[i]->device < 0)
      return fail(ACOPF_E_NO_DEVICE, "acopf_batch_create: host-only model");
    if (models[i]->device != models[0]->device)
      return fail(ACOPF_E_INVALID_ARG, "acopf_batch_create: models on different devices");
  }
  acopf_batch* b = new (std::nothrow) acopf_batch;
  if (!b) return fail(ACOPF_E_OOM, "host allocation failed");
  b->device = models[0]->device;
  b->count = count;
  DeviceScope ds(b->device);
  if (ds.error() != cudaSuccess) {
    delete b;
    return cuda_fail(ds.error(), "acopf_batch_create: cudaSetDevice");
  }
  try {
    b->models.assign(models, models + count);
    b->inst.resize(count);
    b->args.resize(count);
    // Sizes: scratch per instance, then the tables and the item lists.
    acopf::ArenaPlan p;
    std::vector<size_t> ws_off(count);
    std::vector<acopf::WorkspacePlan> ws(count);
    std::vector<int4> p1, p2;
    for (int32_t i = 0; i < count; ++i) {
      ws[i] = acopf::workspace_plan(models[i]->hm.L);
      ws_off[i] = p.take<char>(ws[i].bytes);
      acopf::append_items(models[i]->hm.L, i, p1, p2);
    }
    b->n1 = int64_t(p1.size());
    b->n2 = int64_t(p2.size());
    if (b->n1 > INT32_MAX || b->n2 > INT32_MAX) {
      delete b;
      return fail(ACOPF_E_INVALID_ARG, "acopf_batch_create: too many work items");
    }
    const size_t o_models = p.take<acopf::DevModel>(count);
    const size_t o_args = p.take<acopf::EvalArgs>(count);
    const size_t o_items = p.take<int4>(size_t(b->n1 + b->n2));
    cudaError_t e = cudaMalloc(&b->scratch, p.off);
    if (e != cudaSuccess) {
      b->scratch = nullptr;
      release(b);
      return cuda_fail(e, "acopf_batch_create: cudaMalloc");
    }
    b->scratch_bytes = p.off;
    char* base = static_cast<char*>(b->scratch);
    e = cudaMemset(base, 0, p.off);  // arrival counters start at zero
    if (e != cudaSuccess) {
      release(b);
      return cuda_fail(e, "acopf_batch_create: cudaMemset");
    }
    b->variant.resize(count);
    for (int32_t i = 0; i < count; ++i) {
      b->inst[i] = models[i]->dm;
      acopf::bind_workspace(b->inst[i], base + ws_off[i], ws[i]);
      b->variant[i] = uint8_t(b->inst[i].has_shunt ? 1 : 0);
    }
    b->d_models = reinterpret_cast<acopf::DevModel*>(base + o_models);
    b->d_args = reinterpret_cast<acopf::EvalArgs*>(base + o_args);
    b->d_items = reinterpret_cast<int4*>(base + o_items);
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = acopf::batch_occupancy(&b->occ1, &b->occ2);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
      release(b);
      return cuda_fail(e, "acopf_batch_create");
    }
  } catch (const std::bad_alloc&) {
    release(b);
    return fail(ACOPF_E_OOM, "host allocation failed");
  }
  acopf_status st = set_schedule(b, ACOPF_SCHED_ORDER_SIZE | ACOPF_SCHED_PDL);
  if (st != ACOPF_OK) {
    release(b);
    return st;
  }
  *out = b;
  return ACOPF_OK;
}

acopf_status acopf_batch_destroy(acopf_batch* batch) {
  if (!batch) return ACOPF_OK;
  DeviceScope ds(batch->device);
  release(batch);
  return ACOPF_OK;
}

acopf_status acopf_batch_set_io(acopf_batch* batch, const acopf_batch_io* io, int32_t count,
                                acopf_stream stream) {
  if (!batch || !io) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_set_io: null pointer");
  if (count != batch->count)
    return fail(ACOPF_E_INVALID_ARG, "acopf_batch_set_io: count differs from the batch's");
  for (int32_t i = 0; i < count; ++i) {
    const acopf_batch_io& r = io[i];
    if (!r.x || !r.y || !r.sigma_x || !r.sigma_s || !r.f || !r.grad || !r.cons || !r.jvals ||
        !r.hvals || !r.kvals)
      return fail(ACOPF_E_INVALID_ARG,
                  "acopf_batch_set_io: null pointer in instance " + std::to_string(i));
    if ((r.Pd == nullptr) != (r.Qd == nullptr))
      return fail(ACOPF_E_INVALID_ARG, "acopf_batch_set_io: give both Pd and Qd, or neither");
    acopf_status st = acopf::check_eval_scalars(r.obj_weight, r.delta_w, r.delta_c);
    if (st != ACOPF_OK) return st;
  }
  DeviceScope ds(batch->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_batch_set_io");
  std::vector<acopf::DevModel> inst(batch->inst);
  std::vector<acopf::EvalArgs> args(count);
  for (int32_t i = 0; i < count; ++i) {
    const acopf_batch_io& r = io[i];
    if (r.Pd) {
      inst[i].Pd = r.Pd;
      inst[i].Qd = r.Qd;
    }
    acopf::EvalArgs& a = args[i];
    std::memset(&a, 0, sizeof(a));
    a.x = r.x;
    a.y = r.y;
    a.obj_weight = r.obj_weight;
    a.sigma_x = r.sigma_x;
    a.sigma_s = r.sigma_s;
    a.delta_w = r.delta_w;
    a.delta_c = r.delta_c;
    a.f = r.f;
    a.grad = r.grad;
    a.cons = r.cons;
    a.jvals = r.jvals;
    a.hvals = r.hvals;
    a.kvals = r.kvals;
  }
  // Pageable sources: each copy returns once its source has been staged,
  // so the host vectors may change afterwards.
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<uint8_t> variant(count);
  for (int32_t i = 0; i < count; ++i)
    variant[i] = uint8_t((io[i].delta_w != 0.0 || io[i].delta_c != 0.0 ? 2 : 0) +
                         (inst[i].has_shunt ? 1 : 0));
  cudaError_t e = cudaSuccess;
  if (variant != batch->variant) {  // regroup the phase-1 items by code variant
    batch->variant.swap(variant);
    build_items(batch, batch->schedule);
    e = cudaMemcpyAsync(batch->d_items, batch->items_host.data(),
                        batch->items_host.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    destroy_graph(batch);  // the launches per variant may have changed
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(batch->d_models, inst.data(), count * sizeof(acopf::DevModel),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(batch->d_args, args.data(), count * sizeof(acopf::EvalArgs),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "acopf_batch_set_io");
  batch->args = std::move(args);
  batch->io_set = true;
  return ACOPF_OK;
}

acopf_status acopf_batch_eval_assemble(acopf_batch* batch, acopf_stream stream) {
  if (!batch) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_eval_assemble: null batch");
  if (!batch->io_set)
    return fail(ACOPF_E_INVALID_ARG, "acopf_batch_eval_assemble: call acopf_batch_set_io first");
  DeviceScope ds(batch->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_batch_eval_assemble");
  return run(batch, reinterpret_cast<cudaStream_t>(stream));
}

acopf_status acopf_batch_set_schedule(acopf_batch* batch, int32_t schedule) {
  if (!batch) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_set_schedule: null batch");
  DeviceScope ds(batch->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_batch_set_schedule");
  return set_schedule(batch, schedule);
}

acopf_status acopf_batch_autotune(acopf_batch* batch, acopf_stream stream, int32_t reps,
                                  int32_t* best, float* times_ms) {
  if (!batch || !best) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_autotune: null pointer");
  if (reps < 1) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_autotune: reps must be >= 1");
  if (!batch->io_set)
    return fail(ACOPF_E_INVALID_ARG, "acopf_batch_autotune: call acopf_batch_set_io first");
  DeviceScope ds(batch->device);
  if (ds.error() != cudaSuccess) return cuda_fail(ds.error(), "acopf_batch_autotune");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    return cuda_fail(e, "acopf_batch_autotune: cudaEventCreate");
  }
  acopf_status st = ACOPF_OK;
  int32_t arg = -1;
  float best_ms = 0.0f;
  for (int32_t c = 0; c < ACOPF_BATCH_SCHEDULES && st == ACOPF_OK; ++c) {
    if (times_ms) times_ms[c] = -1.0f;
    if (!schedule_valid(c)) continue;
    st = set_schedule(batch, c);
    for (int w = 0; w < 2 && st == ACOPF_OK; ++w) st = run(batch, s);
    if (st != ACOPF_OK) break;
    e = cudaEventRecord(ev[0], s);
    for (int32_t r = 0; r < reps && st == ACOPF_OK && e == cudaSuccess; ++r) st = run(batch, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "acopf_batch_autotune");
      break;
    }
    ms /= float(reps);
    if (times_ms) times_ms[c] = ms;
    if (arg < 0 || ms < best_ms) {
      arg = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (st != ACOPF_OK) return st;
  *best = arg;
  return set_schedule(batch, arg);
}

acopf_status acopf_batch_info(const acopf_batch* batch, int32_t* schedule, int64_t* items_phase1,
                              int64_t* items_phase2, int64_t* device_bytes) {
  if (!batch) return fail(ACOPF_E_INVALID_ARG, "acopf_batch_info: null batch");
  if (schedule) *schedule = batch->schedule;
  if (items_phase1) *items_phase1 = batch->n1;
  if (items_phase2) *items_phase2 = batch->n2;
  if (device_bytes) *device_bytes = int64_t(batch->scratch_bytes);
  return ACOPF_OK;
}

}  // extern "C"
