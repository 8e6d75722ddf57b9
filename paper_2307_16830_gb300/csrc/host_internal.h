// Host-side internals shared by the C ABI translation units (model, batch
// and server entry points).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "acopf_internal.h"

struct acopf_model {
  acopf::HostModel hm;
  int device = -1;
  acopf::DevModel dm{};
  void* arena = nullptr;
  size_t arena_bytes = 0;
  // device staging for acopf_eval_assemble_host
  double* stage = nullptr;
  size_t stage_bytes = 0;
  // per-phase profiling (acopf_profile_begin / _end)
  std::vector<cudaEvent_t> prof_events;  // 3 per profiled call
  int32_t prof_capacity = 0;
  int32_t prof_calls = 0;
  // condensation / step recovery: Jacobian by rows and by columns, row
  // scratch (allocated by the first acopf_condense / acopf_recover_step)
  void* step_arena = nullptr;
  acopf::DevStep step{};
};

namespace acopf {

extern thread_local std::string g_last_error;
void set_last_error(const std::string& msg);
acopf_status fail(acopf_status s, const std::string& msg);
acopf_status cuda_fail(cudaError_t e, const char* where);

// Makes a device current for the scope of a call.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    err_ = cudaGetDevice(&prev_);
    if (err_ == cudaSuccess && prev_ != dev) {
      err_ = cudaSetDevice(dev);
      switched_ = err_ == cudaSuccess;
    }
  }
  ~DeviceScope() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  cudaError_t error() const { return err_; }

 private:
  int prev_ = 0;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carves a device arena into 256-byte aligned pieces.
struct ArenaPlan {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    const size_t o = off;
    off = align_up(off + count * sizeof(T), 256);
    return o;
  }
};

// The scratch one evaluation writes and reads back (slot partials, bus
// diagonals, generator-warp objective sums and their arrival counter).
// Every evaluation in flight at the same time needs its own; the counter
// must be zero before first use (each call leaves it zero).
struct WorkspacePlan {
  size_t part_slot = 0, bus_diag = 0, obj_part = 0, ticket = 0, bytes = 0;
};

inline WorkspacePlan workspace_plan(const Layout& L) {
  ArenaPlan p;
  WorkspacePlan w;
  w.part_slot = p.take<SlotPart>(2 * size_t(L.nl));
  w.bus_diag = p.take<BusDiag>(size_t(L.nb));
  w.obj_part = p.take<double>(size_t(ceil_div(L.ng, 32)) + 1);
  w.ticket = p.take<unsigned int>(1);
  w.bytes = p.off;
  return w;
}

// Points dm's scratch at a workspace laid out by `w` at `base`.
inline void bind_workspace(DevModel& dm, char* base, const WorkspacePlan& w) {
  dm.part_slot = reinterpret_cast<SlotPart*>(base + w.part_slot);
  dm.bus_diag = reinterpret_cast<BusDiag*>(base + w.bus_diag);
  dm.obj_part = reinterpret_cast<double*>(base + w.obj_part);
  dm.obj_ticket = reinterpret_cast<unsigned int*>(base + w.ticket);
}

// Device bytes of a model (its arena: network data, structure, scratch).
inline size_t model_device_bytes(const acopf_model* m) { return m->arena_bytes; }

// Phase-1 and phase-2 work items of one fused evaluation of `L` (instance
// index `inst`), in the block order of the single-instance launch.
void append_items(const Layout& L, int32_t inst, std::vector<int4>& p1, std::vector<int4>& p2);

// Frees the model's condensation arena (stepapi.cpp).
void free_step(acopf_model* m);

// Builds the Jacobian's row and column lists and the row scratch of the
// condensation (m->step), once (stepapi.cpp).
acopf_status step_lists(acopf_model* m);
// The model a Cholesky object was created for.
acopf_model* chol_model(const acopf_chol* c);

// Validates the scalar arguments of an evaluation.
acopf_status check_eval_scalars(double obj_weight, double delta_w, double delta_c);

}  // namespace acopf
