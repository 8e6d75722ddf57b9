// Internal declarations shared by the host symbolic phase, the kernels and
// the C ABI of libacopf.  Not installed; the public interface is acopf.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/acopf.h"

namespace acopf {

// Offsets of the variable and constraint groups and of the COO sections.
// Everything within one model fits int32 (checked at build time).
struct Layout {
  int32_t nb = 0, nl = 0, ng = 0, nref = 0;
  // variables
  int32_t VA = 0, VM = 0, PG = 0, QG = 0, P = 0, Q = 0, n = 0;
  // constraints
  int32_t REF = 0, PF = 0, QF = 0, PT = 0, QT = 0, ANG = 0, SF = 0, ST = 0, PB = 0, QB = 0, m = 0;
  // Jacobian COO sections
  int32_t JREF = 0, JPF = 0, JQF = 0, JPT = 0, JQT = 0, JANG = 0, JSF = 0, JST = 0;
  int32_t JPBV = 0, JQBV = 0, JPBG = 0, JQBG = 0, JPBA = 0, JQBA = 0, nnzj = 0;
  // Hessian COO sections
  int32_t HBLK = 0, HTH = 0, HG = 0, HB = 0, nnzh = 0;
  int32_t nnzk = 0;
  // lanes of the bus-row phase (row chunks, a multiple of 32)
  int32_t nrc = 0;
};

// Branch pi-model coefficients, structure of arrays: coef[k * nl + l] with
// k = 0..7 -> g_ff, b_ff, g_ft, b_ft, g_tf, b_tf, g_tt, b_tt.
enum { CG_FF = 0, CB_FF, CG_FT, CB_FT, CG_TF, CB_TF, CG_TT, CB_TT, NCOEF };

// Partial sums that the branch phase of the KKT assembly leaves for the bus
// phase (device scratch), one per slot.  Slots list the arcs of each bus in
// the order (other end, arc id); the slot of arc a at bus i (other end j,
// branch l) holds the branch's contributions to
//   aa: (va_i, va_i)   ma: (vm_i, va_i)   mm: (vm_i, vm_i)   mx: (vm_i, va_j)
//   vv: (va_i, va_j)   ww: (vm_i, vm_j)   (vv, ww are the same at both ends).
struct alignas(16) SlotPart {
  double aa, ma, mm, mx, vv, ww;
};

// The bus's own terms of its two diagonal entries of M_cond, left by the
// bus-input blocks of phase 1 for the bus rows of phase 2 (device scratch,
// in the bus processing order):
//   va = Sigma_x(va_i) + delta_w + D_ref (reference buses),
//   vm = Sigma_x(vm_i) + delta_w + W_bus + D_P (2 Gs vm)^2 + D_Q (2 Bs vm)^2.
struct alignas(16) BusDiag {
  double va, vm;
};

// Read-only device view of a model, passed to kernels by value.
struct DevModel {
  Layout L;
  // branches
  const int32_t* f;
  const int32_t* t;
  const double* coef;
  // buses
  const double* Pd;
  const double* Qd;
  const double* Gs;
  const double* Bs;
  const int32_t* ref_row;      // per bus: its reference row, or -1
  const int32_t* arc_ptr;      // nb + 1
  const int32_t* arcs_by_idx;  // 2 nl: arcs of each bus, ascending arc id
  // Bus phase processing order: buses sorted by (number of arcs, number of
  // generators) so that the 32 buses of a warp run loops of equal length.
  // Slots and balance terms are laid out in this order.
  const int32_t* porder;       // nb: bus at processing position p
  const int32_t* pslot_ptr;    // nb + 1: slots of position p
  const int32_t* slot_nbr;     // 2 nl: other end of each slot's arc
  const int32_t* slot_of_arc;  // 2 nl: slot of each arc
  const int32_t* gen_ptr;      // nb + 1
  const int32_t* gens_at;      // ng: generators of each bus, ascending id
  const int32_t* pbal_ptr;     // nb + 1: balance terms of position p
  const int32_t* bal_idx;      // ng + 2 nl: x index of pg (generators, ascending) then of
                               // p_a (arcs, ascending) in each bus's active balance row
  // generators
  const int32_t* gbus;
  const double* c2;
  const double* c1;
  const double* c0;
  // M_cond structure
  const int32_t* krowptr;      // n + 1
  // Per branch: start of its four arc rows p_l, q_l, p_{nl+l}, q_{nl+l} in
  // M_cond, and the generator count and rank (number of earlier arcs) at
  // its from and to buses packed as ngf | rankf << 8 | ngt << 16 | rankt << 24
  // (kCountsWide when one of them exceeds 255: the kernel then reads them
  // from gen_ptr and the row starts).
  const int4* brow;            // nl
  const uint32_t* bcnt;        // nl
  // Bus-row phase: lane c runs row chunk c, two int4 each: {bus i (-1: an
  // idle lane), position p, first slot, end slot} and {the chunk's first
  // positions in rows va_i, vm_i (va columns) and vm_i (vm columns), the
  // lane of the bus's first chunk | chunk count << 5}.  A bus's chunks are
  // consecutive lanes of one warp, split between runs of equal neighbours.
  const int4* rchunk;          // 2 L.nrc
  // scratch
  SlotPart* part_slot;         // 2 nl
  BusDiag* bus_diag;           // nb
  double* obj_part;            // one per generator warp
  unsigned int* obj_ticket;    // arrival counter of the generator warps (reset by the last)
  // launch options
  int32_t has_shunt;           // some bus has Gs != 0 or Bs != 0
  int32_t pdl;                 // chain the phases with programmatic dependent launch
};

// Host model: everything the symbolic phase builds.
struct HostModel {
  Layout L;
  std::vector<int32_t> f, t, gbus, ref_row, ref_bus;
  std::vector<double> coef;  // NCOEF * nl
  std::vector<double> Pd, Qd, Gs, Bs, c2, c1, c0;
  std::vector<int32_t> arc_ptr, arcs_by_idx, arcs_by_nbr, gen_ptr, gens_at;
  std::vector<int32_t> porder, pslot_ptr, slot_nbr, slot_of_arc, pbal_ptr, bal_idx;
  std::vector<int32_t> brow;   // 4 per branch
  std::vector<uint32_t> bcnt;
  std::vector<int32_t> rchunk;  // 8 per bus-row lane (DevModel::rchunk)
  std::vector<int32_t> jrows, jcols, hrows, hcols, krowptr, kcolind;
  std::vector<double> xl, xu, gl, gu;
};

// Builds the host model; on failure returns a status and sets `err`.
acopf_status build_host_model(const acopf_buses* B, const acopf_branches* Lb, const acopf_gens* G,
                              HostModel& hm, std::string& err);

constexpr uint32_t kCountsWide = 0xFFFFFFFFu;

// Kernel launch configuration.
constexpr int kBranchThreads = 128;
constexpr int kBusThreads = 128;
constexpr int kGenThreads = 128;
// Balance-row terms a warp of bus threads stages in shared memory (P and Q
// values, 16 bytes each); warps with more terms sum from global memory.
constexpr int kBalCap = 192;
// Slots of one bus-row chunk (one round of loads in flight); a bus with
// more than 32 x kRowChunk slots takes larger chunks.
constexpr int kRowChunk = 4;

inline int32_t ceil_div(int64_t a, int64_t b) { return static_cast<int32_t>((a + b - 1) / b); }


// What a launch computes.
enum : unsigned {
  OUT_OBJ = 1u,
  OUT_GRAD = 2u,
  OUT_CONS = 4u,
  OUT_JAC = 8u,
  OUT_HESS = 16u,
  OUT_KKT = 32u,
  OUT_ALL = 63u,
};

struct EvalArgs {
  const double* x;
  const double* y;
  double obj_weight;
  const double* sigma_x;
  const double* sigma_s;
  double delta_w;
  double delta_c;
  // inputs of the array-fed assembly
  const double* hvals_in;
  const double* jvals_in;
  // outputs
  double* f;
  double* grad;
  double* cons;
  double* jvals;
  double* hvals;
  double* kvals;
};

// Condensation around M_cond and step recovery (step.cu): device views.
// The Jacobian's COO entries by row (jr_*) and by column (jt_*), each list in
// ascending slot order; `w` is the per-row scratch C q_s + D q_y.
struct DevStep {
  int32_t n, m;
  const int32_t* jr_ptr;   // m + 1
  const int32_t* jr_slot;  // nnzj
  const int32_t* jr_col;   // nnzj
  const int32_t* jt_ptr;   // n + 1
  const int32_t* jt_slot;  // nnzj
  const int32_t* jt_row;   // nnzj
  double* w;               // m
  double* res_part;        // kResPart per block of the residual kernel
  int32_t res_blocks;      // its grid (fixed per device, so its sums have a fixed order)
};

// An interior iterate and the right-hand sides of its Newton system (device).
struct StepIterate {
  const double *x, *s, *xl, *xu, *sl, *su;
  const double *zl_x, *zu_x, *zl_s, *zu_s;
  const double *p_x, *p_s, *p_y, *p_zl_x, *p_zu_x, *p_zl_s, *p_zu_s;
};

cudaError_t launch_condense(const DevStep& st, const StepIterate& it, const double* jvals,
                            double delta_w, double delta_c, double* sigma_x, double* sigma_s,
                            double* q_s, double* rhs, bool pdl, cudaStream_t s);
// Grid of the residual kernel on a device with `sms` SMs (its scratch holds
// kResPart doubles per block).
constexpr int kResPart = 7;
int residual_blocks(int sms);
// out[0..8]: E at mu and its parts.
cudaError_t launch_kkt_residual(const DevStep& st, const StepIterate& it, const double* y,
                                const double* grad, const double* cons, const double* jvals,
                                double mu, double* out, cudaStream_t s);
// The same, and, when mu2 >= 0, out[9] = E at mu2 from the same pass.
cudaError_t launch_kkt_residual2(const DevStep& st, const StepIterate& it, const double* y,
                                 const double* grad, const double* cons, const double* jvals,
                                 double mu, double mu2, double* out, cudaStream_t s);
cudaError_t launch_recover(const DevStep& st, const StepIterate& it, const double* jvals,
                           double delta_w, double delta_c, const double* sigma_s,
                           const double* q_s, const double* dx, double* ds, double* dy,
                           double* dzl_x, double* dzu_x, double* dzl_s, double* dzu_s,
                           cudaStream_t s);


// Launchers (kernels.cu).  Each returns the CUDA error of its launches.
// `mid`, when not null, is recorded between the two phases (phase 2 then
// launches without programmatic dependent launch).
cudaError_t launch_eval(const DevModel& dm, unsigned what, const EvalArgs& a, cudaStream_t s,
                        cudaEvent_t mid = nullptr);
cudaError_t launch_assemble(const DevModel& dm, const EvalArgs& a, cudaStream_t s);
// FP64 throughput probe: op 0 fma, 1 add, 2 mul; 256 threads x blocks, each
// 8 chains of `iters` operations.
cudaError_t launch_fp64_probe(int op, double* out, int blocks, int iters, cudaStream_t s);
// Batched fused evaluation over work lists.  Phase-1 items (instance, role,
// block, blocks of the role) are grouped by code variant c = 2 reg + shunt
// (reg: delta_w or delta_c nonzero; shunt: the model has a shunt), variant
// c owning items1[seg1[c], seg1[c + 1]); each present variant is one launch
// of min(items, cap1) blocks.  Phase 2 runs n2 items on grid2 blocks (grid
// < items: persistent blocks stride over the list).
cudaError_t launch_batch(const DevModel* models, const EvalArgs* ios, const int4* items1,
                         const int64_t* seg1, int64_t cap1, const int4* items2, int n2, int grid2,
                         bool pdl, cudaStream_t s);
// Resident blocks per SM of the two batch kernels.
cudaError_t batch_occupancy(int* phase1, int* phase2);
int launches_for(unsigned what);

}  // namespace acopf
