// Device view of the supernodal factor, its task graphs, and the launchers
// of chol.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace acopf {

// Supernodes have at most this many columns (the solves stage a
// supernode's diagonal block in shared memory).
constexpr int kCholMaxWidth = 64;
// Small supernodes (one warp each, inside group tasks): at most this many
// rows and columns.
constexpr int kCholWarpRows = 32;
constexpr int kCholWarpCols = 8;
// A child's rows below its columns fit a row-map scratch of this size.
constexpr int kCholMaxRelRows = 4096;
// Block tasks: panel plus update matrix staged in at most this many doubles,
// and at most this many rows.
constexpr int kCholBlockDoubles = 11264;
constexpr int kCholBlockRows = 512;
// Tiles of the tiled supernodes' fronts.
constexpr int kCholTile = 32;

// One task graph on the device: tasks (x = kind | k << 8, y, z, w), their
// dependencies in CSR form, a finished flag per task and the counter the
// blocks take tasks from (both zeroed before each run); optionally the
// tasks of another graph each task also waits for (xdep, CSR, as indices
// into that graph's flags xdone; xdep_ptr NULL: none).
struct CholTasks {
  const int4* task;
  const int32_t* dep_ptr;
  const int32_t* dep;
  int32_t* done;
  int32_t* next;
  long long* trace;  // NULL, or 6 words per task (kind, argument, taken, ready, finished, SM)
  int32_t n;
  const int32_t* xdep_ptr;
  const int32_t* xdep;
  const int32_t* xdone;
};

// Device copies of the symbolic arrays (see symbolic.h, chol_plan.h) and
// the factor.
struct CholDev {
  int32_t n;
  const int32_t* sn_first;   // ns + 1
  const int32_t* sn_rowptr;  // ns + 1
  const int32_t* rowidx;
  const int64_t* sn_off;     // ns + 1
  const int32_t* kid_ptr;    // ns + 1
  const int32_t* kid;
  const int32_t* rel_off;    // ns
  const int32_t* relmap;
  const int64_t* u_off;      // ns + 1
  const int64_t* z_off;      // ns + 1
  const int32_t* grp_ptr;    // groups + 1
  const int32_t* grp_sn;
  const int32_t* grp_lptr;   // groups + 1
  const int32_t* grp_lev;
  const int32_t* brk_off;    // ns: a tiled supernode's child's breakpoints in tile_brk
  const int32_t* tile_brk;
  const int4* kid_desc;      // per kid slot q: {m of kid[q], rel_off, u_off low, u_off high}
  const int32_t* kid_brk;    // per kid slot q: brk_off of kid[q]
  const int32_t* fg_ptr;     // forward-solve gather lists (chol_plan.h)
  const int32_t* fg_idx;
  double* Lx;                // the supernodal blocks
  double* Ux;                // the update matrices
  double* Zx;                // the update vectors of a solve
  double* Dinv;              // n: 1 / L[j][j] of the last factorization (the solves multiply)
  int32_t* bad;              // smallest failed pivot column (>= n: none)
  int32_t* abort;            // nonzero: a task gave up waiting (the run failed)
};

cudaError_t launch_gather(double* out, const double* in, const int32_t* idx, int n,
                          cudaStream_t s);
cudaError_t launch_scatter(double* out, const double* in, const int32_t* idx, int n,
                           cudaStream_t s);
cudaError_t launch_chol_assemble(double* Lx, const int64_t* amap, const double* kvals,
                                 int64_t nnz, cudaStream_t s);

// One bottom level (list: its count supernodes, device): the factorization,
// forward and backward substitution, one thread per supernode.
// `stage`: the level's largest h w + m (m + 1) / 2 (at most kCholBottomStage).
constexpr int kCholBottomStage = 142;
size_t chol_bottom_smem_bytes(int stage);
cudaError_t launch_chol_bottom(const CholDev& d, const int32_t* list, int count, int stage,
                               double tol, cudaStream_t s);
cudaError_t launch_chol_bottom_fwd(const CholDev& d, const int32_t* list, int count, double* y,
                                   cudaStream_t s);
cudaError_t launch_chol_bottom_bwd(const CholDev& d, const int32_t* list, int count, double* x,
                                   cudaStream_t s);
// Dynamic shared memory of the task kernels, and the opt-in that lets them
// use it (set once per device, before any launch or capture); blocks per SM
// the block-task and the factorization's warp-task kernels are launched
// with.
size_t chol_task_smem_bytes();
cudaError_t chol_task_setup(int* blocks_per_sm, int* warp_blocks_per_sm);
// The factorization, forward and backward solve task kernels with `blocks`
// persistent blocks (tasks, done flags and counter as described above).
// `early`: the kernel is launched as a programmatic dependent of the
// kernel before it (the factorization's and the forward solve's warp-task
// kernels), whose flags its tasks wait for (xdep).
cudaError_t launch_chol_factor_tasks(const CholDev& d, const CholTasks& t, double tol, int blocks,
                                     bool early, cudaStream_t s);
cudaError_t launch_chol_forward_tasks(const CholDev& d, const CholTasks& t, double* y, int blocks,
                                      bool early, cudaStream_t s);
cudaError_t launch_chol_backward_tasks(const CholDev& d, const CholTasks& t, double* x, int blocks,
                                       cudaStream_t s);
// The factorization's warp tasks (one warp-small supernode per warp, after
// the bottom levels and before the block-task kernel) with `blocks` blocks.
cudaError_t launch_chol_factor_warps(const CholDev& d, const CholTasks& t, double tol, int blocks,
                                     cudaStream_t s);
// The solves' warp tasks (one small supernode per warp) with `blocks` blocks;
// `early` as above (the backward one after the backward block-task kernel).
cudaError_t launch_chol_solve_warps(const CholDev& d, const CholTasks& t, double* v, bool forward,
                                    int blocks, bool early, cudaStream_t s);

}  // namespace acopf
