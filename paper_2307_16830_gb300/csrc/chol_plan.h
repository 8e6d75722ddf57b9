// Task graphs of the numeric factorization of M_cond and of its solves
// (host): built once per pattern from the supernodal symbolic phase.
//
// The factorization runs as one persistent kernel whose blocks take tasks
// in list order and wait (bounded) for each task's dependencies before
// running it; the list is a topological order of the task graph, so the
// lowest unfinished task a running block holds can always proceed.  Tasks:
//   group   a connected set of small supernodes (at most kCholWarpRows rows
//           and kCholWarpCols columns each), factored by one block level by
//           level within the set, one warp per supernode;
//   block   one supernode whose panel and update matrix fit the block's
//           shared-memory staging, factored by one block;
//   tiled   the front of a larger supernode in kCholTile x kCholTile tiles:
//           asm (children's update matrices added into one tile), potrf
//           (Cholesky of a diagonal tile of the panel), trsm (a tile below
//           it times the inverse transpose of that factor), upd (one tile
//           minus the product of two trsm tiles); the parent's tasks wait
//           for the last writers of the update matrix's tiles (kTaskFin,
//           a join task with no work, is no longer generated).
// The small supernodes whose descendants are all small or bottom ones
// (warp-small) are factored by a kernel of warp tasks, one supernode per
// warp, in the forward solve's warp list (the same dependencies: children
// first), launched before the task kernel, which may start while it runs:
// a task that needs a warp-small child waits for that warp task's flag.
// The group tasks hold the other small supernodes.  The solves take the warp-small supernodes one per warp and
// the others (but the bottom ones) one per block.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "acopf.h"

namespace acopf {

struct CholSymbolic;

// Task kinds (the low 8 bits of a task's first word; for potrf, trsm and
// upd the panel tile column k sits in the bits above).
enum CholTaskKind : int32_t {
  kTaskGroup = 0,
  kTaskBlock = 1,
  kTaskAsm = 2,
  kTaskPotrf = 3,
  kTaskTrsm = 4,
  kTaskUpd = 5,
  kTaskFin = 6,
};

// Supernode classes.
enum CholSnClass : int8_t { kSnSmall = 0, kSnBlock = 1, kSnTiled = 2, kSnBottom = 3 };

// Bottom supernodes: at most kCholBottomRows rows and kCholBottomCols
// columns, all descendants bottom supernodes too, on the levels (heights
// above the leaves) that hold at least kCholBottomMinCount of them.  They
// are factored before the task kernel, one launch per level, one thread per
// supernode (a level's supernodes sorted by shape so a warp's loops have
// one length): the pivots of 32 supernodes share each FP64 instruction.
constexpr int32_t kCholBottomRows = 16;
constexpr int32_t kCholBottomCols = 4;
constexpr int32_t kCholBottomMinCount = 32768;

// Tile edge of the tiled supernodes' fronts.
constexpr int32_t kCholTileEdge = 32;
// Shared-memory staging (doubles) of a block task: its panel and its update
// matrix together.
constexpr int32_t kCholBlockStage = 11264;
// Rows of a block-task supernode at most (its children's row maps are
// staged in shared memory).
constexpr int32_t kCholBlockMaxRows = 512;

// A task graph: task t is words task[4t .. 4t + 4) = {kind | k << 8, a, b,
// c} (group: a = group; block, fin: a = supernode; asm, trsm: a =
// supernode, b = tile row, c = tile column; potrf: a = supernode, b = c =
// k; upd: a = supernode, b = tile row, c = tile column, k the panel tile
// column of the product), its dependencies dep[dep_ptr[t] .. dep_ptr[t+1])
// (all earlier in the list) and the tasks of the graph launched before it
// that it needs, xdep[xdep_ptr[t] .. xdep_ptr[t+1]): for the
// factorization's and the forward solve's block tasks, their warp-small
// children (positions in forward_warp's list); for the backward solve's
// warp tasks, a parent solved by a block task (position in backward's
// list); empty for the other graphs.
struct CholGraph {
  std::vector<int32_t> task, dep_ptr, dep, xdep_ptr, xdep;
  int32_t n_tasks() const { return int32_t(task.size() / 4); }
};

// Groups: group g holds supernodes grp_sn[grp_ptr[g] .. grp_ptr[g+1]) in
// nlv = grp_lptr[g+1] - grp_lptr[g] - 1 levels: level v is grp_sn[grp_lev[
// grp_lptr[g] + v] .. grp_lev[grp_lptr[g] + v + 1]) (positions into grp_sn),
// a supernode's children in the group on lower levels than itself.
// Bottom levels: level v's supernodes are bot_sn[bot_ptr[v] .. bot_ptr[v+1]),
// bot_stage[v] their largest h w + m (m + 1) / 2 (a thread's staging).
// Tile breakpoints: for a child c of a tiled supernode, tile_brk[brk_off[c]
// + I] (I = 0 .. tiles of the parent's front) is the first of c's update
// rows whose parent row lies in tile row I or later (brk_off[c] = 0 for
// the other supernodes).
// Forward-solve gather lists: the update-vector entries (offsets into the
// update vectors, z_off[c] + i) of a supernode's children that add into
// row position r of supernode t are fg_idx[fg_ptr[j] .. fg_ptr[j+1]),
// j = sn_rowptr[t] + r, in the order of t's children (each child adds at
// most once to a row).  A solve task sums them for its own rows, every row
// in the same order, without a pass per child.
struct CholPlan {
  std::vector<int8_t> sn_class;
  std::vector<int32_t> fg_ptr, fg_idx;
  std::vector<int32_t> bot_ptr, bot_sn, bot_stage, brk_off, tile_brk;
  std::vector<int32_t> grp_ptr, grp_sn, grp_lptr, grp_lev;
  // factorization's task kernel; warp tasks (forward_warp, backward_warp:
  // one warp-small supernode each, every dependency earlier in the list;
  // forward_warp also orders the factorization's warp tasks) and block
  // tasks of the solves (forward, backward: the other supernodes)
  CholGraph factor, forward, backward, forward_warp, backward_warp;
  // the list schedule's estimates: makespan, critical path, and the
  // critical path's time by task kind
  double est_factor_us = 0.0, est_critical_us = 0.0, est_critical_by_kind[8] = {};
};

// Thresholds of the plan (the defaults are the library's).
struct CholPlanParams {
  double group_fma = 20000.0;  // work of one group task at most
  int32_t group_members = 64;
  double tile_fma = 30000.0;  // supernodes above this work are tiled
  int32_t workers = 304;       // concurrent blocks the list schedule assumes
  int32_t warps = 4864;        // concurrent warps of the warp tasks
};

// Builds the plan for the symbolic factorization sy (its supernodes, row
// structures and children).
acopf_status chol_plan(const CholSymbolic& sy, const CholPlanParams& prm, CholPlan& plan,
                       std::string& err);

}  // namespace acopf
