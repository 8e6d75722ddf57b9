// Symbolic phase of the sparse Cholesky factorization of M_cond (host).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "acopf.h"

namespace acopf {

// Limits: adjacency entries of the elimination graph during the ordering,
// and columns of one supernode.
constexpr int64_t kMaxGraphEntries = int64_t(1) << 28;
constexpr int32_t kMaxSupernodeWidth = 64;
// Supernodes of at most kWarpMaxRows rows and kWarpMaxCols columns are
// handled by one warp; panels of at most kPanelSmemDoubles doubles are
// staged in shared memory.
constexpr int32_t kWarpMaxRows = 32;
constexpr int32_t kWarpMaxCols = 8;
constexpr int32_t kPanelSmemDoubles = 20480;
// Block-handled supernodes staging more than this many doubles go to a
// launch of their own, so the rest of a level keeps several blocks per SM.
constexpr int32_t kMediumSmemDoubles = 3072;
// Rows below a supernode's columns (the numeric kernels stage a child's row
// map of this many entries).
constexpr int32_t kMaxRowsBelow = 4096;

// The factor L of P M_cond P' (P = perm) in supernodes: supernode s holds
// columns [sn_first[s], sn_first[s+1]) (w of them), its rows R_s =
// rowidx[sn_rowptr[s] .. sn_rowptr[s+1]) (h of them: its own columns first,
// then ascending), and its values as an h x w column-major block at
// sn_off[s].  Multifrontal links: the children of t are kid[kid_ptr[t] ..
// kid_ptr[t+1]) (ascending); child c's update matrix (m x m column-major,
// m = h - w, rows R_c[w:]) sits at u_off[c] and its update vector (m) at
// z_off[c]; relmap[rel_off[c] + i] is the position of R_c[w + i] in
// R_parent.  level_sn lists the supernodes level by level (level_ptr),
// every supernode after its descendants, and within a level the
// level_large[v] large supernodes (not small enough for a warp) first, and
// among those the level_big[v] whose shared-memory staging (panel, or panel
// and update matrix, within kPanelSmemDoubles) exceeds kMediumSmemDoubles;
// level_smem_big[v] and level_smem[v] are the largest staging of the big
// and of the other large supernodes, level_small_stage[v] the largest panel
// plus update matrix of its small ones.  The 32 x 32 lower tiles of the update
// matrices that are not staged with their panel are tiles[tile_ptr[v] ..
// tile_ptr[v+1]) ({supernode, tile row, tile column, 0}).  amap maps
// each entry of M_cond's lower CSR to its place in the blocks.
struct CholSymbolic {
  int32_t n = 0, ns = 0;
  std::vector<int32_t> perm;
  std::vector<int32_t> sn_first, sn_rowptr, rowidx, sn_parent;
  std::vector<int64_t> sn_off, amap, u_off, z_off;
  std::vector<int32_t> kid_ptr, kid, rel_off, relmap, level_ptr, level_sn, level_large;
  std::vector<int32_t> tile_ptr, level_smem, level_big, level_smem_big, level_small_stage;
  std::vector<int32_t> tiles;  // 4 per tile
  acopf_chol_stats stats{};
};

// Builds the symbolic factorization of the symmetric matrix whose lower
// triangle has the CSR pattern (rp, ci) (columns ascending, diagonal last
// in every row).  On failure returns a status and sets `err`.
acopf_status chol_symbolic(int32_t n, const std::vector<int32_t>& rp,
                           const std::vector<int32_t>& ci, CholSymbolic& sy, std::string& err);

}  // namespace acopf
