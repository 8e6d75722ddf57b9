// Symbolic phase of the sparse Cholesky factorization of M_cond (host).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "acopf.h"

namespace acopf {

// Limits: adjacency entries of the elimination graph during the ordering,
// columns of one supernode, and rows below a supernode's columns.
constexpr int64_t kMaxGraphEntries = int64_t(1) << 28;
constexpr int32_t kMaxSupernodeWidth = 64;
constexpr int32_t kMaxRowsBelow = 4096;

// The factor L of P M_cond P' (P = perm) in supernodes: supernode s holds
// columns [sn_first[s], sn_first[s+1]) (w of them), its rows R_s =
// rowidx[sn_rowptr[s] .. sn_rowptr[s+1]) (h of them: its own columns first,
// then ascending), and its values as an h x w column-major block at
// sn_off[s].  Supernodes are numbered in a postorder of the supernodal
// elimination tree (every child before its parent).  Multifrontal links:
// the children of t are kid[kid_ptr[t] .. kid_ptr[t+1]) (ascending); child
// c's update matrix (m x m column-major, m = h - w, rows R_c[w:]) sits at
// u_off[c] and its update vector (m) at z_off[c]; relmap[rel_off[c] + i] is
// the position of R_c[w + i] in R_parent (ascending in i).  amap maps each
// entry of M_cond's lower CSR to its place in the blocks.
struct CholSymbolic {
  int32_t n = 0, ns = 0;
  std::vector<int32_t> perm;
  std::vector<int32_t> sn_first, sn_rowptr, rowidx, sn_parent;
  std::vector<int64_t> sn_off, amap, u_off, z_off;
  std::vector<int32_t> kid_ptr, kid, rel_off, relmap;
  acopf_chol_stats stats{};
};

// Approximate minimum degree order (amd.cpp) of the symmetric pattern whose
// adjacency (no diagonal, both triangles) is ai[ap[i] .. ap[i+1]): `order`
// lists the nodes in elimination order.  False if the order is incomplete.
bool approximate_minimum_degree(int32_t n, const std::vector<int32_t>& ap,
                                const std::vector<int32_t>& ai, std::vector<int32_t>& order);

// Builds the symbolic factorization of the symmetric matrix whose lower
// triangle has the CSR pattern (rp, ci) (columns ascending, diagonal last
// in every row).  On failure returns a status and sets `err`.
acopf_status chol_symbolic(int32_t n, const std::vector<int32_t>& rp,
                           const std::vector<int32_t>& ci, CholSymbolic& sy, std::string& err);

}  // namespace acopf
