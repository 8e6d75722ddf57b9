// Symbolic phase of the sparse Cholesky factorization of M_cond (host):
// fill-reducing order, elimination tree, supernodes, the layout of the
// factor and the multifrontal links (children, row maps, update matrices)
// the numeric kernels follow.
//
// Sec. V factorizes M_cond with a fill-reducing order fixed once per
// pattern and refactors numerically every iteration; this is the once-per-
// pattern part.  The order is approximate minimum degree (amd.cpp), the
// order family the paper's solvers use.
#include "symbolic.h"

#include <algorithm>
#include <new>
#include <string>
#include <utility>

namespace acopf {
namespace {

}  // namespace

acopf_status chol_symbolic(int32_t n, const std::vector<int32_t>& rp,
                           const std::vector<int32_t>& ci, CholSymbolic& sy, std::string& err) {
  try {
    sy = CholSymbolic{};
    sy.n = n;
    const int64_t nnz_low = rp[size_t(n)];
    // --- fill-reducing order: approximate minimum degree (amd.cpp) -------
    std::vector<int32_t> ap(size_t(n) + 1, 0), ai;
    for (int32_t i = 0; i < n; ++i)
      for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k)
        if (ci[size_t(k)] != i) {
          ap[size_t(i) + 1]++;
          ap[size_t(ci[size_t(k)]) + 1]++;
        }
    for (int32_t i = 0; i < n; ++i) ap[size_t(i) + 1] += ap[size_t(i)];
    ai.resize(size_t(ap[size_t(n)]));
    {
      std::vector<int32_t> nx(ap.begin(), ap.end() - 1);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
          const int32_t j = ci[size_t(k)];
          if (j == i) continue;
          ai[size_t(nx[size_t(i)]++)] = j;
          ai[size_t(nx[size_t(j)]++)] = i;
        }
    }
    std::vector<int32_t> md;
    if (!approximate_minimum_degree(n, ap, ai, md)) {
      err = "the fill-reducing order failed";
      return ACOPF_E_INVALID_ARG;
    }
    std::vector<int32_t>().swap(ai);
    std::vector<int32_t> ipmd(static_cast<size_t>(n));
    for (int32_t k = 0; k < n; ++k) ipmd[size_t(md[size_t(k)])] = k;

    // --- elimination tree of the reordered matrix (Liu) ----------------
    // lower rows of B = P M P': for each row r the columns c < r
    auto lower_rows = [&](const std::vector<int32_t>& ip, std::vector<int32_t>& brp,
                          std::vector<int32_t>& bci) {
      brp.assign(size_t(n) + 1, 0);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
          const int32_t a = ip[size_t(i)], b = ip[size_t(ci[size_t(k)])];
          if (a != b) brp[size_t(std::max(a, b)) + 1]++;
        }
      for (int32_t i = 0; i < n; ++i) brp[size_t(i) + 1] += brp[size_t(i)];
      bci.resize(size_t(brp[size_t(n)]));
      std::vector<int32_t> nx(brp.begin(), brp.end() - 1);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
          const int32_t a = ip[size_t(i)], b = ip[size_t(ci[size_t(k)])];
          if (a != b) bci[size_t(nx[size_t(std::max(a, b))]++)] = std::min(a, b);
        }
    };
    auto etree = [&](const std::vector<int32_t>& brp, const std::vector<int32_t>& bci,
                     std::vector<int32_t>& parent) {
      parent.assign(static_cast<size_t>(n), -1);
      std::vector<int32_t> anc(static_cast<size_t>(n), -1);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = brp[size_t(i)]; k < brp[size_t(i) + 1]; ++k) {
          int32_t r = bci[size_t(k)];
          while (anc[size_t(r)] != -1 && anc[size_t(r)] != i) {
            const int32_t t = anc[size_t(r)];
            anc[size_t(r)] = i;
            r = t;
          }
          if (anc[size_t(r)] == -1) {
            anc[size_t(r)] = i;
            parent[size_t(r)] = i;
          }
        }
    };
    std::vector<int32_t> brp, bci, parent;
    lower_rows(ipmd, brp, bci);
    etree(brp, bci, parent);

    // --- postorder (children in ascending order, depth first) -----------
    std::vector<int32_t> head(static_cast<size_t>(n), -1), next(static_cast<size_t>(n), -1), post;
    post.reserve(size_t(n));
    for (int32_t v = n - 1; v >= 0; --v)
      if (parent[size_t(v)] >= 0) {
        next[size_t(v)] = head[size_t(parent[size_t(v)])];
        head[size_t(parent[size_t(v)])] = v;
      }
    std::vector<int32_t> stack;
    for (int32_t root = 0; root < n; ++root) {
      if (parent[size_t(root)] != -1) continue;
      stack.push_back(root);
      while (!stack.empty()) {
        const int32_t v = stack.back();
        const int32_t c = head[size_t(v)];
        if (c == -1) {
          post.push_back(v);
          stack.pop_back();
        } else {
          head[size_t(v)] = next[size_t(c)];
          stack.push_back(c);
        }
      }
    }
    // final order: position k holds M's row md[post[k]]
    sy.perm.resize(size_t(n));
    std::vector<int32_t> ip(static_cast<size_t>(n));
    for (int32_t k = 0; k < n; ++k) {
      sy.perm[size_t(k)] = md[size_t(post[size_t(k)])];
      ip[size_t(sy.perm[size_t(k)])] = k;
    }
    lower_rows(ip, brp, bci);
    etree(brp, bci, parent);

    // --- column counts (row subtrees) -----------------------------------
    std::vector<int64_t> cnt(static_cast<size_t>(n), 0);
    std::vector<int32_t> mark(static_cast<size_t>(n), -1), nchild(static_cast<size_t>(n), 0);
    for (int32_t i = 0; i < n; ++i) {
      mark[size_t(i)] = i;
      for (int32_t k = brp[size_t(i)]; k < brp[size_t(i) + 1]; ++k)
        for (int32_t j = bci[size_t(k)]; j != -1 && mark[size_t(j)] != i; j = parent[size_t(j)]) {
          mark[size_t(j)] = i;
          cnt[size_t(j)]++;
        }
    }
    for (int32_t j = 0; j < n; ++j)
      if (parent[size_t(j)] >= 0) nchild[size_t(parent[size_t(j)])]++;

    // --- fundamental supernodes: j joins j-1's supernode when j is j-1's
    // parent, its only child, and L(:, j) is L(:, j-1) without row j
    sy.sn_first.clear();
    for (int32_t j = 0; j < n; ++j) {
      const bool join = j > 0 && parent[size_t(j) - 1] == j && nchild[size_t(j)] == 1 &&
                        cnt[size_t(j) - 1] == cnt[size_t(j)] + 1 &&
                        j - sy.sn_first.back() < kMaxSupernodeWidth;
      if (!join) sy.sn_first.push_back(j);
    }
    sy.ns = int32_t(sy.sn_first.size());
    sy.sn_first.push_back(n);
    const int32_t ns = sy.ns;
    std::vector<int32_t> sn_of(static_cast<size_t>(n));
    for (int32_t s = 0; s < ns; ++s)
      for (int32_t j = sy.sn_first[size_t(s)]; j < sy.sn_first[size_t(s) + 1]; ++j)
        sn_of[size_t(j)] = s;
    sy.sn_parent.assign(static_cast<size_t>(ns), -1);
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t p = parent[size_t(sy.sn_first[size_t(s) + 1]) - 1];
      sy.sn_parent[size_t(s)] = p < 0 ? -1 : sn_of[size_t(p)];
    }

    // --- row structures: own columns, the lower entries of B's columns in
    // the supernode, and the children's rows below their columns
    std::vector<int32_t> crp(static_cast<size_t>(n) + 1, 0), cri;  // lower B by columns
    for (int32_t i = 0; i < n; ++i)
      for (int32_t k = brp[size_t(i)]; k < brp[size_t(i) + 1]; ++k) crp[size_t(bci[size_t(k)]) + 1]++;
    for (int32_t j = 0; j < n; ++j) crp[size_t(j) + 1] += crp[size_t(j)];
    cri.resize(size_t(crp[size_t(n)]));
    {
      std::vector<int32_t> nx(crp.begin(), crp.end() - 1);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = brp[size_t(i)]; k < brp[size_t(i) + 1]; ++k)
          cri[size_t(nx[size_t(bci[size_t(k)])]++)] = i;
    }
    std::vector<std::vector<int32_t>> kids(static_cast<size_t>(ns));
    for (int32_t s = 0; s < ns; ++s)
      if (sy.sn_parent[size_t(s)] >= 0) kids[size_t(sy.sn_parent[size_t(s)])].push_back(s);
    sy.sn_rowptr.assign(size_t(ns) + 1, 0);
    sy.rowidx.clear();
    std::fill(mark.begin(), mark.end(), -1);
    std::vector<int32_t> rows;
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t f = sy.sn_first[size_t(s)], l = sy.sn_first[size_t(s) + 1];
      rows.clear();
      for (int32_t j = f; j < l; ++j) {
        rows.push_back(j);
        mark[size_t(j)] = s;
      }
      for (int32_t j = f; j < l; ++j)
        for (int32_t k = crp[size_t(j)]; k < crp[size_t(j) + 1]; ++k) {
          const int32_t r = cri[size_t(k)];
          if (mark[size_t(r)] != s) {
            mark[size_t(r)] = s;
            rows.push_back(r);
          }
        }
      for (const int32_t c : kids[size_t(s)]) {
        const int32_t wc = sy.sn_first[size_t(c) + 1] - sy.sn_first[size_t(c)];
        for (int32_t p = sy.sn_rowptr[size_t(c)] + wc; p < sy.sn_rowptr[size_t(c) + 1]; ++p) {
          const int32_t r = sy.rowidx[size_t(p)];
          if (mark[size_t(r)] != s) {
            mark[size_t(r)] = s;
            rows.push_back(r);
          }
        }
      }
      std::sort(rows.begin() + (l - f), rows.end());
      sy.rowidx.insert(sy.rowidx.end(), rows.begin(), rows.end());
      sy.sn_rowptr[size_t(s) + 1] = int32_t(sy.rowidx.size());
      if (int64_t(sy.rowidx.size()) > INT32_MAX / 2) {
        err = "the factor's row structures exceed the 32-bit index range";
        return ACOPF_E_INVALID_ARG;
      }
    }

    for (int32_t s = 0; s < ns; ++s) {
      const int32_t m = (sy.sn_rowptr[size_t(s) + 1] - sy.sn_rowptr[size_t(s)]) -
                        (sy.sn_first[size_t(s) + 1] - sy.sn_first[size_t(s)]);
      if (m > kMaxRowsBelow) {
        err = "a supernode has " + std::to_string(m) + " rows below its columns (at most " +
              std::to_string(kMaxRowsBelow) + " are supported)";
        return ACOPF_E_INVALID_ARG;
      }
    }

    // --- storage: supernode s is an h x w column-major block -------------
    sy.sn_off.assign(size_t(ns) + 1, 0);
    for (int32_t s = 0; s < ns; ++s) {
      const int64_t w = sy.sn_first[size_t(s) + 1] - sy.sn_first[size_t(s)];
      const int64_t h = sy.sn_rowptr[size_t(s) + 1] - sy.sn_rowptr[size_t(s)];
      sy.sn_off[size_t(s) + 1] = sy.sn_off[size_t(s)] + w * h;
    }

    // --- assembly map: lower entry k of M -> its place in the blocks -----
    // (entries grouped by their column in the order, then one supernode at a
    // time with the positions of its rows in a scatter map)
    sy.amap.resize(size_t(nnz_low));
    {
      std::vector<int32_t> cptr(size_t(n) + 1, 0), ck(static_cast<size_t>(nnz_low));
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k)
          cptr[size_t(std::min(ip[size_t(i)], ip[size_t(ci[size_t(k)])])) + 1]++;
      for (int32_t c = 0; c < n; ++c) cptr[size_t(c) + 1] += cptr[size_t(c)];
      std::vector<int32_t> nx(cptr.begin(), cptr.end() - 1);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k)
          ck[size_t(nx[size_t(std::min(ip[size_t(i)], ip[size_t(ci[size_t(k)])]))]++)] = k;
      std::vector<int32_t> rowpos(static_cast<size_t>(n), -1);
      std::vector<int32_t> krow(static_cast<size_t>(nnz_low));  // entry k's row of M
      for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) krow[size_t(k)] = i;
      for (int32_t s = 0; s < ns; ++s) {
        const int32_t f = sy.sn_first[size_t(s)], l = sy.sn_first[size_t(s) + 1];
        const int32_t* R = sy.rowidx.data() + sy.sn_rowptr[size_t(s)];
        const int32_t h = sy.sn_rowptr[size_t(s) + 1] - sy.sn_rowptr[size_t(s)];
        for (int32_t q = 0; q < h; ++q) rowpos[size_t(R[q])] = q;
        for (int32_t c = f; c < l; ++c)
          for (int32_t t = cptr[size_t(c)]; t < cptr[size_t(c) + 1]; ++t) {
            const int32_t k = ck[size_t(t)];
            const int32_t r = std::max(ip[size_t(krow[size_t(k)])], ip[size_t(ci[size_t(k)])]);
            const int32_t pos = rowpos[size_t(r)];
            if (pos < 0 || R[pos] != r) {
              err = "symbolic phase: an entry of M_cond is missing from the factor's structure";
              return ACOPF_E_INVALID_ARG;
            }
            sy.amap[size_t(k)] = sy.sn_off[size_t(s)] + int64_t(c - f) * h + pos;
          }
        for (int32_t q = 0; q < h; ++q) rowpos[size_t(R[q])] = -1;
      }
    }

    // --- multifrontal links: each supernode's children (ascending), the
    // positions of a child's rows below its columns within its parent's rows,
    // and the offsets of the update matrices (m x m, m = h - w) and vectors
    sy.kid_ptr.assign(size_t(ns) + 1, 0);
    for (int32_t c = 0; c < ns; ++c)
      if (sy.sn_parent[size_t(c)] >= 0) sy.kid_ptr[size_t(sy.sn_parent[size_t(c)]) + 1]++;
    for (int32_t t = 0; t < ns; ++t) sy.kid_ptr[size_t(t) + 1] += sy.kid_ptr[size_t(t)];
    sy.kid.resize(size_t(sy.kid_ptr[size_t(ns)]));
    {
      std::vector<int32_t> nx(sy.kid_ptr.begin(), sy.kid_ptr.end() - 1);
      for (int32_t c = 0; c < ns; ++c)
        if (sy.sn_parent[size_t(c)] >= 0) sy.kid[size_t(nx[size_t(sy.sn_parent[size_t(c)])]++)] = c;
    }
    sy.rel_off.assign(size_t(ns), 0);
    sy.u_off.assign(size_t(ns) + 1, 0);
    sy.z_off.assign(size_t(ns) + 1, 0);
    for (int32_t c = 0; c < ns; ++c) {
      const int32_t wc = sy.sn_first[size_t(c) + 1] - sy.sn_first[size_t(c)];
      const int32_t r0 = sy.sn_rowptr[size_t(c)], hc = sy.sn_rowptr[size_t(c) + 1] - r0;
      const int64_t mc = hc - wc;
      sy.u_off[size_t(c) + 1] = sy.u_off[size_t(c)] + mc * mc;
      sy.z_off[size_t(c) + 1] = sy.z_off[size_t(c)] + mc;
      sy.rel_off[size_t(c)] = int32_t(sy.relmap.size());
      const int32_t t = sy.sn_parent[size_t(c)];
      if (t < 0) {
        if (mc != 0) {
          err = "symbolic phase: a root supernode has rows below its columns";
          return ACOPF_E_INVALID_ARG;
        }
        continue;
      }
      const int32_t ft = sy.sn_first[size_t(t)], wt = sy.sn_first[size_t(t) + 1] - ft;
      const int32_t* Rt = sy.rowidx.data() + sy.sn_rowptr[size_t(t)];
      const int32_t ht = sy.sn_rowptr[size_t(t) + 1] - sy.sn_rowptr[size_t(t)];
      int32_t q = 0;
      for (int32_t p = wc; p < hc; ++p) {
        const int32_t r = sy.rowidx[size_t(r0 + p)];
        if (r < ft) {
          err = "symbolic phase: a child's row precedes its parent's columns";
          return ACOPF_E_INVALID_ARG;
        }
        if (r < ft + wt) {
          q = r - ft;
        } else {
          if (q < wt) q = wt;
          while (q < ht && Rt[q] < r) ++q;
        }
        if (q >= ht || Rt[q] != r) {
          err = "symbolic phase: a child's row is missing from its parent's structure";
          return ACOPF_E_INVALID_ARG;
        }
        sy.relmap.push_back(q);
      }
      if (int64_t(sy.relmap.size()) > INT32_MAX) {
        err = "the update maps exceed the 32-bit index range";
        return ACOPF_E_INVALID_ARG;
      }
    }

    // --- depth of the supernodal tree (a statistic) -------------------------
    std::vector<int32_t> level(static_cast<size_t>(ns), 0);
    int32_t nlev = ns > 0 ? 1 : 0;
    for (int32_t s = 0; s < ns; ++s) {
      const int32_t p = sy.sn_parent[size_t(s)];
      if (p >= 0) {
        level[size_t(p)] = std::max(level[size_t(p)], level[size_t(s)] + 1);
        nlev = std::max(nlev, level[size_t(p)] + 1);
      }
    }

    // --- counts -------------------------------------------------------------
    acopf_chol_stats& st = sy.stats;
    st = acopf_chol_stats{};
    st.n = n;
    st.nnz_full = 2 * nnz_low - n;
    st.nnz_factor = n;
    for (int32_t j = 0; j < n; ++j) {
      const double c = double(cnt[size_t(j)]);
      st.nnz_factor += cnt[size_t(j)];
      st.max_col = std::max<int64_t>(st.max_col, cnt[size_t(j)] + 1);
      st.factor_flops += 1.0 + c + c * (c + 1.0);
    }
    st.n_supernodes = ns;
    st.n_levels = nlev;
    st.storage = sy.sn_off[size_t(ns)];
    st.update_storage = sy.u_off[size_t(ns)] + sy.z_off[size_t(ns)];
  } catch (const std::bad_alloc&) {
    err = "host allocation failed";
    return ACOPF_E_OOM;
  }
  return ACOPF_OK;
}

}  // namespace acopf
