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
#include <atomic>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <utility>

namespace acopf {
namespace {

// Host threads of the parallel passes.
constexpr int32_t kSymbolicThreads = 8;
// Relaxed supernodes: a merge that stays within kRelaxSmallCols columns and
// kRelaxSmallRows rows may carry up to kRelaxSmallZeros of its entries as
// explicit zeros, any other up to kRelaxZeros.
constexpr int32_t kRelaxSmallCols = 8, kRelaxSmallRows = 32;
constexpr double kRelaxSmallZeros = 0.3, kRelaxZeros = 0.05;

// Runs fn(t0, t1) over [0, n) in up to kSymbolicThreads slices (fewer for
// small n; the calling thread takes the first slice and any a thread could
// not be started for).
template <typename Fn>
void parallel_slices(int32_t n, int64_t work, Fn fn) {
  const int32_t nth = int32_t(std::min<int64_t>(kSymbolicThreads, 1 + work / 262144));
  auto lo = [&](int32_t t) { return int32_t(int64_t(n) * t / nth); };
  std::vector<std::thread> pool;
  int32_t t = 1;
  try {
    for (; t < nth; ++t) pool.emplace_back(fn, lo(t), lo(t + 1));
  } catch (const std::system_error&) {  // no thread: the slice runs here
  }
  for (int32_t u = t; u < nth; ++u) fn(lo(u), lo(u + 1));
  fn(lo(0), lo(1));
  for (auto& th : pool) th.join();
}

}  // namespace

acopf_status chol_symbolic(int32_t n, const std::vector<int32_t>& rp,
                           const std::vector<int32_t>& ci, CholSymbolic& sy, std::string& err) {
  try {
    sy = CholSymbolic{};
    sy.n = n;
    const int64_t nnz_low = rp[size_t(n)];
    // --- the symmetric pattern without its diagonal (both triangles) ------
    std::vector<int32_t> gp(size_t(n) + 1, 0), gi;
    {
      // node v's list: its row's lower entries (input order), then the rows
      // below it that hold v (ascending).  Slices of the rows in parallel:
      // each slice counts the transposed entries it contributes per node,
      // a prefix over (node, slice) gives every slice its own cursors, and
      // the slices (ascending rows) fill in parallel without atomics: the
      // same lists as a sequential pass.
      constexpr int32_t S = kSymbolicThreads;
      std::vector<int32_t> ap(size_t(n) + 1, 0), ai, nlow(static_cast<size_t>(n));
      std::vector<int32_t> cur(size_t(S) * size_t(n), 0);  // slice q's count, then cursor, of node v
      auto slice_lo = [&](int32_t q) { return int32_t(int64_t(n) * q / S); };
      auto by_slice = [&](auto fn) {
        std::vector<std::thread> pool;
        int32_t q = 1;
        try {
          for (; q < S; ++q) pool.emplace_back(fn, q);
        } catch (const std::system_error&) {
        }
        for (int32_t u = q; u < S; ++u) fn(u);
        fn(0);
        for (auto& th : pool) th.join();
      };
      by_slice([&](int32_t q) {
        int32_t* c = cur.data() + size_t(q) * size_t(n);
        for (int32_t i = slice_lo(q); i < slice_lo(q + 1); ++i) {
          int32_t nl = 0;
          for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
            const int32_t j = ci[size_t(k)];
            if (j == i) continue;
            ++nl;
            ++c[j];
          }
          nlow[size_t(i)] = nl;
        }
      });
      for (int32_t v = 0; v < n; ++v) {
        int32_t o = ap[size_t(v)] + nlow[size_t(v)];
        for (int32_t q = 0; q < S; ++q) {
          int32_t& c = cur[size_t(q) * size_t(n) + size_t(v)];
          const int32_t cnt = c;
          c = o;
          o += cnt;
        }
        ap[size_t(v) + 1] = o;
      }
      ai.resize(size_t(ap[size_t(n)]));
      by_slice([&](int32_t q) {
        int32_t* c = cur.data() + size_t(q) * size_t(n);
        for (int32_t i = slice_lo(q); i < slice_lo(q + 1); ++i) {
          int32_t o = ap[size_t(i)];
          for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
            const int32_t j = ci[size_t(k)];
            if (j == i) continue;
            ai[size_t(o++)] = j;
            ai[size_t(c[j]++)] = i;
          }
        }
      });
      // --- locality: the nodes renumbered breadth first (each component
      // from its lowest unvisited node), so that the order and the passes
      // after it, which walk the graph, find neighbours near each other in
      // memory.  bfs[v] is the input node numbered v, nid its inverse.
      std::vector<int32_t> bfs, nid(static_cast<size_t>(n), -1);
      bfs.reserve(size_t(n));
      for (int32_t r = 0; r < n; ++r) {
        if (nid[size_t(r)] >= 0) continue;
        nid[size_t(r)] = int32_t(bfs.size());
        bfs.push_back(r);
        for (size_t h = bfs.size() - 1; h < bfs.size(); ++h) {
          const int32_t v = bfs[h];
          for (int32_t k = ap[size_t(v)]; k < ap[size_t(v) + 1]; ++k) {
            const int32_t u = ai[size_t(k)];
            if (nid[size_t(u)] < 0) {
              nid[size_t(u)] = int32_t(bfs.size());
              bfs.push_back(u);
            }
          }
        }
      }
      gi.resize(ai.size());
      for (int32_t v = 0; v < n; ++v)
        gp[size_t(v) + 1] = gp[size_t(v)] + ap[size_t(bfs[size_t(v)]) + 1] - ap[size_t(bfs[size_t(v)])];
      parallel_slices(n, int64_t(ai.size()), [&](int32_t v0, int32_t v1) {
        for (int32_t v = v0; v < v1; ++v) {
          const int32_t o = bfs[size_t(v)];
          int32_t t = gp[size_t(v)];
          for (int32_t k = ap[size_t(o)]; k < ap[size_t(o) + 1]; ++k) gi[size_t(t++)] = nid[size_t(ai[size_t(k)])];
        }
      });
      sy.perm.swap(bfs);  // (for now: the renumbering)
    }
    // --- fill-reducing order: approximate minimum degree (amd.cpp) -------
    std::vector<int32_t> md;  // md[k]: the (renumbered) node eliminated k-th
    if (!approximate_minimum_degree(n, gp, gi, md)) {
      err = "the fill-reducing order failed";
      return ACOPF_E_INVALID_ARG;
    }
    // lower rows of the matrix in an order (ord[k]: the node at position k,
    // ipos its inverse), gathered row by row from the adjacency; with
    // `upper`, the entries above the diagonal by rows too (= the lower
    // triangle by columns)
    // (rows counted, then filled, in parallel slices of the order)
    auto gather_rows = [&](const std::vector<int32_t>& ord, const std::vector<int32_t>& ipos,
                           std::vector<int32_t>& lrp, std::vector<int32_t>& lci,
                           std::vector<int32_t>* urp, std::vector<int32_t>* uci) {
      lrp.assign(size_t(n) + 1, 0);
      if (urp) urp->assign(size_t(n) + 1, 0);
      parallel_slices(n, int64_t(gi.size()), [&](int32_t k0, int32_t k1) {
        for (int32_t k = k0; k < k1; ++k) {
          const int32_t v = ord[size_t(k)];
          int32_t nlow = 0;
          for (int32_t q = gp[size_t(v)]; q < gp[size_t(v) + 1]; ++q)
            nlow += ipos[size_t(gi[size_t(q)])] < k;
          lrp[size_t(k) + 1] = nlow;
          if (urp) (*urp)[size_t(k) + 1] = gp[size_t(v) + 1] - gp[size_t(v)] - nlow;
        }
      });
      for (int32_t k = 0; k < n; ++k) lrp[size_t(k) + 1] += lrp[size_t(k)];
      lci.resize(size_t(lrp[size_t(n)]));
      if (urp) {
        for (int32_t k = 0; k < n; ++k) (*urp)[size_t(k) + 1] += (*urp)[size_t(k)];
        uci->resize(size_t((*urp)[size_t(n)]));
      }
      parallel_slices(n, int64_t(gi.size()), [&](int32_t k0, int32_t k1) {
        for (int32_t k = k0; k < k1; ++k) {
          const int32_t v = ord[size_t(k)];
          int32_t pl = lrp[size_t(k)], pu = urp ? (*urp)[size_t(k)] : 0;
          for (int32_t q = gp[size_t(v)]; q < gp[size_t(v) + 1]; ++q) {
            const int32_t a = ipos[size_t(gi[size_t(q)])];
            if (a < k)
              lci[size_t(pl++)] = a;
            else if (urp)
              (*uci)[size_t(pu++)] = a;
          }
        }
      });
    };

    // --- elimination tree of the reordered matrix (Liu) ----------------
    std::vector<int32_t> brp, bci, parent(static_cast<size_t>(n), -1);
    {
      std::vector<int32_t> ipmd(static_cast<size_t>(n));
      for (int32_t k = 0; k < n; ++k) ipmd[size_t(md[size_t(k)])] = k;
      gather_rows(md, ipmd, brp, bci, nullptr, nullptr);
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
    }

    // --- postorder (children in ascending order, depth first) -----------
    // Without a search: a parent's number exceeds its children's, so one
    // ascending pass sums the subtree sizes and places each child's subtree
    // after its smaller siblings' inside its parent's range (roots one after
    // another, ascending), one descending pass turns those offsets into
    // ranges, and each node ends its own range.
    std::vector<int32_t> post(static_cast<size_t>(n));
    {
      std::vector<int32_t> size(static_cast<size_t>(n), 1), off(static_cast<size_t>(n), 0),
          acc(static_cast<size_t>(n), 0);
      for (int32_t v = 0; v < n; ++v)
        if (parent[size_t(v)] >= 0) size[size_t(parent[size_t(v)])] += size[size_t(v)];
      int32_t roots = 0;
      for (int32_t v = 0; v < n; ++v) {
        const int32_t p = parent[size_t(v)];
        if (p >= 0) {
          off[size_t(v)] = acc[size_t(p)];
          acc[size_t(p)] += size[size_t(v)];
        } else {
          off[size_t(v)] = roots;
          roots += size[size_t(v)];
        }
      }
      for (int32_t v = n - 1; v >= 0; --v) {  // off becomes the first position of v's subtree
        const int32_t p = parent[size_t(v)];
        if (p >= 0) off[size_t(v)] += off[size_t(p)];
        post[size_t(off[size_t(v)] + size[size_t(v)] - 1)] = v;
      }
    }
    // final order: position k holds the renumbered node ordf[k] = md[post[k]],
    // the input node perm[k].  A postorder of the elimination tree is an
    // equivalent order: the tree of the reordered matrix is the same tree,
    // relabelled.
    std::vector<int32_t> ordf(static_cast<size_t>(n)), ipf(static_cast<size_t>(n));
    {
      std::vector<int32_t> fpos(static_cast<size_t>(n)), par(static_cast<size_t>(n));
      for (int32_t k = 0; k < n; ++k) fpos[size_t(post[size_t(k)])] = k;
      for (int32_t k = 0; k < n; ++k) {
        const int32_t p = parent[size_t(post[size_t(k)])];
        par[size_t(k)] = p < 0 ? -1 : fpos[size_t(p)];
        ordf[size_t(k)] = md[size_t(post[size_t(k)])];
        ipf[size_t(ordf[size_t(k)])] = k;
      }
      parent.swap(par);
      std::vector<int32_t> perm(static_cast<size_t>(n));
      for (int32_t k = 0; k < n; ++k) perm[size_t(k)] = sy.perm[size_t(ordf[size_t(k)])];
      sy.perm.swap(perm);
    }
    std::vector<int32_t> crp, cri;  // the lower triangle by columns
    gather_rows(ordf, ipf, brp, bci, &crp, &cri);
    std::vector<int32_t>().swap(gi);

    // --- column counts (row subtrees; rows in parallel slices, each with
    // its own marks, the counts added atomically) --------------------------
    std::vector<int64_t> cnt(static_cast<size_t>(n), 0);
    std::vector<int32_t> mark(static_cast<size_t>(n), -1), nchild(static_cast<size_t>(n), 0);
    parallel_slices(n, int64_t(bci.size()) * 2, [&](int32_t i0, int32_t i1) {
      std::vector<int32_t> own;
      int32_t* mk = mark.data();
      if (i0 != 0) {  // the first slice uses the shared marks, the others their own
        own.assign(static_cast<size_t>(n), -1);
        mk = own.data();
      }
      for (int32_t i = i0; i < i1; ++i) {
        mk[i] = i;
        for (int32_t k = brp[size_t(i)]; k < brp[size_t(i) + 1]; ++k)
          for (int32_t j = bci[size_t(k)]; j != -1 && mk[j] != i; j = parent[size_t(j)]) {
            mk[j] = i;
            __atomic_fetch_add(&cnt[size_t(j)], int64_t(1), __ATOMIC_RELAXED);
          }
      }
    });
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
    // --- relaxed supernodes: a supernode absorbs the child whose columns end
    // where its own begin when the merged supernode stays within
    // kMaxSupernodeWidth columns and the explicit zeros it carries (rows of
    // the parent's structure missing from the child's columns) are few
    // enough for its size class.  The merged columns' rows are the child's
    // columns then the parent's rows; the zeros stay exactly zero in the
    // numeric factorization.
    {
      const int32_t nf = int32_t(sy.sn_first.size());
      sy.sn_first.push_back(n);
      std::vector<int32_t> mfirst(static_cast<size_t>(nf)), mw(static_cast<size_t>(nf)),
          mh(static_cast<size_t>(nf));
      std::vector<int64_t> mz(static_cast<size_t>(nf), 0);
      std::vector<char> absorbed(static_cast<size_t>(nf), 0);
      for (int32_t t = 0; t < nf; ++t) {
        const int32_t f = sy.sn_first[size_t(t)], w = sy.sn_first[size_t(t) + 1] - f;
        const int32_t h = int32_t(cnt[size_t(f)]) + 1;
        mfirst[size_t(t)] = f;
        mw[size_t(t)] = w;
        mh[size_t(t)] = h;
        if (t == 0 || parent[size_t(f) - 1] < f || parent[size_t(f) - 1] >= f + w) continue;
        const int32_t c = t - 1;  // the child ending at column f
        const int64_t W = mw[size_t(c)] + w, H = mw[size_t(c)] + h;
        const int64_t z = mz[size_t(c)] + int64_t(mw[size_t(c)]) * (H - mh[size_t(c)]);
        const double frac = double(z) / double(W * H - W * (W - 1) / 2);
        const bool ok = W <= kMaxSupernodeWidth &&
                        ((W <= kRelaxSmallCols && H <= kRelaxSmallRows && frac <= kRelaxSmallZeros) ||
                         frac <= kRelaxZeros);
        if (!ok) continue;
        absorbed[size_t(c)] = 1;
        mfirst[size_t(t)] = mfirst[size_t(c)];
        mw[size_t(t)] = int32_t(W);
        mh[size_t(t)] = int32_t(H);
        mz[size_t(t)] = z;
      }
      std::vector<int32_t> first;
      for (int32_t t = 0; t < nf; ++t)
        if (!absorbed[size_t(t)]) first.push_back(mfirst[size_t(t)]);
      sy.sn_first.swap(first);
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

    // --- children of each supernode (ascending) --------------------------
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

    // --- row structures: own columns, the lower entries of the reordered
    // matrix's columns in the supernode, and the children's rows below
    // their columns
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
      for (int32_t q = sy.kid_ptr[size_t(s)]; q < sy.kid_ptr[size_t(s) + 1]; ++q) {
        const int32_t c = sy.kid[size_t(q)];
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
    // (entry (i, j) lands in column c = min(pos i, pos j) of its supernode, at
    // row r = max(...): a row among the supernode's own columns directly, one
    // below them by binary search; the input's rows visited in the order, in
    // parallel slices)
    sy.amap.resize(size_t(nnz_low));
    {
      std::vector<int32_t> ipin(static_cast<size_t>(n));  // input node -> position
      for (int32_t k = 0; k < n; ++k) ipin[size_t(sy.perm[size_t(k)])] = k;
      std::atomic<bool> missing{false};
      auto slice = [&](int32_t a0, int32_t a1) {  // the input's rows at positions [a0, a1)
        for (int32_t a = a0; a < a1; ++a) {
          const int32_t i = sy.perm[size_t(a)];
          for (int32_t k = rp[size_t(i)]; k < rp[size_t(i) + 1]; ++k) {
            const int32_t b = ipin[size_t(ci[size_t(k)])];
            const int32_t c = std::min(a, b), r = std::max(a, b), sn = sn_of[size_t(c)];
            const int32_t f = sy.sn_first[size_t(sn)], w = sy.sn_first[size_t(sn) + 1] - f;
            const int32_t* R = sy.rowidx.data() + sy.sn_rowptr[size_t(sn)];
            const int32_t h = sy.sn_rowptr[size_t(sn) + 1] - sy.sn_rowptr[size_t(sn)];
            int32_t pos = r - f;
            if (pos >= w) {
              pos = int32_t(std::lower_bound(R + w, R + h, r) - R);
              if (pos == h || R[pos] != r) {
                missing = true;
                return;
              }
            }
            sy.amap[size_t(k)] = sy.sn_off[size_t(sn)] + int64_t(c - f) * h + pos;
          }
        }
      };
      const int32_t nth = int32_t(std::min<int64_t>(kSymbolicThreads, 1 + nnz_low / 262144));
      auto lo = [&](int32_t t) { return int32_t(int64_t(n) * t / nth); };
      std::vector<std::thread> pool;
      int32_t t = 1;
      try {
        for (; t < nth; ++t) pool.emplace_back(slice, lo(t), lo(t + 1));
      } catch (const std::system_error&) {  // no thread: the slice runs here
      }
      for (int32_t u = t; u < nth; ++u) slice(lo(u), lo(u + 1));
      slice(lo(0), lo(1));
      for (auto& th : pool) th.join();
      if (missing) {
        err = "symbolic phase: an entry of M_cond is missing from the factor's structure";
        return ACOPF_E_INVALID_ARG;
      }
    }

    // --- multifrontal links: the positions of a child's rows below its
    // columns within its parent's rows, and the offsets of the update
    // matrices (m x m, m = h - w) and vectors
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
