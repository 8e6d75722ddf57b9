// Approximate minimum degree order of a symmetric sparsity pattern, written
// from the method of Amestoy, Davis and Duff ("An approximate minimum degree
// ordering algorithm", SIAM J. Matrix Anal. Appl. 17(4), 1996).
//
// The elimination graph is kept as a quotient graph: an eliminated pivot p
// becomes an element whose list L_p holds the (principal) variables of its
// clique, and a variable's list holds the elements it belongs to followed by
// the variables it is still directly adjacent to.  Per pivot:
//   1. L_p = the pivot's variables plus the variables of its elements, which
//      are absorbed into p;
//   2. for every element e adjacent to a variable of L_p, |L_e \ L_p| is
//      counted in one pass (a stamp w[e] set to |L_e| + stamp, minus the
//      weight of each variable of L_p found in L_e);
//   3. each variable i of L_p gets the approximate external degree
//      min(n - k, d_i + |L_p \ i|, |A_i \ i| + |L_p \ i| + sum |L_e \ L_p|),
//      its list is pruned (elements with L_e inside L_p are absorbed into p:
//      aggressive absorption; variables of L_p are dropped), and it is
//      eliminated together with p when p is its only neighbour (mass
//      elimination);
//   4. variables of L_p with identical lists are merged into supervariables
//      (candidates found by a hash of their lists).
// Ties in the degree go to the variable most recently placed in its degree
// list: the order is deterministic.  The result lists the pivots in
// elimination order, each followed by the variables merged into it.
#include "symbolic.h"

#include <algorithm>
#include <utility>

namespace acopf {

namespace {

constexpr int32_t kNone = -1;

// A well-mixed 64-bit image of a node number; a list's hash is the sum of
// its entries' images (independent of the entries' order).
inline uint64_t mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

struct Quotient {
  int32_t n;
  std::vector<int32_t> iw;           // the lists
  std::vector<int64_t> pe;           // start of node i's list in iw
  std::vector<int32_t> len, elen;    // list length; number of elements at its front
  std::vector<int32_t> nv;           // weight of a principal variable (0: merged away)
  std::vector<int32_t> degree;       // variable: approximate degree; element: |L_e|
  std::vector<int64_t> w;            // element stamps (0: absorbed)
  std::vector<int8_t> kind;          // 0 variable, 1 element, 2 gone (absorbed / merged / eliminated)
  std::vector<int32_t> head, next, last;  // degree lists
  std::vector<int32_t> mhead, mtail, mnext;  // members of a supervariable, in order
  int64_t used = 0;

  void list_insert(int32_t i, int32_t d) {
    degree[size_t(i)] = d;
    last[size_t(i)] = kNone;
    next[size_t(i)] = head[size_t(d)];
    if (head[size_t(d)] != kNone) last[size_t(head[size_t(d)])] = i;
    head[size_t(d)] = i;
  }
  void list_remove(int32_t i) {
    const int32_t d = degree[size_t(i)];
    if (last[size_t(i)] != kNone)
      next[size_t(last[size_t(i)])] = next[size_t(i)];
    else
      head[size_t(d)] = next[size_t(i)];
    if (next[size_t(i)] != kNone) last[size_t(next[size_t(i)])] = last[size_t(i)];
  }
  void merge_members(int32_t into, int32_t from) {
    mnext[size_t(mtail[size_t(into)])] = mhead[size_t(from)];
    mtail[size_t(into)] = mtail[size_t(from)];
  }
  // Moves every live list to the front of a fresh workspace of at least
  // `need` free entries.
  void compact(int64_t need) {
    std::vector<int32_t> fresh;
    int64_t live = 0;
    for (int32_t i = 0; i < n; ++i)
      if (kind[size_t(i)] != 2) live += len[size_t(i)];
    fresh.reserve(size_t(live + need + live / 4 + 16));
    for (int32_t i = 0; i < n; ++i) {
      if (kind[size_t(i)] == 2) continue;
      const int64_t p = pe[size_t(i)];
      pe[size_t(i)] = int64_t(fresh.size());
      fresh.insert(fresh.end(), iw.begin() + p, iw.begin() + p + len[size_t(i)]);
    }
    used = int64_t(fresh.size());
    fresh.resize(fresh.capacity());
    iw.swap(fresh);
  }
  void reserve(int64_t need) {
    if (used + need > int64_t(iw.size())) compact(need);
  }
};

}  // namespace

bool approximate_minimum_degree(int32_t n, const std::vector<int32_t>& ap,
                                const std::vector<int32_t>& ai, std::vector<int32_t>& order) {
  Quotient q;
  q.n = n;
  const int64_t nnz = ap[size_t(n)];
  q.iw.assign(size_t(nnz + nnz / 2 + 4 * int64_t(n) + 16), 0);
  std::copy(ai.begin(), ai.begin() + nnz, q.iw.begin());
  q.used = nnz;
  q.pe.resize(size_t(n));
  q.len.resize(size_t(n));
  q.elen.assign(size_t(n), 0);
  q.nv.assign(size_t(n), 1);
  q.degree.resize(size_t(n));
  q.w.assign(size_t(n), 1);
  q.kind.assign(size_t(n), 0);
  q.head.assign(size_t(n) + 1, kNone);
  q.next.assign(size_t(n), kNone);
  q.last.assign(size_t(n), kNone);
  q.mhead.resize(size_t(n));
  q.mtail.resize(size_t(n));
  q.mnext.assign(size_t(n), kNone);
  for (int32_t i = 0; i < n; ++i) {
    q.pe[size_t(i)] = ap[size_t(i)];
    q.len[size_t(i)] = ap[size_t(i) + 1] - ap[size_t(i)];
    q.mhead[size_t(i)] = q.mtail[size_t(i)] = i;
  }
  for (int32_t i = 0; i < n; ++i) q.list_insert(i, q.len[size_t(i)]);
  order.clear();
  order.reserve(size_t(n));
  int64_t wflg = 2;
  int32_t nel = 0, mindeg = 0;
  std::vector<int32_t> lp, old;                    // the new element's variables; a list's copy
  std::vector<std::pair<uint64_t, int32_t>> hashed;  // (hash, variable) for supervariables
  while (nel < n) {
    // --- the pivot: a variable of least approximate degree -----------------
    while (mindeg < n && q.head[size_t(mindeg)] == kNone) ++mindeg;
    if (mindeg >= n) return false;
    const int32_t p = q.head[size_t(mindeg)];
    q.list_remove(p);
    int32_t nvpiv = q.nv[size_t(p)];
    nel += nvpiv;
    q.nv[size_t(p)] = -nvpiv;  // negative: in L_p (excluded from it)
    // --- 1. L_p: p's own variables and the variables of its elements ------
    int64_t bound = q.len[size_t(p)];
    for (int32_t k = 0; k < q.elen[size_t(p)]; ++k) {
      const int32_t e = q.iw[size_t(q.pe[size_t(p)] + k)];
      if (q.w[size_t(e)] != 0) bound += q.len[size_t(e)];
    }
    q.reserve(bound);
    int64_t degme = 0;
    lp.clear();
    auto take = [&](int32_t j) {
      if (q.kind[size_t(j)] != 0 || q.nv[size_t(j)] <= 0) return;  // not a principal variable, or taken
      degme += q.nv[size_t(j)];
      q.nv[size_t(j)] = -q.nv[size_t(j)];
      lp.push_back(j);
      q.list_remove(j);
    };
    {
      const int64_t p0 = q.pe[size_t(p)];
      const int32_t ne = q.elen[size_t(p)], nl = q.len[size_t(p)];
      for (int32_t k = 0; k < ne; ++k) {
        const int32_t e = q.iw[size_t(p0 + k)];
        if (q.w[size_t(e)] == 0) continue;  // absorbed before
        for (int32_t t = 0; t < q.len[size_t(e)]; ++t) take(q.iw[size_t(q.pe[size_t(e)] + t)]);
        q.w[size_t(e)] = 0;  // e is absorbed into p
        q.kind[size_t(e)] = 2;
      }
      for (int32_t k = ne; k < nl; ++k) take(q.iw[size_t(p0 + k)]);
    }
    q.kind[size_t(p)] = 1;
    q.pe[size_t(p)] = q.used;
    q.len[size_t(p)] = int32_t(lp.size());
    q.elen[size_t(p)] = 0;
    std::copy(lp.begin(), lp.end(), q.iw.begin() + q.used);
    q.used += int64_t(lp.size());
    q.degree[size_t(p)] = int32_t(degme);
    q.w[size_t(p)] = 1;
    // --- 2. |L_e \ L_p| for the elements around L_p ------------------------
    wflg += int64_t(n) + 2;
    for (const int32_t i : lp) {
      const int64_t nvi = -q.nv[size_t(i)];
      for (int32_t k = 0; k < q.elen[size_t(i)]; ++k) {
        const int32_t e = q.iw[size_t(q.pe[size_t(i)] + k)];
        int64_t& we = q.w[size_t(e)];
        if (we == 0 || e == p) continue;
        if (we < wflg) we = wflg + q.degree[size_t(e)];
        we -= nvi;
      }
    }
    // --- 3. degrees, pruning, absorption, mass elimination ---------------
    hashed.clear();
    const int32_t nleft = n - nel;
    for (const int32_t i : lp) {
      const int32_t nvi = -q.nv[size_t(i)];
      const int64_t i0 = q.pe[size_t(i)];
      const int32_t ne = q.elen[size_t(i)], nl = q.len[size_t(i)];
      int64_t ext = 0;
      uint64_t hash = 0;
      // The new list (p, then live elements, then variables) is written in
      // place: it is shorter than the old one, which held p as a variable or
      // an element now absorbed into p.  The old list is read from a copy.
      old.assign(q.iw.begin() + i0, q.iw.begin() + i0 + nl);
      int64_t out = i0;
      q.iw[size_t(out++)] = p;
      for (int32_t k = 0; k < ne; ++k) {
        const int32_t e = old[size_t(k)];
        if (e == p || q.w[size_t(e)] == 0) continue;
        const int64_t dext = q.w[size_t(e)] - wflg;
        if (dext > 0) {
          ext += dext;
          q.iw[size_t(out++)] = e;
          hash += mix(uint64_t(e));
        } else {  // L_e inside L_p: aggressive absorption
          q.w[size_t(e)] = 0;
          q.kind[size_t(e)] = 2;
        }
      }
      const int32_t new_elen = int32_t(out - i0);
      for (int32_t k = ne; k < nl; ++k) {
        const int32_t j = old[size_t(k)];
        if (q.kind[size_t(j)] != 0 || q.nv[size_t(j)] <= 0) continue;  // in L_p, merged, eliminated
        ext += q.nv[size_t(j)];
        q.iw[size_t(out++)] = j;
        hash += mix(uint64_t(j));
      }
      q.elen[size_t(i)] = new_elen;
      q.len[size_t(i)] = int32_t(out - i0);
      if (new_elen == 1 && q.len[size_t(i)] == 1) {
        // p is i's only neighbour: i is eliminated together with p
        q.nv[size_t(i)] = 0;
        q.kind[size_t(i)] = 2;
        degme -= nvi;
        nvpiv += nvi;
        nel += nvi;
        q.merge_members(p, i);
        continue;
      }
      const int64_t lpi = degme - nvi;  // |L_p \ i| (degme already excludes the masses above)
      int64_t d = std::min<int64_t>(int64_t(q.degree[size_t(i)]) + lpi, ext + lpi);
      d = std::min<int64_t>(d, int64_t(nleft) - nvi);
      q.degree[size_t(i)] = int32_t(std::max<int64_t>(d, 0));
      hashed.push_back({hash + mix(uint64_t(q.len[size_t(i)]) << 32), i});
    }
    // --- 4. supervariables: identical lists among L_p's variables ---------
    std::sort(hashed.begin(), hashed.end());
    for (size_t a = 0; a < hashed.size();) {
      size_t b = a + 1;
      while (b < hashed.size() && hashed[b].first == hashed[a].first) ++b;
      for (size_t x = a; x + 1 < b; ++x) {  // (a bucket of one has nothing to merge)
        const int32_t i = hashed[x].second;
        if (q.nv[size_t(i)] == 0) continue;  // merged into an earlier one
        // mark i's list
        wflg += int64_t(n) + 2;
        const int64_t i0 = q.pe[size_t(i)];
        for (int32_t k = 0; k < q.len[size_t(i)]; ++k) q.w[size_t(q.iw[size_t(i0 + k)])] = -wflg;
        for (size_t y = x + 1; y < b; ++y) {
          const int32_t j = hashed[y].second;
          if (q.nv[size_t(j)] == 0 || q.len[size_t(j)] != q.len[size_t(i)] ||
              q.elen[size_t(j)] != q.elen[size_t(i)])
            continue;
          const int64_t j0 = q.pe[size_t(j)];
          bool same = true;
          for (int32_t k = 0; k < q.len[size_t(j)] && same; ++k)
            same = q.w[size_t(q.iw[size_t(j0 + k)])] == -wflg;
          if (!same) continue;
          q.nv[size_t(i)] += q.nv[size_t(j)];  // both negative (in L_p)
          q.nv[size_t(j)] = 0;
          q.kind[size_t(j)] = 2;
          q.merge_members(i, j);
        }
        // restore the element stamps the marks overwrote (variables' w is unused)
        for (int32_t k = 0; k < q.len[size_t(i)]; ++k) {
          const int32_t v = q.iw[size_t(i0 + k)];
          if (q.kind[size_t(v)] == 1) q.w[size_t(v)] = 1;
        }
      }
      a = b;
    }
    // --- finish: L_p's variables back in the degree lists -----------------
    int64_t out = q.pe[size_t(p)];
    const int64_t p0 = out;
    for (int32_t k = 0; k < q.len[size_t(p)]; ++k) {
      const int32_t i = q.iw[size_t(p0 + k)];
      if (q.nv[size_t(i)] >= 0) continue;  // merged or mass-eliminated
      q.nv[size_t(i)] = -q.nv[size_t(i)];
      const int32_t d = std::min(q.degree[size_t(i)], nleft - q.nv[size_t(i)]);
      q.list_insert(i, std::max(d, 0));
      mindeg = std::min(mindeg, q.degree[size_t(i)]);
      q.iw[size_t(out++)] = i;
    }
    q.len[size_t(p)] = int32_t(out - p0);
    q.nv[size_t(p)] = nvpiv;
    q.degree[size_t(p)] = int32_t(degme);
    for (int32_t j = q.mhead[size_t(p)]; j != kNone; j = q.mnext[size_t(j)]) order.push_back(j);
    if (q.len[size_t(p)] == 0) {  // no variable left next to it: the element is done
      q.kind[size_t(p)] = 2;
      q.w[size_t(p)] = 0;
    }
  }
  return int32_t(order.size()) == n;
}

}  // namespace acopf
