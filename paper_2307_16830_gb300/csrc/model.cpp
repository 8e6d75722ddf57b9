// Host symbolic phase of libacopf: validation, layout, pi-model coefficients,
// bus incidence lists, the COO patterns of the Jacobian and Hessian and the
// CSR pattern of the condensed KKT matrix.
//
// The paper analyses the sparsity of each computational pattern once and
// expands it over the pattern's data (Sec. III.C).  Here every pattern's
// entries are laid out by a closed rule, so the Jacobian and Hessian
// patterns are written directly in pattern order and the condensed matrix
// M_cond = W + Sigma_x + A'DA (Sec. IV.C) gets its lower-CSR pattern row by
// row from the network topology:
//   row va_i: va_j for each distinct neighbour j < i, then va_i;
//   row vm_i: va_j for each distinct neighbour j and for j = i (ascending;
//             va_i only if bus i has a branch), vm_j for each distinct
//             neighbour j < i, then vm_i;
//   row pg_g (bus i): vm_i, pg_h for the earlier generators h of bus i, pg_g;
//   row qg_g: the same with qg;
//   row p_a (arc a at bus i of branch f-t): va_lo, va_hi, vm_lo, vm_hi
//             (lo/hi = min/max of f, t), pg of every generator of bus i,
//             p_b for the earlier arcs b of bus i, p_a;
//   row q_a:  the four bus entries, qg of the generators of bus i, p_a,
//             q_b for the earlier arcs b of bus i, q_a.
// These are exactly the lower-triangle pairs that share a Jacobian row
// (flow rows couple an arc variable with its branch's four bus variables,
// thermal rows couple p_a with q_a, balance rows couple vm_i, the generators
// and the arcs of bus i) or a Hessian entry (the branch blocks and
// diagonals).  The kernels write each row in this same order.
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <sstream>

#include "acopf_internal.h"

namespace acopf {
namespace {

constexpr int64_t kMaxIndex = std::numeric_limits<int32_t>::max() - 1;

bool finite(double v) { return std::isfinite(v); }

template <typename T>
bool null_when_needed(int32_t n, const T* p) {
  return n > 0 && p == nullptr;
}

}  // namespace

acopf_status build_host_model(const acopf_buses* B, const acopf_branches* Lb, const acopf_gens* G,
                              HostModel& hm, std::string& err) {
  std::ostringstream msg;
  auto bad = [&](acopf_status s) {
    err = msg.str();
    return s;
  };
  if (!B || !Lb || !G) {
    msg << "null bus, branch or generator table";
    return bad(ACOPF_E_INVALID_ARG);
  }
  const int64_t nb = B->n, nl = Lb->n, ng = G->n;
  if (nb < 1 || nl < 0 || ng < 0) {
    msg << "need n_bus >= 1, n_branch >= 0, n_gen >= 0 (got " << nb << ", " << nl << ", " << ng
        << ")";
    return bad(ACOPF_E_INVALID_ARG);
  }
  if (null_when_needed(B->n, B->type) || null_when_needed(B->n, B->Pd) ||
      null_when_needed(B->n, B->Qd) || null_when_needed(B->n, B->Gs) ||
      null_when_needed(B->n, B->Bs) || null_when_needed(B->n, B->Vmin) ||
      null_when_needed(B->n, B->Vmax)) {
    msg << "a bus array is NULL";
    return bad(ACOPF_E_INVALID_ARG);
  }
  if (null_when_needed(Lb->n, Lb->f) || null_when_needed(Lb->n, Lb->t) ||
      null_when_needed(Lb->n, Lb->r) || null_when_needed(Lb->n, Lb->x) ||
      null_when_needed(Lb->n, Lb->b) || null_when_needed(Lb->n, Lb->tap) ||
      null_when_needed(Lb->n, Lb->shift) || null_when_needed(Lb->n, Lb->rate_a) ||
      null_when_needed(Lb->n, Lb->angmin) || null_when_needed(Lb->n, Lb->angmax)) {
    msg << "a branch array is NULL";
    return bad(ACOPF_E_INVALID_ARG);
  }
  if (null_when_needed(G->n, G->bus) || null_when_needed(G->n, G->Pmin) ||
      null_when_needed(G->n, G->Pmax) || null_when_needed(G->n, G->Qmin) ||
      null_when_needed(G->n, G->Qmax) || null_when_needed(G->n, G->c2) ||
      null_when_needed(G->n, G->c1) || null_when_needed(G->n, G->c0)) {
    msg << "a generator array is NULL";
    return bad(ACOPF_E_INVALID_ARG);
  }

  // ---- validation --------------------------------------------------------
  for (int64_t i = 0; i < nb; ++i) {
    if (!finite(B->Pd[i]) || !finite(B->Qd[i]) || !finite(B->Gs[i]) || !finite(B->Bs[i]) ||
        std::isnan(B->Vmin[i]) || std::isnan(B->Vmax[i])) {
      msg << "bus " << i << ": non-finite Pd/Qd/Gs/Bs or NaN voltage bound";
      return bad(ACOPF_E_BAD_MODEL);
    }
  }
  for (int64_t l = 0; l < nl; ++l) {
    const int32_t f = Lb->f[l], t = Lb->t[l];
    if (f < 0 || f >= nb || t < 0 || t >= nb) {
      msg << "branch " << l << ": bus index out of range (" << f << ", " << t << ")";
      return bad(ACOPF_E_BAD_MODEL);
    }
    if (f == t) {
      msg << "branch " << l << ": self-loop at bus " << f;
      return bad(ACOPF_E_BAD_MODEL);
    }
    const double r = Lb->r[l], x = Lb->x[l];
    if (!finite(r) || !finite(x) || !(r * r + x * x > 0.0)) {
      msg << "branch " << l << ": impedance r + jx must be finite and nonzero";
      return bad(ACOPF_E_BAD_MODEL);
    }
    if (!finite(Lb->b[l]) || !finite(Lb->tap[l]) || !finite(Lb->shift[l]) ||
        std::isnan(Lb->rate_a[l]) || std::isnan(Lb->angmin[l]) || std::isnan(Lb->angmax[l])) {
      msg << "branch " << l << ": non-finite b/tap/shift or NaN limit";
      return bad(ACOPF_E_BAD_MODEL);
    }
  }
  for (int64_t g = 0; g < ng; ++g) {
    if (G->bus[g] < 0 || G->bus[g] >= nb) {
      msg << "generator " << g << ": bus index " << G->bus[g] << " out of range";
      return bad(ACOPF_E_BAD_MODEL);
    }
    if (!finite(G->c2[g]) || !finite(G->c1[g]) || !finite(G->c0[g]) || std::isnan(G->Pmin[g]) ||
        std::isnan(G->Pmax[g]) || std::isnan(G->Qmin[g]) || std::isnan(G->Qmax[g])) {
      msg << "generator " << g << ": non-finite cost or NaN bound";
      return bad(ACOPF_E_BAD_MODEL);
    }
  }

  // ---- layout ------------------------------------------------------------
  Layout& L = hm.L;
  int64_t nref = 0;
  for (int64_t i = 0; i < nb; ++i) nref += (B->type[i] == 3);
  const int64_t n = 2 * nb + 2 * ng + 4 * nl;
  const int64_t m = nref + 7 * nl + 2 * nb;
  const int64_t nnzj = nref + 30 * nl + 2 * nb + 2 * ng;
  const int64_t nnzh = 14 * nl + ng + nb;
  if (n > kMaxIndex || m > kMaxIndex || nnzj > kMaxIndex || nnzh > kMaxIndex) {
    msg << "model too large for 32-bit indices";
    return bad(ACOPF_E_BAD_MODEL);
  }
  L.nb = int32_t(nb);
  L.nl = int32_t(nl);
  L.ng = int32_t(ng);
  L.nref = int32_t(nref);
  L.VA = 0;
  L.VM = L.nb;
  L.PG = 2 * L.nb;
  L.QG = L.PG + L.ng;
  L.P = L.QG + L.ng;
  L.Q = L.P + 2 * L.nl;
  L.n = int32_t(n);
  L.REF = 0;
  L.PF = L.nref;
  L.QF = L.PF + L.nl;
  L.PT = L.QF + L.nl;
  L.QT = L.PT + L.nl;
  L.ANG = L.QT + L.nl;
  L.SF = L.ANG + L.nl;
  L.ST = L.SF + L.nl;
  L.PB = L.ST + L.nl;
  L.QB = L.PB + L.nb;
  L.m = int32_t(m);
  L.JREF = 0;
  L.JPF = L.nref;
  L.JQF = L.JPF + 5 * L.nl;
  L.JPT = L.JQF + 5 * L.nl;
  L.JQT = L.JPT + 5 * L.nl;
  L.JANG = L.JQT + 5 * L.nl;
  L.JSF = L.JANG + 2 * L.nl;
  L.JST = L.JSF + 2 * L.nl;
  L.JPBV = L.JST + 2 * L.nl;
  L.JQBV = L.JPBV + L.nb;
  L.JPBG = L.JQBV + L.nb;
  L.JQBG = L.JPBG + L.ng;
  L.JPBA = L.JQBG + L.ng;
  L.JQBA = L.JPBA + 2 * L.nl;
  L.nnzj = int32_t(nnzj);
  L.HBLK = 0;
  L.HTH = 10 * L.nl;
  L.HG = L.HTH + 4 * L.nl;
  L.HB = L.HG + L.ng;
  L.nnzh = int32_t(nnzh);

  // ---- data copies and pi-model coefficients ------------------------------
  hm.f.assign(Lb->f, Lb->f + nl);
  hm.t.assign(Lb->t, Lb->t + nl);
  hm.gbus.assign(G->bus, G->bus + ng);
  hm.Pd.assign(B->Pd, B->Pd + nb);
  hm.Qd.assign(B->Qd, B->Qd + nb);
  hm.Gs.assign(B->Gs, B->Gs + nb);
  hm.Bs.assign(B->Bs, B->Bs + nb);
  hm.c2.assign(G->c2, G->c2 + ng);
  hm.c1.assign(G->c1, G->c1 + ng);
  hm.c0.assign(G->c0, G->c0 + ng);
  hm.coef.assign(size_t(NCOEF) * nl, 0.0);
  for (int64_t l = 0; l < nl; ++l) {
    // y = 1/(r + jx) = gs + j bs; T = tau e^{j shift}; Y_ff = (y + jb/2)/|T|^2,
    // Y_ft = -y/conj(T), Y_tf = -y/T, Y_tt = y + jb/2.
    const double r = Lb->r[l], x = Lb->x[l], b = Lb->b[l];
    const double tau = (Lb->tap[l] == 0.0) ? 1.0 : Lb->tap[l];
    const double z2 = r * r + x * x;
    const double gs = r / z2, bs = -x / z2;
    const double tr = tau * std::cos(Lb->shift[l]), ti = tau * std::sin(Lb->shift[l]);
    const double t2 = tr * tr + ti * ti;
    double* c = hm.coef.data();
    c[CG_FF * nl + l] = gs / t2;
    c[CB_FF * nl + l] = (bs + 0.5 * b) / t2;
    c[CG_FT * nl + l] = (-gs * tr + bs * ti) / t2;
    c[CB_FT * nl + l] = (-bs * tr - gs * ti) / t2;
    c[CG_TF * nl + l] = (-gs * tr - bs * ti) / t2;
    c[CB_TF * nl + l] = (-bs * tr + gs * ti) / t2;
    c[CG_TT * nl + l] = gs;
    c[CB_TT * nl + l] = bs + 0.5 * b;
  }

  // ---- reference rows ------------------------------------------------------
  hm.ref_row.assign(nb, -1);
  hm.ref_bus.clear();
  for (int64_t i = 0; i < nb; ++i) {
    if (B->type[i] == 3) {
      hm.ref_row[i] = int32_t(hm.ref_bus.size());
      hm.ref_bus.push_back(int32_t(i));
    }
  }

  // ---- bus incidence: arcs and generators per bus ---------------------------
  auto arc_bus = [&](int64_t a) { return a < nl ? hm.f[a] : hm.t[a - nl]; };
  auto arc_nbr = [&](int64_t a) { return a < nl ? hm.t[a] : hm.f[a - nl]; };
  hm.arc_ptr.assign(nb + 1, 0);
  for (int64_t a = 0; a < 2 * nl; ++a) hm.arc_ptr[arc_bus(a) + 1]++;
  for (int64_t i = 0; i < nb; ++i) hm.arc_ptr[i + 1] += hm.arc_ptr[i];
  hm.arcs_by_idx.assign(2 * nl, 0);
  {
    std::vector<int32_t> pos(hm.arc_ptr.begin(), hm.arc_ptr.end() - 1);
    for (int64_t a = 0; a < 2 * nl; ++a) hm.arcs_by_idx[pos[arc_bus(a)]++] = int32_t(a);
  }
  hm.arcs_by_nbr = hm.arcs_by_idx;
  for (int64_t i = 0; i < nb; ++i) {
    std::sort(hm.arcs_by_nbr.begin() + hm.arc_ptr[i], hm.arcs_by_nbr.begin() + hm.arc_ptr[i + 1],
              [&](int32_t a, int32_t b) {
                const int32_t ja = arc_nbr(a), jb = arc_nbr(b);
                return ja != jb ? ja < jb : a < b;
              });
  }
  hm.gen_ptr.assign(nb + 1, 0);
  for (int64_t g = 0; g < ng; ++g) hm.gen_ptr[hm.gbus[g] + 1]++;
  for (int64_t i = 0; i < nb; ++i) hm.gen_ptr[i + 1] += hm.gen_ptr[i];
  hm.gens_at.assign(ng, 0);
  {
    std::vector<int32_t> pos(hm.gen_ptr.begin(), hm.gen_ptr.end() - 1);
    for (int64_t g = 0; g < ng; ++g) hm.gens_at[pos[hm.gbus[g]]++] = int32_t(g);
  }

  // Bus-phase processing order (by arc count, then generator count, then
  // id), and in that order: the slots of each bus (its arcs by (other end,
  // arc id)) and its balance-row terms (generators, then arcs, ascending).
  hm.porder.resize(nb);
  std::iota(hm.porder.begin(), hm.porder.end(), 0);
  std::stable_sort(hm.porder.begin(), hm.porder.end(), [&](int32_t a, int32_t b) {
    const int32_t da = hm.arc_ptr[a + 1] - hm.arc_ptr[a], db = hm.arc_ptr[b + 1] - hm.arc_ptr[b];
    if (da != db) return da < db;
    return hm.gen_ptr[a + 1] - hm.gen_ptr[a] < hm.gen_ptr[b + 1] - hm.gen_ptr[b];
  });
  hm.pslot_ptr.assign(nb + 1, 0);
  hm.pbal_ptr.assign(nb + 1, 0);
  hm.slot_nbr.assign(2 * nl, 0);
  hm.slot_of_arc.assign(2 * nl, 0);
  hm.bal_idx.assign(ng + 2 * nl, 0);
  for (int64_t p = 0; p < nb; ++p) {
    const int32_t i = hm.porder[p];
    int32_t s = hm.pslot_ptr[p];
    for (int32_t k = hm.arc_ptr[i]; k < hm.arc_ptr[i + 1]; ++k, ++s) {
      hm.slot_nbr[s] = arc_nbr(hm.arcs_by_nbr[k]);
      hm.slot_of_arc[hm.arcs_by_nbr[k]] = s;
    }
    hm.pslot_ptr[p + 1] = s;
    int32_t b = hm.pbal_ptr[p];
    for (int32_t e = hm.gen_ptr[i]; e < hm.gen_ptr[i + 1]; ++e) hm.bal_idx[b++] = L.PG + hm.gens_at[e];
    for (int32_t e = hm.arc_ptr[i]; e < hm.arc_ptr[i + 1]; ++e) hm.bal_idx[b++] = L.P + hm.arcs_by_idx[e];
    hm.pbal_ptr[p + 1] = b;
  }

  // ---- Jacobian COO pattern --------------------------------------------------
  hm.jrows.resize(nnzj);
  hm.jcols.resize(nnzj);
  {
    int64_t k = 0;
    auto put = [&](int64_t r, int64_t c) {
      hm.jrows[k] = int32_t(r);
      hm.jcols[k] = int32_t(c);
      ++k;
    };
    for (int64_t r = 0; r < nref; ++r) put(L.REF + r, L.VA + hm.ref_bus[r]);
    const int64_t flow_row[4] = {L.PF, L.QF, L.PT, L.QT};
    const int64_t flow_var[4] = {L.P, L.Q, L.P + nl, L.Q + nl};
    // Branch patterns store entry k of every branch's row contiguously.
    for (int q = 0; q < 4; ++q) {
      for (int64_t l = 0; l < nl; ++l) put(flow_row[q] + l, flow_var[q] + l);
      for (int64_t l = 0; l < nl; ++l) put(flow_row[q] + l, L.VA + hm.f[l]);
      for (int64_t l = 0; l < nl; ++l) put(flow_row[q] + l, L.VA + hm.t[l]);
      for (int64_t l = 0; l < nl; ++l) put(flow_row[q] + l, L.VM + hm.f[l]);
      for (int64_t l = 0; l < nl; ++l) put(flow_row[q] + l, L.VM + hm.t[l]);
    }
    for (int64_t l = 0; l < nl; ++l) put(L.ANG + l, L.VA + hm.f[l]);
    for (int64_t l = 0; l < nl; ++l) put(L.ANG + l, L.VA + hm.t[l]);
    for (int64_t l = 0; l < nl; ++l) put(L.SF + l, L.P + l);
    for (int64_t l = 0; l < nl; ++l) put(L.SF + l, L.Q + l);
    for (int64_t l = 0; l < nl; ++l) put(L.ST + l, L.P + nl + l);
    for (int64_t l = 0; l < nl; ++l) put(L.ST + l, L.Q + nl + l);
    for (int64_t i = 0; i < nb; ++i) put(L.PB + i, L.VM + i);
    for (int64_t i = 0; i < nb; ++i) put(L.QB + i, L.VM + i);
    for (int64_t g = 0; g < ng; ++g) put(L.PB + hm.gbus[g], L.PG + g);
    for (int64_t g = 0; g < ng; ++g) put(L.QB + hm.gbus[g], L.QG + g);
    for (int64_t a = 0; a < 2 * nl; ++a) put(L.PB + arc_bus(a), L.P + a);
    for (int64_t a = 0; a < 2 * nl; ++a) put(L.QB + arc_bus(a), L.Q + a);
  }

  // ---- Hessian COO pattern (lower triangle, with duplicates) ----------------
  hm.hrows.resize(nnzh);
  hm.hcols.resize(nnzh);
  {
    static const int kPair[10][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1},
                                     {2, 2}, {3, 0}, {3, 1}, {3, 2}, {3, 3}};
    int64_t k = 0;
    // entry e of every branch's block stored contiguously
    for (int e = 0; e < 10; ++e) {
      for (int64_t l = 0; l < nl; ++l) {
        const int32_t loc[4] = {L.VA + hm.f[l], L.VA + hm.t[l], L.VM + hm.f[l], L.VM + hm.t[l]};
        const int32_t a = loc[kPair[e][0]], b = loc[kPair[e][1]];
        hm.hrows[k] = std::max(a, b);
        hm.hcols[k] = std::min(a, b);
        ++k;
      }
    }
    for (int e = 0; e < 4; ++e) {
      for (int64_t l = 0; l < nl; ++l) {
        const int32_t d[4] = {int32_t(L.P + l), int32_t(L.Q + l), int32_t(L.P + nl + l),
                              int32_t(L.Q + nl + l)};
        hm.hrows[k] = d[e];
        hm.hcols[k] = d[e];
        ++k;
      }
    }
    for (int64_t g = 0; g < ng; ++g, ++k) hm.hrows[k] = hm.hcols[k] = int32_t(L.PG + g);
    for (int64_t i = 0; i < nb; ++i, ++k) hm.hrows[k] = hm.hcols[k] = int32_t(L.VM + i);
  }

  // ---- condensed KKT lower-CSR pattern, row by row ---------------------------
  // distinct neighbours of each bus, ascending (from the neighbour-sorted arcs)
  std::vector<int32_t> nu(nb, 0), nlo(nb, 0);
  std::vector<int32_t> nbr_ptr(nb + 1, 0), nbrs;
  nbrs.reserve(2 * nl);
  for (int64_t i = 0; i < nb; ++i) {
    int32_t prev = -1;
    for (int32_t k = hm.arc_ptr[i]; k < hm.arc_ptr[i + 1]; ++k) {
      const int32_t j = arc_nbr(hm.arcs_by_nbr[k]);
      if (j != prev) {
        nbrs.push_back(j);
        nu[i]++;
        if (j < i) nlo[i]++;
        prev = j;
      }
    }
    nbr_ptr[i + 1] = int32_t(nbrs.size());
  }
  std::vector<int64_t> len(n, 0);
  for (int64_t i = 0; i < nb; ++i) {
    len[L.VA + i] = nlo[i] + 1;
    // (vm_i, va_i) exists only when bus i has a branch
    len[L.VM + i] = (nu[i] > 0 ? nu[i] + 1 : 0) + nlo[i] + 1;
  }
  for (int64_t i = 0; i < nb; ++i) {
    for (int32_t k = hm.gen_ptr[i]; k < hm.gen_ptr[i + 1]; ++k) {
      const int32_t g = hm.gens_at[k];
      const int64_t rank = k - hm.gen_ptr[i];
      len[L.PG + g] = 1 + rank + 1;
      len[L.QG + g] = 1 + rank + 1;
    }
    const int64_t ngi = hm.gen_ptr[i + 1] - hm.gen_ptr[i];
    for (int32_t k = hm.arc_ptr[i]; k < hm.arc_ptr[i + 1]; ++k) {
      const int32_t a = hm.arcs_by_idx[k];
      const int64_t rank = k - hm.arc_ptr[i];
      len[L.P + a] = 4 + ngi + rank + 1;
      len[L.Q + a] = 4 + ngi + 1 + rank + 1;
    }
  }
  int64_t nnzk = 0;
  for (int64_t r = 0; r < n; ++r) nnzk += len[r];
  if (nnzk > kMaxIndex) {
    msg << "condensed KKT matrix too large for 32-bit indices";
    return bad(ACOPF_E_BAD_MODEL);
  }
  L.nnzk = int32_t(nnzk);
  hm.krowptr.assign(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) hm.krowptr[r + 1] = int32_t(hm.krowptr[r] + len[r]);
  hm.kcolind.assign(nnzk, 0);
  {
    int32_t* ci = hm.kcolind.data();
    for (int64_t i = 0; i < nb; ++i) {
      int32_t* va = ci + hm.krowptr[L.VA + i];
      int32_t* vm = ci + hm.krowptr[L.VM + i];
      bool self = false;
      for (int32_t k = nbr_ptr[i]; k < nbr_ptr[i + 1]; ++k) {
        const int32_t j = nbrs[k];
        if (j < i) *va++ = L.VA + j;
        if (!self && j > i) {
          *vm++ = int32_t(L.VA + i);
          self = true;
        }
        *vm++ = L.VA + j;
      }
      if (!self && nu[i] > 0) *vm++ = int32_t(L.VA + i);
      for (int32_t k = nbr_ptr[i]; k < nbr_ptr[i + 1]; ++k)
        if (nbrs[k] < i) *vm++ = L.VM + nbrs[k];
      *va = int32_t(L.VA + i);
      *vm = int32_t(L.VM + i);
    }
    for (int64_t i = 0; i < nb; ++i) {
      for (int32_t k = hm.gen_ptr[i]; k < hm.gen_ptr[i + 1]; ++k) {
        const int32_t g = hm.gens_at[k];
        int32_t* rp = ci + hm.krowptr[L.PG + g];
        int32_t* rq = ci + hm.krowptr[L.QG + g];
        *rp++ = int32_t(L.VM + i);
        *rq++ = int32_t(L.VM + i);
        for (int32_t h = hm.gen_ptr[i]; h < k; ++h) {
          *rp++ = L.PG + hm.gens_at[h];
          *rq++ = L.QG + hm.gens_at[h];
        }
        *rp = L.PG + g;
        *rq = L.QG + g;
      }
    }
    for (int64_t a = 0; a < 2 * nl; ++a) {
      const int32_t i = arc_bus(a);
      const int64_t l = a < nl ? a : a - nl;
      const int32_t lo = std::min(hm.f[l], hm.t[l]), hi = std::max(hm.f[l], hm.t[l]);
      int32_t* rp = ci + hm.krowptr[L.P + a];
      int32_t* rq = ci + hm.krowptr[L.Q + a];
      const int32_t four[4] = {L.VA + lo, L.VA + hi, L.VM + lo, L.VM + hi};
      for (int e = 0; e < 4; ++e) *rp++ = *rq++ = four[e];
      for (int32_t k = hm.gen_ptr[i]; k < hm.gen_ptr[i + 1]; ++k) {
        *rp++ = L.PG + hm.gens_at[k];
        *rq++ = L.QG + hm.gens_at[k];
      }
      *rq++ = int32_t(L.P + a);
      for (int32_t k = hm.arc_ptr[i]; k < hm.arc_ptr[i + 1]; ++k) {
        const int32_t b = hm.arcs_by_idx[k];
        if (b >= a) break;
        *rp++ = int32_t(L.P + b);
        *rq++ = int32_t(L.Q + b);
      }
      *rp = int32_t(L.P + a);
      *rq = int32_t(L.Q + a);
    }
  }

  // per-branch arc-row descriptors
  hm.brow.assign(4 * nl, 0);
  hm.bcnt.assign(nl, 0);
  {
    std::vector<int32_t> rank(2 * nl, 0);
    for (int64_t i = 0; i < nb; ++i)
      for (int32_t k = hm.arc_ptr[i]; k < hm.arc_ptr[i + 1]; ++k)
        rank[hm.arcs_by_idx[k]] = k - hm.arc_ptr[i];
    for (int64_t l = 0; l < nl; ++l) {
      hm.brow[4 * l + 0] = hm.krowptr[L.P + l];
      hm.brow[4 * l + 1] = hm.krowptr[L.Q + l];
      hm.brow[4 * l + 2] = hm.krowptr[L.P + nl + l];
      hm.brow[4 * l + 3] = hm.krowptr[L.Q + nl + l];
      const int64_t ngf = hm.gen_ptr[hm.f[l] + 1] - hm.gen_ptr[hm.f[l]];
      const int64_t ngt = hm.gen_ptr[hm.t[l] + 1] - hm.gen_ptr[hm.t[l]];
      const int64_t rf = rank[l], rt = rank[nl + l];
      hm.bcnt[l] = (ngf > 255 || ngt > 255 || rf > 255 || rt > 255)
                       ? kCountsWide
                       : uint32_t(ngf | (rf << 8) | (ngt << 16) | (rt << 24));
    }
  }

  // ---- bus-row chunks ---------------------------------------------------------
  // The bus rows' gather (phase 2) in pieces of about kRowChunk slots, one
  // lane each, so that a bus with many branches takes one round of loads on
  // several lanes instead of many rounds on one.  A chunk starts at a run of
  // equal neighbours (parallel branches are summed inside one chunk) and
  // records where its entries start in the bus's rows: the positions the
  // whole-bus walk (one entry per distinct neighbour, va_i's own column
  // skipped in row vm_i) has reached there.  Buses in processing order; a
  // bus's chunks never straddle a warp (the rest of the warp idles).
  {
    std::vector<int32_t>& rc = hm.rchunk;
    rc.clear();
    int32_t lane = 0;
    auto idle = [&]() {
      rc.insert(rc.end(), {-1, 0, 0, 0, 0, 0, 0, 0});
      lane = (lane + 1) & 31;
    };
    struct Chunk {
      int32_t ka, kb, pva, pvmva, pvmvm;
    };
    std::vector<Chunk> ch;
    for (int64_t p = 0; p < nb; ++p) {
      const int32_t i = hm.porder[p], k0 = hm.pslot_ptr[p], k1 = hm.pslot_ptr[p + 1];
      const int32_t bva = hm.krowptr[L.VA + i], eva = hm.krowptr[L.VA + i + 1];
      const int32_t bvm = hm.krowptr[L.VM + i], evm = hm.krowptr[L.VM + i + 1];
      const int32_t nlo = eva - bva - 1, nu = evm - bvm - nlo - 2;
      for (int32_t cap = kRowChunk;; cap *= 2) {
        ch.clear();
        int32_t pva = bva, pvmva = bvm, pvmvm = bvm + nu + 1;
        Chunk cur{k0, k0, pva, pvmva, pvmvm};
        for (int32_t k = k0; k < k1;) {
          const int32_t j = hm.slot_nbr[k];
          int32_t r = k;
          while (r < k1 && hm.slot_nbr[r] == j) ++r;
          if (k > cur.ka && (k - cur.ka) + (r - k) > cap) {
            cur.kb = k;
            ch.push_back(cur);
            cur = Chunk{k, k, pva, pvmva, pvmvm};
          }
          if (j > i && pvmva == bvm + nlo) ++pvmva;
          ++pvmva;
          if (j < i) {
            ++pva;
            ++pvmvm;
          }
          k = r;
        }
        cur.kb = k1;
        ch.push_back(cur);
        if (ch.size() <= 32) break;
      }
      const int32_t nch = int32_t(ch.size());
      if (lane + nch > 32)
        while (lane != 0) idle();
      const int32_t first = lane;
      for (const Chunk& c : ch) {
        rc.insert(rc.end(), {i, int32_t(p), c.ka, c.kb, c.pva, c.pvmva, c.pvmvm, first | (nch << 5)});
        lane = (lane + 1) & 31;
      }
    }
    while (lane != 0) idle();
    L.nrc = int32_t(rc.size() / 8);
  }

  // ---- bounds -----------------------------------------------------------------
  const double inf = std::numeric_limits<double>::infinity();
  hm.xl.assign(n, 0.0);
  hm.xu.assign(n, 0.0);
  hm.gl.assign(m, 0.0);
  hm.gu.assign(m, 0.0);
  for (int64_t i = 0; i < nb; ++i) {
    hm.xl[L.VA + i] = -inf;
    hm.xu[L.VA + i] = inf;
    hm.xl[L.VM + i] = B->Vmin[i];
    hm.xu[L.VM + i] = B->Vmax[i];
  }
  for (int64_t g = 0; g < ng; ++g) {
    hm.xl[L.PG + g] = G->Pmin[g];
    hm.xu[L.PG + g] = G->Pmax[g];
    hm.xl[L.QG + g] = G->Qmin[g];
    hm.xu[L.QG + g] = G->Qmax[g];
  }
  for (int64_t l = 0; l < nl; ++l) {
    const double rate = Lb->rate_a[l] > 0.0 ? Lb->rate_a[l] : inf;
    for (int64_t off : {int64_t(L.P) + l, int64_t(L.P) + nl + l, int64_t(L.Q) + l,
                        int64_t(L.Q) + nl + l}) {
      hm.xl[off] = -rate;
      hm.xu[off] = rate;
    }
    hm.gl[L.ANG + l] = Lb->angmin[l];
    hm.gu[L.ANG + l] = Lb->angmax[l];
    hm.gl[L.SF + l] = -inf;
    hm.gl[L.ST + l] = -inf;
    hm.gu[L.SF + l] = rate * rate;
    hm.gu[L.ST + l] = rate * rate;
  }
  return ACOPF_OK;
}

}  // namespace acopf
