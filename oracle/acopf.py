"""Plain CPU FP64 oracle: ACOPF NLP callbacks and the condensed KKT matrix.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the library
imports this module, and this module imports nothing from the library.

What it computes, and where the paper defines it:

* the NLP ``min f(x) s.t. g(x) = 0, x_lo <= x <= x_hi`` (Sec. II.A) for the
  AC optimal power flow model the paper builds from 15 computational patterns
  (Sec. III.B): generation cost (1), reference angle (2), active/reactive
  branch flows from/to (3-6), angle-difference limits (7), apparent-power
  limits from/to (8-9), bus power balance base terms (10-11), generator
  contributions (12-13) and arc-flow contributions (14-15).  The paper names
  the patterns but does not print the equations; they are the polar
  branch-flow form of the rosetta-opf / PowerModels model that Sec. V.A says
  the experiments use, with the textbook pi-model of a line with an
  off-nominal complex tap.
* the callbacks of Algorithm 1: objective, gradient, constraints, the sparse
  Jacobian A = dg/dx, and the Lagrangian Hessian W = sigma d2f + sum_r y_r d2g_r
  (Sec. II.A; the library's sign convention adds y_r g_r, so the paper's
  L = f - y'g corresponds to passing -y);
* the condensed KKT matrix of Sec. IV.C,
  M_cond = W + delta_w I + Sigma_x + A' D A, with
  C = (delta_c Sigma_s + (1 + delta_c delta_w) I)^-1 and D = (Sigma_s + delta_w I) C.

Every value comes with a magnitude ``M`` = the sum of the absolute values of
the terms that make it up (a trigonometric term u cos(th) counts |u cos(th)|).  Parity tests accept a
GPU value v when |v - oracle| <= 1e-12 M + 1e-14, which is the stated
"1e-12 relative, 1e-14 absolute floor" made well posed when Sigma spans 16
orders of magnitude and terms cancel.

Everything is vectorised with numpy over pattern instances, in the order the
patterns are listed above, with no fusion or reordering beyond that; sparse
matrix products come from scipy.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

REF_BUS_TYPE = 3
TOL_REL = 1e-12
TOL_ABS = 1e-14

__all__ = [
    "Layout", "layout", "branch_admittance", "bounds", "jac_structure",
    "hess_structure", "kkt_structure", "objective", "gradient", "constraints",
    "jacobian", "hessian", "condensation_diag", "condensed_kkt",
    "eval_assemble", "within_tol", "TOL_REL", "TOL_ABS",
]


# ---------------------------------------------------------------------------
# Layout: variables and constraints in pattern order (Sec. III.B).
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Layout:
    nb: int
    nl: int
    ng: int
    ref_buses: np.ndarray
    # variable offsets
    VA: int
    VM: int
    PG: int
    QG: int
    P: int
    Q: int
    n: int
    # constraint offsets
    REF: int
    PF: int
    QF: int
    PT: int
    QT: int
    ANG: int
    SF: int
    ST: int
    PB: int
    QB: int
    m: int


def layout(grid) -> Layout:
    """x = [va, vm, pg, qg, p(arcs), q(arcs)];
    g = [ref, pf, qf, pt, qt, ang, sf, st, Pbal, Qbal].

    Arc a < nl is the from end of branch a (at bus f[a]); arc nl + l is the to
    end of branch l (at bus t[l]).
    """
    nb, nl, ng = grid.n_bus, grid.n_branch, grid.n_gen
    ref_buses = np.flatnonzero(np.asarray(grid.bus_type) == REF_BUS_TYPE)
    VA, VM, PG = 0, nb, 2 * nb
    QG = PG + ng
    P = QG + ng
    Q = P + 2 * nl
    n = Q + 2 * nl
    REF = 0
    PF = REF + ref_buses.size
    QF, PT, QT, ANG, SF, ST = (PF + k * nl for k in range(1, 7))
    PB = ST + nl
    QB = PB + nb
    m = QB + nb
    return Layout(nb, nl, ng, ref_buses, VA, VM, PG, QG, P, Q, n,
                  REF, PF, QF, PT, QT, ANG, SF, ST, PB, QB, m)


def _arc_bus(grid) -> np.ndarray:
    return np.concatenate([np.asarray(grid.f), np.asarray(grid.t)]).astype(np.int64)


# ---------------------------------------------------------------------------
# Branch pi-model (patterns 3-6).
# ---------------------------------------------------------------------------
def branch_admittance(grid):
    """Real and imaginary parts of the four branch admittances.

    Series admittance y = 1/(r + jx) = gs + j bs; charging b split half per
    end; complex tap T = tau e^{j shift} on the from side (tau = 0 read as 1):
    Y_ff = (y + jb/2)/|T|^2, Y_ft = -y/conj(T), Y_tf = -y/T, Y_tt = y + jb/2.
    Returns (g_ff, b_ff, g_ft, b_ft, g_tf, b_tf, g_tt, b_tt).
    """
    r = np.asarray(grid.r, dtype=np.float64)
    xx = np.asarray(grid.x, dtype=np.float64)
    b = np.asarray(grid.b, dtype=np.float64)
    tau = np.where(np.asarray(grid.tap) == 0.0, 1.0, np.asarray(grid.tap, dtype=np.float64))
    phi = np.asarray(grid.shift, dtype=np.float64)
    z2 = r * r + xx * xx
    gs = r / z2
    bs = -xx / z2
    tr = tau * np.cos(phi)
    ti = tau * np.sin(phi)
    t2 = tr * tr + ti * ti
    g_ff = gs / t2
    b_ff = (bs + 0.5 * b) / t2
    g_ft = (-gs * tr + bs * ti) / t2
    b_ft = (-bs * tr - gs * ti) / t2
    g_tf = (-gs * tr - bs * ti) / t2
    b_tf = (-bs * tr + gs * ti) / t2
    g_tt = gs
    b_tt = bs + 0.5 * b
    return g_ff, b_ff, g_ft, b_ft, g_tf, b_tf, g_tt, b_tt


def _flow_forms(grid):
    """Each flow F written as  a vm_f^2 + d vm_t^2 + vm_f vm_t (u cos th + w sin th)
    with th = va_f - va_t.  Returns, per flow P_f, Q_f, P_t, Q_t, the tuple
    (a, d, u, w) of per-branch arrays."""
    g_ff, b_ff, g_ft, b_ft, g_tf, b_tf, g_tt, b_tt = branch_admittance(grid)
    z = np.zeros_like(g_ff)
    # P_f = g_ff vm_f^2 + V (g_ft c + b_ft s)
    # Q_f = -b_ff vm_f^2 + V (g_ft s - b_ft c)
    # P_t = g_tt vm_t^2 + V (g_tf c - b_tf s)
    # Q_t = -b_tt vm_t^2 + V (-g_tf s - b_tf c)
    return [
        (g_ff, z, g_ft, b_ft),
        (-b_ff, z, -b_ft, g_ft),
        (z, g_tt, g_tf, -b_tf),
        (z, -b_tt, -b_tf, -g_tf),
    ]


def _branch_state(grid, x, L):
    f = np.asarray(grid.f, dtype=np.int64)
    t = np.asarray(grid.t, dtype=np.int64)
    va_f, va_t = x[L.VA + f], x[L.VA + t]
    vm_f, vm_t = x[L.VM + f], x[L.VM + t]
    th = va_f - va_t
    return f, t, va_f, va_t, vm_f, vm_t, np.cos(th), np.sin(th)


def _flow_value_and_derivs(form, vm_f, vm_t, c, s):
    """Value, first and second derivatives of one flow, with magnitudes.

    With T(th) = u cos th + w sin th, T' = -u sin th + w cos th, T'' = -T:
      F        = a vm_f^2 + d vm_t^2 + V T              (V = vm_f vm_t)
      dF/dth   = V T'          dF/dvm_f = 2 a vm_f + vm_t T
                               dF/dvm_t = 2 d vm_t + vm_f T
      d2F/dth2 = -V T          d2F/dth dvm_f = vm_t T'   d2F/dth dvm_t = vm_f T'
      d2F/dvm_f2 = 2a          d2F/dvm_f dvm_t = T       d2F/dvm_t2 = 2d
    and d/dva_f = d/dth, d/dva_t = -d/dth.
    """
    a, d, u, w = form
    V = vm_f * vm_t
    T = u * c + w * s
    T1 = -u * s + w * c
    TM = np.abs(u * c) + np.abs(w * s)         # sum of |terms| of T
    T1M = np.abs(u * s) + np.abs(w * c)        # sum of |terms| of T'
    out = {
        "F": (a * vm_f ** 2 + d * vm_t ** 2 + V * T,
              np.abs(a) * vm_f ** 2 + np.abs(d) * vm_t ** 2 + V * TM),
        "th": (V * T1, V * T1M),
        "vmf": (2 * a * vm_f + vm_t * T, 2 * np.abs(a) * vm_f + vm_t * TM),
        "vmt": (2 * d * vm_t + vm_f * T, 2 * np.abs(d) * vm_t + vm_f * TM),
        "thth": (-V * T, V * TM),
        "thvmf": (vm_t * T1, vm_t * T1M),
        "thvmt": (vm_f * T1, vm_f * T1M),
        "vmfvmf": (2 * a, 2 * np.abs(a)),
        "vmfvmt": (T, TM),
        "vmtvmt": (2 * d, 2 * np.abs(d)),
    }
    return out


# ---------------------------------------------------------------------------
# Bounds.
# ---------------------------------------------------------------------------
def bounds(grid):
    """(x_lo, x_hi, g_lo, g_hi).  va free; vm, pg, qg boxed by the data; arc
    flows within +-rate_a and thermal rows at most rate_a^2 (unbounded when
    rate_a <= 0); angle rows within [angmin, angmax]; all other rows = 0."""
    L = layout(grid)
    inf = np.inf
    rate = np.asarray(grid.rate_a, dtype=np.float64)
    rb = np.where(rate > 0, rate, inf)
    xl = np.concatenate([np.full(L.nb, -inf), grid.Vmin, grid.Pmin, grid.Qmin,
                         -rb, -rb, -rb, -rb])
    xu = np.concatenate([np.full(L.nb, inf), grid.Vmax, grid.Pmax, grid.Qmax,
                         rb, rb, rb, rb])
    gl = np.zeros(L.m)
    gu = np.zeros(L.m)
    gl[L.ANG:L.ANG + L.nl] = grid.angmin
    gu[L.ANG:L.ANG + L.nl] = grid.angmax
    gl[L.SF:L.ST + L.nl] = -inf
    gu[L.SF:L.SF + L.nl] = rb * rb
    gu[L.ST:L.ST + L.nl] = rb * rb
    return xl.astype(np.float64), xu.astype(np.float64), gl, gu


# ---------------------------------------------------------------------------
# Sparsity structure (Sec. III.C: one pattern per instruction, expanded over
# its data).
# ---------------------------------------------------------------------------
def jac_structure(grid):
    """(rows, cols) of the Jacobian in COO order, int32.

    Order: ref rows; pf rows with entries [p_l, va_f, va_t, vm_f, vm_t]; qf
    [q_l, ...]; pt [p_{nl+l}, ...]; qt [q_{nl+l}, ...]; ang [va_f, va_t];
    sf [p_l, q_l]; st [p_{nl+l}, q_{nl+l}]; balance vm terms (P then Q, per
    bus); generator terms (P then Q, per generator); arc terms (P then Q, per
    arc).  Within each branch pattern the entries are stored entry-major:
    entry k of every branch, then entry k + 1 (the pattern's parameterised
    sparsity expanded over its data, Sec. III.C)."""
    L = layout(grid)
    nl = L.nl
    f = np.asarray(grid.f, dtype=np.int64)
    t = np.asarray(grid.t, dtype=np.int64)
    br = np.arange(nl)
    bus_cols = np.stack([L.VA + f, L.VA + t, L.VM + f, L.VM + t], axis=1)
    rows, cols = [], []
    rows.append(L.REF + np.arange(L.ref_buses.size))
    cols.append(L.VA + L.ref_buses)
    for base, var in ((L.PF, L.P + br), (L.QF, L.Q + br),
                      (L.PT, L.P + nl + br), (L.QT, L.Q + nl + br)):
        rows.append(np.tile(base + br, 5))
        cols.append(np.concatenate([var[:, None], bus_cols], axis=1).T.ravel())
    rows.append(np.tile(L.ANG + br, 2))
    cols.append(np.concatenate([L.VA + f, L.VA + t]))
    rows.append(np.tile(L.SF + br, 2))
    cols.append(np.concatenate([L.P + br, L.Q + br]))
    rows.append(np.tile(L.ST + br, 2))
    cols.append(np.concatenate([L.P + nl + br, L.Q + nl + br]))
    buses = np.arange(L.nb)
    rows += [L.PB + buses, L.QB + buses]
    cols += [L.VM + buses, L.VM + buses]
    gbus = np.asarray(grid.gen_bus, dtype=np.int64)
    gens = np.arange(L.ng)
    rows += [L.PB + gbus, L.QB + gbus]
    cols += [L.PG + gens, L.QG + gens]
    abus = _arc_bus(grid)
    arcs = np.arange(2 * nl)
    rows += [L.PB + abus, L.QB + abus]
    cols += [L.P + arcs, L.Q + arcs]
    return (np.concatenate(rows).astype(np.int32),
            np.concatenate(cols).astype(np.int32))


_HPAIRS = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (3, 3)]
"""Local order of the 10 lower-triangle entries of a branch's block over
(va_f, va_t, vm_f, vm_t) = local indices (0, 1, 2, 3)."""


def hess_structure(grid):
    """(rows, cols) of the lower-triangle Lagrangian Hessian in COO order.

    The 10 entries of each branch's (va_f, va_t, vm_f, vm_t) block in the
    local order (va_f,va_f) (va_t,va_f) (va_t,va_t) (vm_f,va_f) (vm_f,va_t)
    (vm_f,vm_f) (vm_t,va_f) (vm_t,va_t) (vm_t,vm_f) (vm_t,vm_t), each stored as
    (max, min) of the global indices, entry-major (entry e of every branch,
    then entry e + 1); then the diagonals of p_l, q_l, p_{nl+l}, q_{nl+l},
    entry-major; then (pg_g, pg_g) per generator; then (vm_i, vm_i) per bus.
    Entries with equal (row, col) are kept separately (COO with duplicates)."""
    L = layout(grid)
    nl = L.nl
    f = np.asarray(grid.f, dtype=np.int64)
    t = np.asarray(grid.t, dtype=np.int64)
    loc = np.stack([L.VA + f, L.VA + t, L.VM + f, L.VM + t], axis=1)
    ri = np.stack([loc[:, i] for i, _ in _HPAIRS], axis=1)
    ci = np.stack([loc[:, j] for _, j in _HPAIRS], axis=1)
    r_blk = np.maximum(ri, ci).T.ravel()
    c_blk = np.minimum(ri, ci).T.ravel()
    br = np.arange(nl)
    th = np.concatenate([L.P + br, L.Q + br, L.P + nl + br, L.Q + nl + br])
    gens = L.PG + np.arange(L.ng)
    buses = L.VM + np.arange(L.nb)
    rows = np.concatenate([r_blk, th, gens, buses])
    cols = np.concatenate([c_blk, th, gens, buses])
    return rows.astype(np.int32), cols.astype(np.int32)


def _jac_matrix(grid, vals):
    L = layout(grid)
    r, c = jac_structure(grid)
    return sp.csr_matrix((vals, (r, c)), shape=(L.m, L.n))


def _hess_lower_matrix(grid, vals):
    L = layout(grid)
    r, c = hess_structure(grid)
    return sp.csr_matrix((vals, (r, c)), shape=(L.n, L.n))


def kkt_structure(grid):
    """(rowptr, colind) of the lower triangle of M_cond in CSR, int32.

    The pattern is the structural union of the Hessian, the diagonal and
    A'A (every pair of entries of every Jacobian row), independent of the
    values: it is taken from matrices of structural ones, so no cancellation
    can drop an entry.  Columns ascend within each row."""
    L = layout(grid)
    jr, jc = jac_structure(grid)
    hr, hc = hess_structure(grid)
    Jo = sp.csr_matrix((np.ones(jr.size), (jr, jc)), shape=(L.m, L.n))
    Ho = sp.csr_matrix((np.ones(hr.size), (hr, hc)), shape=(L.n, L.n))
    S = (Jo.T @ Jo) + Ho + Ho.T + sp.identity(L.n, format="csr")
    S = sp.tril(S, format="csr")
    S.sum_duplicates()
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32)


# ---------------------------------------------------------------------------
# Objective and gradient (pattern 1).
# ---------------------------------------------------------------------------
def objective(grid, x):
    """f = sum_g c2 pg^2 + c1 pg + c0.  Returns (f, M)."""
    L = layout(grid)
    pg = x[L.PG:L.PG + L.ng]
    c2, c1, c0 = (np.asarray(v, dtype=np.float64) for v in (grid.c2, grid.c1, grid.c0))
    terms = c2 * pg * pg + c1 * pg + c0
    mag = np.abs(c2) * pg * pg + np.abs(c1 * pg) + np.abs(c0)
    return float(np.sum(terms)), float(np.sum(mag))


def gradient(grid, x):
    """df/dx: 2 c2 pg + c1 on the pg entries, 0 elsewhere.  Returns (grad, M)."""
    L = layout(grid)
    pg = x[L.PG:L.PG + L.ng]
    c2, c1 = np.asarray(grid.c2, dtype=np.float64), np.asarray(grid.c1, dtype=np.float64)
    g = np.zeros(L.n)
    mag = np.zeros(L.n)
    g[L.PG:L.PG + L.ng] = 2.0 * c2 * pg + c1
    mag[L.PG:L.PG + L.ng] = 2.0 * np.abs(c2 * pg) + np.abs(c1)
    return g, mag


# ---------------------------------------------------------------------------
# Constraints (patterns 2-15).
# ---------------------------------------------------------------------------
def constraints(grid, x):
    """g(x) in constraint order.  Returns (g, M).

    ref:  va_i                                   (pattern 2)
    pf:   p_l - P_f,  qf: q_l - Q_f,  pt: p_{nl+l} - P_t,  qt: q_{nl+l} - Q_t   (3-6)
    ang:  va_f - va_t                            (7)
    sf:   p_l^2 + q_l^2,  st: p_{nl+l}^2 + q_{nl+l}^2                         (8-9)
    Pbal: Pd + Gs vm^2 - sum_{g at i} pg + sum_{arcs at i} p_a               (10, 12, 14)
    Qbal: Qd - Bs vm^2 - sum_{g at i} qg + sum_{arcs at i} q_a               (11, 13, 15)
    """
    L = layout(grid)
    nl = L.nl
    g = np.zeros(L.m)
    M = np.zeros(L.m)
    va = x[L.VA:L.VA + L.nb]
    g[L.REF:L.PF] = va[L.ref_buses]
    M[L.REF:L.PF] = np.abs(va[L.ref_buses])
    f, t, va_f, va_t, vm_f, vm_t, c, s = _branch_state(grid, x, L)
    p = x[L.P:L.P + 2 * nl]
    q = x[L.Q:L.Q + 2 * nl]
    flowvars = [p[:nl], q[:nl], p[nl:], q[nl:]]
    for k, (base, form) in enumerate(zip((L.PF, L.QF, L.PT, L.QT), _flow_forms(grid))):
        F, FM = _flow_value_and_derivs(form, vm_f, vm_t, c, s)["F"]
        g[base:base + nl] = flowvars[k] - F
        M[base:base + nl] = np.abs(flowvars[k]) + FM
    g[L.ANG:L.ANG + nl] = va_f - va_t
    M[L.ANG:L.ANG + nl] = np.abs(va_f) + np.abs(va_t)
    g[L.SF:L.SF + nl] = p[:nl] ** 2 + q[:nl] ** 2
    M[L.SF:L.SF + nl] = g[L.SF:L.SF + nl]
    g[L.ST:L.ST + nl] = p[nl:] ** 2 + q[nl:] ** 2
    M[L.ST:L.ST + nl] = g[L.ST:L.ST + nl]
    # Balance rows: base terms, then generator and arc contributions added
    # per bus (patterns 3 of Sec. II.C, here summed bus by bus).
    vm = x[L.VM:L.VM + L.nb]
    Pd, Qd = np.asarray(grid.Pd, np.float64), np.asarray(grid.Qd, np.float64)
    Gs, Bs = np.asarray(grid.Gs, np.float64), np.asarray(grid.Bs, np.float64)
    Pb = Pd + Gs * vm * vm
    Qb = Qd - Bs * vm * vm
    PbM = np.abs(Pd) + np.abs(Gs) * vm * vm
    QbM = np.abs(Qd) + np.abs(Bs) * vm * vm
    gbus = np.asarray(grid.gen_bus, dtype=np.int64)
    pg = x[L.PG:L.PG + L.ng]
    qg = x[L.QG:L.QG + L.ng]
    abus = _arc_bus(grid)
    Pb = Pb - np.bincount(gbus, weights=pg, minlength=L.nb) \
        + np.bincount(abus, weights=p, minlength=L.nb)
    Qb = Qb - np.bincount(gbus, weights=qg, minlength=L.nb) \
        + np.bincount(abus, weights=q, minlength=L.nb)
    PbM = PbM + np.bincount(gbus, weights=np.abs(pg), minlength=L.nb) \
        + np.bincount(abus, weights=np.abs(p), minlength=L.nb)
    QbM = QbM + np.bincount(gbus, weights=np.abs(qg), minlength=L.nb) \
        + np.bincount(abus, weights=np.abs(q), minlength=L.nb)
    g[L.PB:L.PB + L.nb] = Pb
    g[L.QB:L.QB + L.nb] = Qb
    M[L.PB:L.PB + L.nb] = PbM
    M[L.QB:L.QB + L.nb] = QbM
    return g, M


# ---------------------------------------------------------------------------
# Jacobian A = dg/dx (values in jac_structure order).
# ---------------------------------------------------------------------------
def jacobian(grid, x):
    """Jacobian values in COO order.  Returns (vals, M)."""
    L = layout(grid)
    nl = L.nl
    vals, mags = [], []
    one_ref = np.ones(L.ref_buses.size)
    vals.append(one_ref)
    mags.append(one_ref)
    f, t, va_f, va_t, vm_f, vm_t, c, s = _branch_state(grid, x, L)
    for form in _flow_forms(grid):
        d = _flow_value_and_derivs(form, vm_f, vm_t, c, s)
        # row = var - F:  [1, -dF/dva_f, -dF/dva_t, -dF/dvm_f, -dF/dvm_t]
        v = np.concatenate([np.ones(nl), -d["th"][0], d["th"][0], -d["vmf"][0], -d["vmt"][0]])
        mm = np.concatenate([np.ones(nl), d["th"][1], d["th"][1], d["vmf"][1], d["vmt"][1]])
        vals.append(v)
        mags.append(mm)
    ang = np.concatenate([np.ones(nl), -np.ones(nl)])
    vals.append(ang)
    mags.append(np.abs(ang))
    p = x[L.P:L.P + 2 * nl]
    q = x[L.Q:L.Q + 2 * nl]
    for sl in (slice(0, nl), slice(nl, 2 * nl)):
        v = np.concatenate([2.0 * p[sl], 2.0 * q[sl]])
        vals.append(v)
        mags.append(np.abs(v))
    vm = x[L.VM:L.VM + L.nb]
    Gs, Bs = np.asarray(grid.Gs, np.float64), np.asarray(grid.Bs, np.float64)
    vals += [2.0 * Gs * vm, -2.0 * Bs * vm]
    mags += [np.abs(2.0 * Gs * vm), np.abs(2.0 * Bs * vm)]
    vals += [-np.ones(L.ng), -np.ones(L.ng)]
    mags += [np.ones(L.ng), np.ones(L.ng)]
    vals += [np.ones(2 * nl), np.ones(2 * nl)]
    mags += [np.ones(2 * nl), np.ones(2 * nl)]
    return np.concatenate(vals), np.concatenate(mags)


# ---------------------------------------------------------------------------
# Lagrangian Hessian W = sigma d2f + sum_r y_r d2g_r (lower COO).
# ---------------------------------------------------------------------------
def hessian(grid, x, y, obj_weight=1.0):
    """Hessian values in hess_structure order.  Returns (vals, M).

    Each branch entry sums, over the four flow rows r = var - F_r, the
    constraint's own second derivative -d2F_r weighted by y_r.  Thermal rows
    p^2 + q^2 give 2 y on each diagonal; the cost gives 2 sigma c2; the
    balance rows give 2 Gs y_P - 2 Bs y_Q on (vm_i, vm_i).
    """
    L = layout(grid)
    nl = L.nl
    f, t, va_f, va_t, vm_f, vm_t, c, s = _branch_state(grid, x, L)
    blk = np.zeros((nl, 10))
    blkM = np.zeros((nl, 10))
    for base, form in zip((L.PF, L.QF, L.PT, L.QT), _flow_forms(grid)):
        yr = y[base:base + nl]
        d = _flow_value_and_derivs(form, vm_f, vm_t, c, s)
        # second derivatives of F over local (va_f, va_t, vm_f, vm_t), in _HPAIRS order
        sec = [
            d["thth"],                                   # (va_f, va_f)
            (-d["thth"][0], d["thth"][1]),               # (va_t, va_f)
            d["thth"],                                   # (va_t, va_t)
            d["thvmf"],                                  # (vm_f, va_f)
            (-d["thvmf"][0], d["thvmf"][1]),             # (vm_f, va_t)
            d["vmfvmf"],                                 # (vm_f, vm_f)
            d["thvmt"],                                  # (vm_t, va_f)
            (-d["thvmt"][0], d["thvmt"][1]),             # (vm_t, va_t)
            d["vmfvmt"],                                 # (vm_t, vm_f)
            d["vmtvmt"],                                 # (vm_t, vm_t)
        ]
        for k, (val, mag) in enumerate(sec):
            blk[:, k] += yr * (-val)
            blkM[:, k] += np.abs(yr) * mag
    y_sf = y[L.SF:L.SF + nl]
    y_st = y[L.ST:L.ST + nl]
    th = np.stack([2.0 * y_sf, 2.0 * y_sf, 2.0 * y_st, 2.0 * y_st], axis=0)
    c2 = np.asarray(grid.c2, dtype=np.float64)
    hg = obj_weight * 2.0 * c2
    Gs, Bs = np.asarray(grid.Gs, np.float64), np.asarray(grid.Bs, np.float64)
    yP = y[L.PB:L.PB + L.nb]
    yQ = y[L.QB:L.QB + L.nb]
    hb = 2.0 * Gs * yP - 2.0 * Bs * yQ
    hbM = np.abs(2.0 * Gs * yP) + np.abs(2.0 * Bs * yQ)
    vals = np.concatenate([blk.T.ravel(), th.ravel(), hg, hb])
    mags = np.concatenate([blkM.T.ravel(), np.abs(th).ravel(), np.abs(hg), hbM])
    return vals, mags


# ---------------------------------------------------------------------------
# Condensed KKT matrix (Sec. IV.C).
# ---------------------------------------------------------------------------
def condensation_diag(sigma_s, delta_w=0.0, delta_c=0.0):
    """D = (Sigma_s + delta_w I) C with C = (delta_c Sigma_s + (1 + delta_c delta_w) I)^-1.
    Returns (D, |D| magnitude)."""
    sigma_s = np.asarray(sigma_s, dtype=np.float64)
    C = 1.0 / (delta_c * sigma_s + (1.0 + delta_c * delta_w))
    D = (sigma_s + delta_w) * C
    DM = (np.abs(sigma_s) + abs(delta_w)) * np.abs(C)
    return D, DM


def condensed_kkt(grid, hvals, jvals, sigma_x, sigma_s, delta_w=0.0, delta_c=0.0,
                  hmag=None, jmag=None, structure=None):
    """Values of the lower triangle of M_cond = W + delta_w I + Sigma_x + A' D A
    on kkt_structure's pattern.  Returns (kvals, M).

    W is the symmetric matrix whose lower triangle is the (duplicate-summed)
    Hessian COO; A is the Jacobian.  hmag / jmag are the magnitudes of the
    given H / J values (their absolute values when omitted)."""
    L = layout(grid)
    hvals = np.asarray(hvals, dtype=np.float64)
    jvals = np.asarray(jvals, dtype=np.float64)
    hmag = np.abs(hvals) if hmag is None else np.asarray(hmag, dtype=np.float64)
    jmag = np.abs(jvals) if jmag is None else np.asarray(jmag, dtype=np.float64)
    D, DM = condensation_diag(sigma_s, delta_w, delta_c)
    A = _jac_matrix(grid, jvals)
    AM = _jac_matrix(grid, jmag)
    Wl = _hess_lower_matrix(grid, hvals)
    WlM = _hess_lower_matrix(grid, hmag)
    W = Wl + Wl.T - sp.diags(Wl.diagonal())
    WM = WlM + WlM.T - sp.diags(WlM.diagonal())
    dx = np.asarray(sigma_x, dtype=np.float64) + delta_w
    dxM = np.abs(np.asarray(sigma_x, dtype=np.float64)) + abs(delta_w)
    K = W + sp.diags(dx) + A.T @ sp.diags(D) @ A
    KM = WM + sp.diags(dxM) + AM.T @ sp.diags(DM) @ AM
    rowptr, colind = kkt_structure(grid) if structure is None else structure
    rows = np.repeat(np.arange(L.n), np.diff(rowptr))
    K = K.tocsr()
    KM = KM.tocsr()
    kv = np.asarray(K[rows, colind]).ravel()
    km = np.asarray(KM[rows, colind]).ravel()
    return kv, km


def eval_assemble(grid, point, structure=None):
    """Everything one evaluate-and-assemble call produces, as a dict of
    (value, magnitude) pairs: f, grad, cons, jac, hess, kkt."""
    x = np.asarray(point.x, dtype=np.float64)
    f = objective(grid, x)
    gr = gradient(grid, x)
    cons = constraints(grid, x)
    jac = jacobian(grid, x)
    hess = hessian(grid, x, np.asarray(point.y, dtype=np.float64), point.obj_weight)
    kkt = condensed_kkt(grid, hess[0], jac[0], point.sigma_x, point.sigma_s,
                        point.delta_w, point.delta_c, hmag=hess[1], jmag=jac[1],
                        structure=structure)
    return {"f": f, "grad": gr, "cons": cons, "jac": jac, "hess": hess, "kkt": kkt}


def within_tol(value, oracle_value, magnitude, rel=TOL_REL, abs_=TOL_ABS):
    """Elementwise parity test |v - o| <= rel * M + abs."""
    value = np.asarray(value, dtype=np.float64)
    oracle_value = np.asarray(oracle_value, dtype=np.float64)
    magnitude = np.asarray(magnitude, dtype=np.float64)
    return np.abs(value - oracle_value) <= rel * magnitude + abs_
