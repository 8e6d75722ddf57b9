"""Plain CPU FP64 oracle: the condensation around M_cond and the step recovery.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV.C eliminates the bound-dual block of the Newton system (the 7x7
block system whose first three block rows carry W, A and the slacks) to the
augmented system M_aug [dx; ds; dy] = [q_x; q_s; q_y], and then the slack
and multiplier block to the condensed system M_cond dx = q_x + A'(C q_s +
D q_y).  This module computes, at an interior iterate:

* Sigma_x = Zl_x (X - Xl)^-1 + Zu_x (Xu - X)^-1, Sigma_s likewise over the
  slacks s with bounds sl, su;
* q_x = p_x + (X - Xl)^-1 p_zl_x - (Xu - X)^-1 p_zu_x, q_s likewise,
  q_y = p_y, where the p's are the right-hand sides of the Newton system;
* the condensed right-hand side r = q_x + A'(C q_s + D q_y) with
  C = (delta_c Sigma_s + (1 + delta_c delta_w) I)^-1, D = (Sigma_s + delta_w I) C;
* the recovery of ds, dy from dx and of the four bound-dual steps.

A bound at +-inf has no dual, no complementarity row and no barrier term:
its terms are taken as zero (the limit of the formulas).

Reading: Sec. IV.C prints ds = C (delta_c q_s - (q_y + A dx)).  Solving the
printed M_aug (third block row A dx - ds - delta_c dy = q_y, second block
row (Sigma_s + delta_w) ds - dy = q_s) gives ds = C (A dx + delta_c q_s - q_y),
the sign of A dx differing; the oracle follows the system, and the pins check
the recovered step against the printed 7x7 Newton system itself.

Every value comes with a magnitude (the sum of the absolute values of the
terms that make it up), as in the callbacks' oracle.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .acopf import _jac_matrix, condensation_diag

__all__ = ["Iterate", "inv_gap", "condense", "recover", "kkt_parts", "kkt_residual",
           "residual_scaling", "S_MAX"]


@dataclasses.dataclass
class Iterate:
    """An interior iterate with the right-hand sides of its Newton system.
    x (n) within [xl, xu], s (m) within [sl, su]; bound duals zl_x, zu_x (n),
    zl_s, zu_s (m), zero at infinite bounds; right-hand sides p_x (n), p_s,
    p_y (m), p_zl_x, p_zu_x (n), p_zl_s, p_zu_s (m)."""
    x: np.ndarray
    s: np.ndarray
    xl: np.ndarray
    xu: np.ndarray
    sl: np.ndarray
    su: np.ndarray
    zl_x: np.ndarray
    zu_x: np.ndarray
    zl_s: np.ndarray
    zu_s: np.ndarray
    p_x: np.ndarray
    p_s: np.ndarray
    p_y: np.ndarray
    p_zl_x: np.ndarray
    p_zu_x: np.ndarray
    p_zl_s: np.ndarray
    p_zu_s: np.ndarray


def inv_gap(v, lo, hi):
    """(V - Vlo)^-1 and (Vhi - V)^-1 per component; zero where the bound is
    infinite."""
    v, lo, hi = (np.asarray(a, dtype=np.float64) for a in (v, lo, hi))
    with np.errstate(divide="ignore", invalid="ignore"):
        il = np.where(np.isfinite(lo), 1.0 / (v - lo), 0.0)
        iu = np.where(np.isfinite(hi), 1.0 / (hi - v), 0.0)
    return il, iu


def _block(v, lo, hi, zl, zu, p, pl, pu):
    """Sigma and q of one block (x or s), with magnitudes."""
    il, iu = inv_gap(v, lo, hi)
    sig = zl * il + zu * iu
    sigm = np.abs(zl * il) + np.abs(zu * iu)
    q = p + il * pl - iu * pu
    qm = np.abs(p) + np.abs(il * pl) + np.abs(iu * pu)
    return sig, sigm, q, qm


def condense(grid, jvals, it: Iterate, delta_w=0.0, delta_c=0.0, jmag=None):
    """Sigma_x, Sigma_s, q_s and the condensed right-hand side r (Sec. IV.C).
    Returns a dict of (value, magnitude) pairs: sigma_x, sigma_s, q_s, rhs."""
    jvals = np.asarray(jvals, dtype=np.float64)
    jmag = np.abs(jvals) if jmag is None else np.asarray(jmag, dtype=np.float64)
    sx, sxm, qx, qxm = _block(it.x, it.xl, it.xu, it.zl_x, it.zu_x, it.p_x, it.p_zl_x,
                              it.p_zu_x)
    ss, ssm, qs, qsm = _block(it.s, it.sl, it.su, it.zl_s, it.zu_s, it.p_s, it.p_zl_s,
                              it.p_zu_s)
    qy = np.asarray(it.p_y, dtype=np.float64)
    C = 1.0 / (delta_c * ss + (1.0 + delta_c * delta_w))
    D, _ = condensation_diag(ss, delta_w, delta_c)
    w = C * qs + D * qy
    # magnitude of w: |C| |q_s| (with q_s's own magnitude) + |D| |q_y|
    wm = np.abs(C) * qsm + (np.abs(ss) + abs(delta_w)) * np.abs(C) * np.abs(qy)
    A = _jac_matrix(grid, jvals)
    AM = _jac_matrix(grid, jmag)
    rhs = qx + A.T @ w
    rhsm = qxm + AM.T @ wm
    return {"sigma_x": (sx, sxm), "sigma_s": (ss, ssm), "q_s": (qs, qsm),
            "rhs": (rhs, rhsm)}


def recover(grid, jvals, it: Iterate, dx, delta_w=0.0, delta_c=0.0, jmag=None):
    """The rest of the step from dx: ds, dy (from M_aug, see the module's
    reading) and the bound-dual steps (Sec. IV.C)
      dzl_x = (X - Xl)^-1 (p_zl_x - Zl_x dx),  dzu_x = (Xu - X)^-1 (p_zu_x + Zu_x dx),
      dzl_s = (S - Sl)^-1 (p_zl_s - Zl_s ds),  dzu_s = (Su - S)^-1 (p_zu_s + Zu_s ds).
    Returns a dict of (value, magnitude) pairs: ds, dy, dzl_x, dzu_x, dzl_s, dzu_s."""
    jvals = np.asarray(jvals, dtype=np.float64)
    jmag = np.abs(jvals) if jmag is None else np.asarray(jmag, dtype=np.float64)
    dx = np.asarray(dx, dtype=np.float64)
    ss, ssm, qs, qsm = _block(it.s, it.sl, it.su, it.zl_s, it.zu_s, it.p_s, it.p_zl_s,
                              it.p_zu_s)
    qy = np.asarray(it.p_y, dtype=np.float64)
    C = 1.0 / (delta_c * ss + (1.0 + delta_c * delta_w))
    A = _jac_matrix(grid, jvals)
    AM = _jac_matrix(grid, jmag)
    adx = A @ dx
    adxm = AM @ np.abs(dx)
    inner = adx + delta_c * qs - qy
    innerm = adxm + abs(delta_c) * qsm + np.abs(qy)
    ds = C * inner
    dsm = np.abs(C) * innerm
    g = ss + delta_w
    dy = g * ds - qs
    dym = (ssm + abs(delta_w)) * dsm + qsm
    ilx, iux = inv_gap(it.x, it.xl, it.xu)
    ils, ius = inv_gap(it.s, it.sl, it.su)
    out = {"ds": (ds, dsm), "dy": (dy, dym)}
    for name, inv, z, p, d, dm, sign in (
            ("dzl_x", ilx, it.zl_x, it.p_zl_x, dx, np.abs(dx), -1.0),
            ("dzu_x", iux, it.zu_x, it.p_zu_x, dx, np.abs(dx), 1.0),
            ("dzl_s", ils, it.zl_s, it.p_zl_s, ds, dsm, -1.0),
            ("dzu_s", ius, it.zu_s, it.p_zu_s, ds, dsm, 1.0)):
        val = inv * (p + sign * z * d)
        mag = np.abs(inv) * (np.abs(p) + np.abs(z) * dm)
        out[name] = (val, mag)
    return out


# ---------------------------------------------------------------------------
# Scaled residual of the first-order conditions (the termination test of
# Algorithm 1; Sec. IV calls it a scaled version of the residual of Eq. first
# and refers to Waechter and Biegler 2006 for the details).  Reading: the
# scaling of that reference, eq. (5), with s_max = 100:
#   E = max(||r_d||_inf / s_d, ||r_p||_inf, ||r_c||_inf / s_c),
#   s_d = max(s_max, (||y||_1 + ||z||_1) / (m + n_z)) / s_max,
#   s_c = max(s_max, ||z||_1 / n_z) / s_max,
# over the conditions of Eq. first:
#   r_d = [grad f - A'y - zl_x + zu_x ; y - zl_s + zu_s]   (n + m)
#   r_p = g(x) - s                                         (m)
#   r_c = [Zl_x (x - xl) - mu ; Zu_x (xu - x) - mu ; Zl_s (s - sl) - mu ; Zu_s (su - s) - mu]
# with only the finite bounds carrying a dual (n_z of them).
# ---------------------------------------------------------------------------
S_MAX = 100.0


def residual_scaling(y_l1, z_l1, m, n_z):
    """(s_d, s_c) of the scaled residual."""
    s_d = max(S_MAX, (y_l1 + z_l1) / (m + n_z)) / S_MAX
    s_c = max(S_MAX, z_l1 / n_z) / S_MAX if n_z else 1.0
    return s_d, s_c


def kkt_parts(grid, grad, cons, jvals, it: Iterate, y, mu):
    """The residual vectors: (r_d_x, r_d_s, r_p, r_c, z of the finite bounds)."""
    grad, cons, y = (np.asarray(a, dtype=np.float64) for a in (grad, cons, y))
    A = _jac_matrix(grid, np.asarray(jvals, dtype=np.float64))
    rdx = grad - A.T @ y - it.zl_x + it.zu_x
    rds = y - it.zl_s + it.zu_s
    rp = cons - it.s
    parts = []
    zs = []
    for v, b, z, sign in ((it.x, it.xl, it.zl_x, 1.0), (it.x, it.xu, it.zu_x, -1.0),
                          (it.s, it.sl, it.zl_s, 1.0), (it.s, it.su, it.zu_s, -1.0)):
        f = np.isfinite(b)
        parts.append(z[f] * (sign * (v[f] - b[f])) - mu)
        zs.append(z[f])
    return rdx, rds, rp, np.concatenate(parts), np.concatenate(zs)


def kkt_residual(grid, grad, cons, jvals, it: Iterate, y, mu):
    """The parts of the scaled residual: dict with dual_inf, primal_inf,
    compl_inf, y_l1, z_l1, n_z, s_d, s_c, residual."""
    y = np.asarray(y, dtype=np.float64)
    rdx, rds, rp, rc, zall = kkt_parts(grid, grad, cons, jvals, it, y, mu)
    n_z = zall.size
    m = y.size
    y_l1, z_l1 = float(np.sum(np.abs(y))), float(np.sum(np.abs(zall)))
    s_d, s_c = residual_scaling(y_l1, z_l1, m, n_z)
    dual_inf = float(max(np.max(np.abs(rdx)), np.max(np.abs(rds))))
    primal_inf = float(np.max(np.abs(rp)))
    compl_inf = float(np.max(np.abs(rc))) if n_z else 0.0
    return {"dual_inf": dual_inf, "primal_inf": primal_inf, "compl_inf": compl_inf,
            "y_l1": y_l1, "z_l1": z_l1, "n_z": n_z, "s_d": s_d, "s_c": s_c,
            "residual": max(dual_inf / s_d, primal_inf, compl_inf / s_c)}
