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

__all__ = ["Iterate", "inv_gap", "condense", "recover"]


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
