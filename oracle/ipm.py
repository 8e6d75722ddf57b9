"""Plain CPU FP64 oracle: the condensed-space interior-point method (Algorithm 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Algorithm 1 of the paper, in its order: relax the equality constraints
(Eq. relax, Sec. IV.A: the slack bounds are the constraint bounds widened by
eps_tol, so an equality row g_r = 0 becomes -eps_tol <= s_r <= eps_tol), then
repeat until the scaled residual of Eq. first is below eps_tol: solve the
condensed system with delta_w = delta_c = 0, regularise and re-solve when the
factorization shows the wrong inertia, choose the step sizes by line search,
update the iterate (Eq. iter), update the filter and the barrier parameter.

The paper defers the line search, the barrier update and the inertia
correction to the interior-point reference it cites (Waechter and Biegler
2006); this oracle takes that reference's rules, written from its
description, with its default constants: the fraction-to-boundary rule with
tau = max(tau_min, 1 - mu); the filter line search (switching condition,
Armijo condition on the barrier objective, sufficient decrease in the
constraint violation or the barrier objective, filter acceptance) with its
second-order correction (`second_order_correction`: when the first trial
point is rejected and does not reduce the violation, the same matrix is
solved again with the constraint residual replaced by
c_soc = alpha c(x_k) + c(x_trial), at most soc_max times while the violation
keeps falling by kappa_soc; reading d11); the monotone
barrier update mu <- max(eps/10, min(kappa_mu mu, mu^theta_mu)) when the
barrier problem's error is below kappa_eps mu; the inertia correction on
delta_w (delta_c = 0); the safeguard of the bound multipliers
(kappa_sigma); the initial point pushed into the interior of the bounds;
when the line search fails, a feasibility restoration (reading d10,
`restoration`) that either returns a point the filter accepts or ends the
solve with status "infeasible".

Readings:
* (d7) Eq. first uses the Lagrangian f - y'(g - s) (its first row carries
  -grad g' y); the printed Newton matrix carries +A' and -I in the column of
  Delta y, so its Delta y is the negative of the Newton step of y in Eq.
  first.  The oracle solves the printed system (through the condensation and
  recovery of oracle.step), takes W = grad^2 f - sum_r y_r grad^2 g_r (the
  callbacks' Hessian with multipliers -y) and updates y <- y - alpha Delta y.
* (d8) the initial point: voltage angles 0, magnitudes 1, generator outputs
  and flows at the middle of their bounds (0 when unbounded), pushed into
  the interior; slacks at g(x0) pushed into their bounds; y = 0; bound
  multipliers 1 at finite bounds.
* (d11) second-order correction: c(x) = g(x) - s; the corrected step is the
  whole primal-dual solution of the corrected system (x, s and y move by the
  fraction-to-boundary step alpha_soc along it, the bound multipliers by
  their own fraction-to-boundary step along its Delta z); the corrected
  point's switching and Armijo tests use the first trial step alpha_{k,0},
  as the reference states.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .acopf import bounds, constraints, gradient, hessian, jacobian, layout, objective
from .acopf import condensed_kkt
from .chol import is_positive_definite, solve_condensed
from .step import Iterate, condense, kkt_residual, recover

__all__ = ["IpmOptions", "IpmResult", "ipm_start", "ipm_solve", "relaxed_bounds",
           "push_interior", "fraction_to_boundary", "barrier_objective", "restoration",
           "second_order_correction"]


@dataclasses.dataclass
class IpmOptions:
    tol: float = 1e-4            # eps_tol: convergence and relaxation (Sec. IV.A)
    max_iter: int = 200
    mu_init: float = 0.1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    bound_push: float = 1e-2     # kappa_1
    bound_frac: float = 1e-2     # kappa_2
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-8
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-4
    alpha_min_frac: float = 0.05
    kappa_sigma: float = 1e10
    delta_w0: float = 1e-4
    delta_w_min: float = 1e-20
    delta_w_max: float = 1e40
    kappa_w_minus: float = 1.0 / 3.0
    kappa_w_plus: float = 8.0
    kappa_w_plus_bar: float = 100.0
    max_backtracks: int = 60
    soc_max: int = 4              # second-order corrections per line search at most (p_max)
    kappa_soc: float = 0.99       # ... each must cut the violation below this fraction of the last
    resto_max_iter: int = 200     # restoration iterations at most
    resto_stall: int = 10         # ... and without a 1 % decrease of the violation for this many
    resto_mu_min: float = 1e-9    # the restoration's barrier parameter at least
    resto_reduction: float = 0.9  # restoration ends below this fraction of the violation
    resto_reduction_repeat: float = 1e-3  # ... when re-entered without progress since its last exit


@dataclasses.dataclass
class IpmResult:
    status: str
    iterations: int
    objective: float
    residual: float
    x: np.ndarray
    s: np.ndarray
    y: np.ndarray
    zl_x: np.ndarray
    zu_x: np.ndarray
    zl_s: np.ndarray
    zu_s: np.ndarray
    mu: float
    history: list


def relaxed_bounds(gl, gu, tol):
    """Slack bounds of Eq. relax: each finite constraint bound widened by
    tol max(1, |bound|)."""
    gl, gu = np.asarray(gl, dtype=np.float64), np.asarray(gu, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        sl = np.where(np.isfinite(gl), gl - tol * np.maximum(1.0, np.abs(gl)), -np.inf)
        su = np.where(np.isfinite(gu), gu + tol * np.maximum(1.0, np.abs(gu)), np.inf)
    return sl, su


def push_interior(v, lo, hi, k1, k2):
    """The reference's initial-point rule: move v at least
    p = min(k1 max(1, |bound|), k2 (hi - lo)) inside each finite bound."""
    v = np.asarray(v, dtype=np.float64).copy()
    lo_f, hi_f = np.isfinite(lo), np.isfinite(hi)
    both = lo_f & hi_f
    with np.errstate(invalid="ignore"):
        width = np.where(both, hi - lo, np.inf)
        pl = np.minimum(k1 * np.maximum(1.0, np.abs(np.where(lo_f, lo, 0.0))), k2 * width)
        pu = np.minimum(k1 * np.maximum(1.0, np.abs(np.where(hi_f, hi, 0.0))), k2 * width)
    v = np.where(lo_f, np.maximum(v, lo + pl), v)
    v = np.where(hi_f, np.minimum(v, hi - pu), v)
    return v


def ipm_start(grid, opts: IpmOptions):
    """Reading d8: the initial primal-dual point and the slack bounds."""
    L = layout(grid)
    xl, xu, gl, gu = bounds(grid)
    sl, su = relaxed_bounds(gl, gu, opts.tol)
    both = np.isfinite(xl) & np.isfinite(xu)
    mid = np.zeros(L.n)
    mid[both] = 0.5 * (xl[both] + xu[both])
    x0 = mid.copy()
    x0[L.VA:L.VA + L.nb] = 0.0
    x0[L.VM:L.VM + L.nb] = 1.0
    x = push_interior(x0, xl, xu, opts.bound_push, opts.bound_frac)
    s = push_interior(np.clip(constraints(grid, x)[0], sl, su), sl, su, opts.bound_push,
                      opts.bound_frac)
    y = np.zeros(L.m)
    ones = lambda b: np.where(np.isfinite(b), 1.0, 0.0)  # noqa: E731
    return dict(x=x, s=s, y=y, zl_x=ones(xl), zu_x=ones(xu), zl_s=ones(sl), zu_s=ones(su),
                xl=xl, xu=xu, sl=sl, su=su)


def fraction_to_boundary(v, dv, lo, hi, tau):
    """Largest alpha in (0, 1] with lo + (1 - tau)(v - lo) <= v + alpha dv and
    the same at hi (finite bounds only)."""
    a = 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        m = np.isfinite(lo) & (dv < 0)
        if m.any():
            a = min(a, float(np.min(-tau * (v[m] - lo[m]) / dv[m])))
        m = np.isfinite(hi) & (dv > 0)
        if m.any():
            a = min(a, float(np.min(tau * (hi[m] - v[m]) / dv[m])))
    return a


def _dual_fraction(z, dz, tau):
    """Largest alpha in (0, 1] keeping z + alpha dz >= (1 - tau) z."""
    m = dz < 0
    if not m.any():
        return 1.0
    return min(1.0, float(np.min(-tau * z[m] / dz[m])))


def _log_gaps(v, lo, hi):
    fl, fu = np.isfinite(lo), np.isfinite(hi)
    return float(np.sum(np.log(v[fl] - lo[fl])) + np.sum(np.log(hi[fu] - v[fu])))


def barrier_objective(f, x, s, b, mu):
    """phi_mu of Eq. barrier: f - mu (sum of the logs of every finite gap)."""
    return f - mu * (_log_gaps(x, b["xl"], b["xu"]) + _log_gaps(s, b["sl"], b["su"]))


def _barrier_directional(grad, x, s, dx, ds, b, mu):
    """grad phi_mu' (dx, ds) = grad f' dx - mu sum dv/(v - lo) + mu sum dv/(hi - v)
    over the finite bounds of x and s."""
    def part(v, dv, lo, hi):
        fl, fu = np.isfinite(lo), np.isfinite(hi)
        return float(-np.sum(dv[fl] / (v[fl] - lo[fl])) + np.sum(dv[fu] / (hi[fu] - v[fu])))
    return float(grad @ dx) + mu * (part(x, dx, b["xl"], b["xu"]) + part(s, ds, b["sl"], b["su"]))


def _reset_z(z, gap, mu, kappa):
    """Safeguard of the bound multipliers: z within [mu/(kappa gap), kappa mu/gap]."""
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.where(np.isfinite(gap) & (z > 0),
                       np.maximum(np.minimum(z, kappa * mu / gap), mu / (kappa * gap)), z)
    return out


def second_order_correction(grid, J, it, kv, dw, c_soc):
    """One second-order-corrected direction of the filter line search (the
    interior-point reference the paper cites, reading d11): the Newton system
    of the iterate `it` (its matrix kv = M_cond with regularisation dw, its
    right-hand side) with the constraint part -(g - s) replaced by -c_soc.
    Returns dx, ds, dy (the step of y, reading d7) and the four
    bound-multiplier steps."""
    it_soc = dataclasses.replace(it, p_y=-c_soc)
    c = condense(grid, J, it_soc, dw, 0.0)
    dx = solve_condensed(grid, kv, c["rhs"][0])
    r = recover(grid, J, it_soc, dx, dw, 0.0)
    out = dict(dx=dx, ds=r["ds"][0], dy=-r["dy"][0])
    for k in ("dzl_x", "dzu_x", "dzl_s", "dzu_s"):
        out[k] = r[k][0]
    return out


def restoration(grid, x, b, mu, accept, opts: IpmOptions):
    """Feasibility restoration (reading d10), entered when the line search
    fails: minimise over x inside its bounds

        psi(x) = 1/2 ||v(x)||^2 - mu_R sum(log gaps of x) + zeta/2 ||x - x_R||^2,
        v(x) = g(x) - P(g(x)),

    P clipping onto the slack box pushed inside as for the initial point
    (the slacks follow g), zeta = sqrt(mu_R), x_R the current point (so the
    proximal term damps each step, Levenberg-Marquardt fashion), mu_R
    starting at the main barrier parameter and divided by 10 whenever the
    violation stalls.  Each step is a Gauss-Newton step,
    (A' W A + Sigma + zeta I) dx = -grad psi with W the 0/1 diagonal of the
    rows outside the box and Sigma the barrier's curvature: M_cond's pattern
    with no Hessian and D = W.  Step sizes: fraction to the boundary
    (tau = 0.99), then halving until psi decreases by 1e-4 alpha grad psi'dx.
    Returns ("ok", x, s) as soon as accept(x, s) holds (the main filter
    accepts the point, whose violation is at most resto_reduction times the
    one where the line search failed), else ("infeasible", x, s) when the violation stops
    decreasing with mu_R at resto_mu_min (less than 1 % over resto_stall
    iterations, or a step below 1e-12), or after resto_max_iter iterations:
    a point of local infeasibility."""
    L = layout(grid)
    xl, xu, sl, su = b["xl"], b["xu"], b["sl"], b["su"]
    lo_s = push_interior(np.full(L.m, -np.inf), sl, su, opts.bound_push, opts.bound_frac)
    hi_s = push_interior(np.full(L.m, np.inf), sl, su, opts.bound_push, opts.bound_frac)
    lo_s = np.where(np.isfinite(sl), lo_s, -np.inf)
    hi_s = np.where(np.isfinite(su), hi_s, np.inf)
    mu_r = mu  # the restoration's own barrier parameter
    x_r = x.copy()
    fl, fu = np.isfinite(xl), np.isfinite(xu)

    def parts(xv):
        g = constraints(grid, xv)[0]
        sv = np.clip(g, lo_s, hi_s)
        return g, sv, g - sv

    def psi(xv, v):
        return (0.5 * float(v @ v) - mu_r * _log_gaps(xv, xl, xu)
                + 0.5 * np.sqrt(mu_r) * float((xv - x_r) @ (xv - x_r)))

    g, s, v = parts(x)
    best, since = float(np.sum(np.abs(v))), 0
    for _ in range(opts.resto_max_iter):
        if accept(x, s):
            return "ok", x, s
        J = jacobian(grid, x)[0]
        w = (v != 0.0).astype(np.float64)
        with np.errstate(divide="ignore"):
            gl_ = np.where(fl, 1.0 / (x - np.where(fl, xl, 0.0)), 0.0)
            gu_ = np.where(fu, 1.0 / (np.where(fu, xu, 0.0) - x), 0.0)
        zeta = np.sqrt(mu_r)
        grad = J_T(grid, J, w * v) + mu_r * (gu_ - gl_) + zeta * (x - x_r)
        sig = mu_r * (gl_ * gl_ + gu_ * gu_) + zeta
        kv, _ = condensed_kkt(grid, np.zeros(hessian(grid, x, np.zeros(L.m), 0.0)[0].size), J,
                              sig, w, 0.0, 0.0)
        dx = solve_condensed(grid, kv, -grad)
        alpha = fraction_to_boundary(x, dx, xl, xu, 0.99)
        p0, slope = psi(x, v), float(grad @ dx)
        while True:
            xt = x + alpha * dx
            gt, st_, vt = parts(xt)
            if psi(xt, vt) <= p0 + 1e-4 * alpha * slope:
                break
            alpha *= 0.5
            if alpha < 1e-12:
                break
        if alpha < 1e-12:  # no decrease along the step: a smaller barrier, else infeasible
            if mu_r <= opts.resto_mu_min:
                return "infeasible", x, s
            mu_r, since = 0.1 * mu_r, 0
            continue
        x, g, s, v = xt, gt, st_, vt
        x_r = x.copy()  # the proximal term damps each step (Levenberg-Marquardt)
        th = float(np.sum(np.abs(v)))
        if th < 0.99 * best:
            best, since = th, 0
        else:
            since += 1
            if since >= opts.resto_stall:  # stalled: a smaller barrier, else local infeasibility
                if mu_r <= opts.resto_mu_min:
                    return "infeasible", x, s
                mu_r, since = 0.1 * mu_r, 0
    return ("ok", x, s) if accept(x, s) else ("infeasible", x, s)


def ipm_solve(grid, opts: IpmOptions | None = None, factor_check=None) -> IpmResult:
    """Algorithm 1 on the AC-OPF model of `grid`.  factor_check(kvals) may
    replace the dense positive-definiteness test (the default)."""
    opts = opts or IpmOptions()
    L = layout(grid)
    st = ipm_start(grid, opts)
    b = {k: st[k] for k in ("xl", "xu", "sl", "su")}
    x, s, y = st["x"], st["s"], st["y"]
    zl_x, zu_x, zl_s, zu_s = st["zl_x"], st["zu_x"], st["zl_s"], st["zu_s"]
    pd = factor_check or (lambda kv: is_positive_definite(grid, kv))
    mu = opts.mu_init
    dw_last = 0.0
    history = []

    def evaluate(xv):
        return (objective(grid, xv)[0], gradient(grid, xv)[0], constraints(grid, xv)[0],
                jacobian(grid, xv)[0])

    def theta_of(cons, sv):
        return float(np.sum(np.abs(cons - sv)))

    f, grad, cons, J = evaluate(x)
    theta0 = theta_of(cons, s)
    theta_max = 1e4 * max(1.0, theta0)
    theta_min = 1e-4 * max(1.0, theta0)
    filt = [(theta_max, -np.inf)]
    status = "max_iter"
    it_count = 0
    res0 = None
    resto_exit = None  # the violation where the last restoration ended
    for it_count in range(opts.max_iter + 1):
        it = Iterate(x=x, s=s, xl=b["xl"], xu=b["xu"], sl=b["sl"], su=b["su"], zl_x=zl_x,
                     zu_x=zu_x, zl_s=zl_s, zu_s=zu_s, p_x=np.zeros(L.n), p_s=np.zeros(L.m),
                     p_y=np.zeros(L.m), p_zl_x=np.zeros(L.n), p_zu_x=np.zeros(L.n),
                     p_zl_s=np.zeros(L.m), p_zu_s=np.zeros(L.m))
        res0 = kkt_residual(grid, grad, cons, J, it, y, 0.0)
        history.append(dict(iter=it_count, f=f, residual=res0["residual"], mu=mu,
                            theta=theta_of(cons, s)))
        if res0["residual"] <= opts.tol:
            status = "converged"
            break
        if it_count == opts.max_iter:
            break
        # barrier update (monotone), possibly several times
        while mu > opts.tol / 10.0:
            if kkt_residual(grid, grad, cons, J, it, y, mu)["residual"] > opts.kappa_eps * mu:
                break
            mu = max(opts.tol / 10.0, min(opts.kappa_mu * mu, mu ** opts.theta_mu))
            filt = [(theta_max, -np.inf)]
        tau = max(opts.tau_min, 1.0 - mu)
        # Newton right-hand side of the printed system: minus Eq. first
        rdx = grad - J_T(grid, J, y) - zl_x + zu_x
        rds = y - zl_s + zu_s
        gx = np.where(np.isfinite(b["xl"]), x - b["xl"], 0.0)
        hx = np.where(np.isfinite(b["xu"]), b["xu"] - x, 0.0)
        gs = np.where(np.isfinite(b["sl"]), s - b["sl"], 0.0)
        hs = np.where(np.isfinite(b["su"]), b["su"] - s, 0.0)
        fin = lambda bd, v: np.where(np.isfinite(bd), v, 0.0)  # noqa: E731
        it.p_x, it.p_s, it.p_y = -rdx, -rds, -(cons - s)
        it.p_zl_x = fin(b["xl"], mu - zl_x * gx)
        it.p_zu_x = fin(b["xu"], mu - zu_x * hx)
        it.p_zl_s = fin(b["sl"], mu - zl_s * gs)
        it.p_zu_s = fin(b["su"], mu - zu_s * hs)
        H = hessian(grid, x, -y, 1.0)[0]
        # inertia correction on delta_w (delta_c = 0)
        dw = 0.0
        for _ in range(200):
            c = condense(grid, J, it, dw, 0.0)
            kv, _ = condensed_kkt(grid, H, J, c["sigma_x"][0], c["sigma_s"][0], dw, 0.0)
            if pd(kv):
                break
            if dw == 0.0:
                dw = opts.delta_w0 if dw_last == 0.0 else max(opts.delta_w_min,
                                                                opts.kappa_w_minus * dw_last)
            else:
                dw *= opts.kappa_w_plus_bar if dw_last == 0.0 else opts.kappa_w_plus
            if dw > opts.delta_w_max:
                status = "inertia correction failed"
                break
        if status == "inertia correction failed":
            break
        if dw > 0.0:
            dw_last = dw
        dx = solve_condensed(grid, kv, c["rhs"][0])
        r = recover(grid, J, it, dx, dw, 0.0)
        ds, dyh = r["ds"][0], r["dy"][0]
        dy = -dyh  # reading d7
        dzl_x, dzu_x, dzl_s, dzu_s = (r[k][0] for k in ("dzl_x", "dzu_x", "dzl_s", "dzu_s"))
        a_max = min(fraction_to_boundary(x, dx, b["xl"], b["xu"], tau),
                    fraction_to_boundary(s, ds, b["sl"], b["su"], tau))
        a_z = min(_dual_fraction(zl_x, dzl_x, tau), _dual_fraction(zu_x, dzu_x, tau),
                  _dual_fraction(zl_s, dzl_s, tau), _dual_fraction(zu_s, dzu_s, tau))
        # filter line search
        theta = theta_of(cons, s)
        phi = barrier_objective(f, x, s, b, mu)
        gphi = _barrier_directional(grad, x, s, dx, ds, b, mu)
        alpha_min = opts.alpha_min_frac * min(
            opts.gamma_theta,
            opts.gamma_phi * theta / (-gphi) if gphi < 0 else np.inf,
            opts.delta * theta ** opts.s_theta / (-gphi) ** opts.s_phi if gphi < 0 else np.inf)
        def acceptable(tht, pht, a):
            """"f" (Armijo step), "h" (filter-type step) or None for a trial
            point of violation tht and barrier objective pht at step a."""
            if any(tht >= fth and pht >= fph for fth, fph in filt):
                return None
            switching = gphi < 0 and a * (-gphi) ** opts.s_phi > opts.delta * theta ** opts.s_theta
            if switching and theta <= theta_min:
                return "f" if pht <= phi + opts.eta_phi * a * gphi else None
            if tht <= (1 - opts.gamma_theta) * theta or pht <= phi - opts.gamma_phi * theta:
                return "h"
            return None

        alpha = a_max
        accepted = None
        n_soc = 0
        for bt in range(opts.max_backtracks):
            xt, st_ = x + alpha * dx, s + alpha * ds
            ft, ct = objective(grid, xt)[0], constraints(grid, xt)[0]
            tht = theta_of(ct, st_)
            pht = barrier_objective(ft, xt, st_, b, mu)
            kind = acceptable(tht, pht, alpha)
            if kind is not None:
                accepted = (kind, xt, st_, ft, ct)
                break
            if bt == 0 and tht >= theta:
                # second-order correction: c_soc = alpha c(x_k) + c(x_trial), then
                # alpha_soc c_soc + c(x_soc) while the violation keeps falling
                c_soc = alpha * (cons - s) + (ct - st_)
                th_old = theta
                for _ in range(opts.soc_max):
                    n_soc += 1
                    d = second_order_correction(grid, J, it, kv, dw, c_soc)
                    a_soc = min(fraction_to_boundary(x, d["dx"], b["xl"], b["xu"], tau),
                                fraction_to_boundary(s, d["ds"], b["sl"], b["su"], tau))
                    xs, ss = x + a_soc * d["dx"], s + a_soc * d["ds"]
                    fs, cs = objective(grid, xs)[0], constraints(grid, xs)[0]
                    ths = theta_of(cs, ss)
                    kind = acceptable(ths, barrier_objective(fs, xs, ss, b, mu), a_max)
                    if kind is not None:
                        accepted = (kind, xs, ss, fs, cs)
                        alpha, dy = a_soc, d["dy"]
                        dzl_x, dzu_x, dzl_s, dzu_s = (d[k] for k in ("dzl_x", "dzu_x", "dzl_s",
                                                                     "dzu_s"))
                        a_z = min(_dual_fraction(zl_x, dzl_x, tau), _dual_fraction(zu_x, dzu_x, tau),
                                  _dual_fraction(zl_s, dzl_s, tau), _dual_fraction(zu_s, dzu_s, tau))
                        break
                    if ths > opts.kappa_soc * th_old:
                        break
                    c_soc = a_soc * c_soc + (cs - ss)
                    th_old = ths
                if accepted is not None:
                    break
            alpha *= 0.5
            if alpha < alpha_min:
                break
        if accepted is None:
            # feasibility restoration: a point the filter (augmented with the
            # current one) accepts with a sufficiently smaller violation
            filt.append(((1 - opts.gamma_theta) * theta, phi - opts.gamma_phi * theta))

            # back without getting below the last restoration's exit: demand
            # (nearly) feasibility this time, which an infeasible network cannot give
            red = (opts.resto_reduction_repeat
                   if resto_exit is not None and theta >= resto_exit else opts.resto_reduction)

            def accept(xv, sv, theta=theta, mu=mu, red=red):
                fv, cv = objective(grid, xv)[0], constraints(grid, xv)[0]
                tv = theta_of(cv, sv)
                pv = barrier_objective(fv, xv, sv, b, mu)
                return tv <= red * theta and not any(
                    tv >= fth and pv >= fph for fth, fph in filt)

            rstat, x, s = restoration(grid, x, b, mu, accept, opts)
            f, cons = objective(grid, x)[0], constraints(grid, x)[0]
            resto_exit = theta_of(cons, s)
            grad, J = gradient(grid, x)[0], jacobian(grid, x)[0]
            history[-1].update(alpha=0.0, alpha_z=0.0, delta_w=dw, restoration=True)
            if rstat != "ok":
                status = "infeasible"
                break
            # multipliers restart: y = 0, bound duals on the central path
            y = np.zeros(L.m)
            with np.errstate(divide="ignore", invalid="ignore"):
                zl_x = np.where(np.isfinite(b["xl"]), mu / (x - b["xl"]), 0.0)
                zu_x = np.where(np.isfinite(b["xu"]), mu / (b["xu"] - x), 0.0)
                zl_s = np.where(np.isfinite(b["sl"]), mu / (s - b["sl"]), 0.0)
                zu_s = np.where(np.isfinite(b["su"]), mu / (b["su"] - s), 0.0)
            continue
        kind, x, s, f, cons = accepted
        if kind == "h":
            filt.append(((1 - opts.gamma_theta) * theta, phi - opts.gamma_phi * theta))
        y = y + alpha * dy
        zl_x, zu_x = zl_x + a_z * dzl_x, zu_x + a_z * dzu_x
        zl_s, zu_s = zl_s + a_z * dzl_s, zu_s + a_z * dzu_s
        with np.errstate(invalid="ignore"):
            zl_x = _reset_z(zl_x, x - b["xl"], mu, opts.kappa_sigma)
            zu_x = _reset_z(zu_x, b["xu"] - x, mu, opts.kappa_sigma)
            zl_s = _reset_z(zl_s, s - b["sl"], mu, opts.kappa_sigma)
            zu_s = _reset_z(zu_s, b["su"] - s, mu, opts.kappa_sigma)
        grad, J = gradient(grid, x)[0], jacobian(grid, x)[0]
        history[-1].update(alpha=alpha, alpha_z=a_z, delta_w=dw, soc=n_soc)
    return IpmResult(status=status, iterations=it_count, objective=float(f),
                     residual=float(res0["residual"]) if res0 else np.inf, x=x, s=s, y=y,
                     zl_x=zl_x, zu_x=zu_x, zl_s=zl_s, zu_s=zu_s, mu=mu, history=history)


def J_T(grid, jvals, y):
    """A' y."""
    from .acopf import _jac_matrix
    return _jac_matrix(grid, np.asarray(jvals, dtype=np.float64)).T @ y
