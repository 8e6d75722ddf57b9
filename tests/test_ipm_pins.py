"""Pins of the interior-point oracle (oracle/ipm.py, Algorithm 1).

* The Newton step (condensation, solve, recovery, with the printed Delta y
  taken as minus the Newton step of y: reading d7) solves the linearization
  of Eq. first: F(v + eps d) = (1 - eps) F(v) to first order, checked by
  evaluating the conditions of Eq. first from the callbacks alone; the
  opposite reading of Delta y fails.
* The solution on the half-loaded 30-bus network matches an independent
  solver (scipy's SLSQP from the same start) and satisfies the bounds and
  the relaxed constraints.
* The second-order correction (reading d11): its direction solves the same
  linearization with the constraint residual replaced by c_soc, i.e. the
  constraint row moves by -eps c_soc and the other rows of Eq. first by
  -eps F, checked from the callbacks alone; the opposite sign of c_soc
  fails; on the half-loaded 7-bus edge case the solve takes a corrected
  step and converges to the point the solve without corrections reaches.
* The initial-point and step-bound rules against hand values.
* The feasibility restoration (reading d10): on the 30-bus network at 0.8
  and 1.0 times its loads, which have no feasible point, the solve stops as
  infeasible at a point whose violation equals the smallest one an
  independent least-squares solver (scipy's trust-region reflective method
  from random starts) finds; at 0.6 times the loads (feasible) it converges.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.ipm import IpmOptions, fraction_to_boundary, ipm_start, push_interior
from paper_2307_16830_gb300 import synth


def _conditions(g, b, x, s, y, z, mu):
    """The left-hand sides of Eq. first (the complementarity rows at finite
    bounds only)."""
    grad = oracle.gradient(g, x)[0]
    cons = oracle.constraints(g, x)[0]
    A = oracle.acopf._jac_matrix(g, oracle.jacobian(g, x)[0])
    fin = lambda bd, v: np.where(np.isfinite(bd), v, 0.0)  # noqa: E731
    with np.errstate(invalid="ignore"):
        return [grad - A.T @ y - z["zl_x"] + z["zu_x"], y - z["zl_s"] + z["zu_s"], cons - s,
                fin(b["xl"], z["zl_x"] * (x - b["xl"]) - mu),
                fin(b["xu"], z["zu_x"] * (b["xu"] - x) - mu),
                fin(b["sl"], z["zl_s"] * (s - b["sl"]) - mu),
                fin(b["su"], z["zu_s"] * (b["su"] - s) - mu)]


def _newton_check(dy_sign):
    g = synth.workload_grid("30bus-opf")
    L = oracle.layout(g)
    st = ipm_start(g, IpmOptions())
    b = {k: st[k] for k in ("xl", "xu", "sl", "su")}
    rng = np.random.default_rng(0)
    x, s = st["x"], st["s"]
    y = rng.standard_normal(L.m) * 0.1
    z = {k: st[k] * (1 + rng.random(st[k].size)) for k in ("zl_x", "zu_x", "zl_s", "zu_s")}
    mu = 0.1
    F0 = _conditions(g, b, x, s, y, z, mu)
    J = oracle.jacobian(g, x)[0]
    it = oracle.Iterate(x=x, s=s, **b, **z, p_x=-F0[0], p_s=-F0[1], p_y=-F0[2], p_zl_x=-F0[3],
                        p_zu_x=-F0[4], p_zl_s=-F0[5], p_zu_s=-F0[6])
    H = oracle.hessian(g, x, -y, 1.0)[0]
    c = oracle.condense(g, J, it, 0.0, 0.0)
    kv, _ = oracle.condensed_kkt(g, H, J, c["sigma_x"][0], c["sigma_s"][0], 0.0, 0.0)
    dx = oracle.solve_condensed(g, kv, c["rhs"][0])
    r = oracle.recover(g, J, it, dx, 0.0, 0.0)
    eps = 1e-7
    z1 = {k: z[k] + eps * r["d" + k][0] for k in z}
    F1 = _conditions(g, b, x + eps * dx, s + eps * r["ds"][0], y + dy_sign * eps * r["dy"][0],
                     z1, mu)
    return [np.max(np.abs(F1[i] - (1 - eps) * F0[i])) / (eps * np.max(np.abs(F0[i])))
            for i in range(7)]


def _soc_check(c_sign):
    """Relative errors of the corrected direction against the linearized
    conditions: rows 0, 1, 3-6 of Eq. first scale by (1 - eps), the
    constraint row moves by -eps c_soc (c_sign = -1 plants a sign mistake)."""
    g = synth.workload_grid("30bus-opf")
    L = oracle.layout(g)
    st = ipm_start(g, IpmOptions())
    b = {k: st[k] for k in ("xl", "xu", "sl", "su")}
    rng = np.random.default_rng(1)
    x, s = st["x"], st["s"]
    y = rng.standard_normal(L.m) * 0.1
    z = {k: st[k] * (1 + rng.random(st[k].size)) for k in ("zl_x", "zu_x", "zl_s", "zu_s")}
    mu = 0.1
    F0 = _conditions(g, b, x, s, y, z, mu)
    J = oracle.jacobian(g, x)[0]
    it = oracle.Iterate(x=x, s=s, **b, **z, p_x=-F0[0], p_s=-F0[1], p_y=-F0[2], p_zl_x=-F0[3],
                        p_zu_x=-F0[4], p_zl_s=-F0[5], p_zu_s=-F0[6])
    H = oracle.hessian(g, x, -y, 1.0)[0]
    c = oracle.condense(g, J, it, 0.0, 0.0)
    kv, _ = oracle.condensed_kkt(g, H, J, c["sigma_x"][0], c["sigma_s"][0], 0.0, 0.0)
    c_soc = 0.7 * F0[2] + 0.05 * rng.standard_normal(L.m) * np.max(np.abs(F0[2]))
    d = oracle.second_order_correction(g, J, it, kv, 0.0, c_sign * c_soc)
    eps = 1e-7
    z1 = {k: z[k] + eps * d["d" + k] for k in z}
    F1 = _conditions(g, b, x + eps * d["dx"], s + eps * d["ds"], y + eps * d["dy"], z1, mu)
    err = []
    for i in range(7):
        want = F0[i] - eps * (c_soc if i == 2 else F0[i])
        scale = np.max(np.abs(c_soc if i == 2 else F0[i]))
        err.append(np.max(np.abs(F1[i] - want)) / (eps * scale))
    return err


def test_second_order_correction_solves_the_corrected_linearization():
    err = _soc_check(1.0)
    assert max(err) < 1e-3, err


def test_opposite_sign_of_the_correction_fails():
    err = _soc_check(-1.0)
    assert err[2] > 0.1, err


def test_corrected_step_taken_and_solution_unchanged():
    g = synth.make_edge_case_grid(7)
    g = dataclasses.replace(g, Pd=g.Pd * 0.5, Qd=g.Qd * 0.5)
    r = oracle.ipm_solve(g, IpmOptions(tol=1e-4))
    assert r.status == "converged", r.status
    assert sum(h.get("soc", 0) for h in r.history) >= 1
    # the same point (to the tolerance) as without corrections
    r0 = oracle.ipm_solve(g, IpmOptions(tol=1e-4, soc_max=0))
    assert r0.status == "converged"
    assert abs(r.objective - r0.objective) <= 1e-4 * abs(r0.objective)
    assert np.max(np.abs(r.x - r0.x)) <= 1e-2


def test_newton_step_solves_the_linearized_conditions():
    err = _newton_check(-1.0)
    assert max(err) < 1e-3, err


def test_opposite_reading_of_delta_y_fails():
    err = _newton_check(+1.0)
    assert max(err[:2]) > 0.1, err


def test_solution_matches_an_independent_solver():
    """SLSQP (scipy) on the same problem from the same start; the oracle at
    tol 1e-6 (its relaxation of the equality rows moves the optimum by
    O(tol))."""
    from scipy.optimize import minimize
    g = synth.workload_grid("30bus-opf")
    r = oracle.ipm_solve(g, IpmOptions(tol=1e-6))
    assert r.status == "converged"
    xl, xu, gl, gu = oracle.bounds(g)
    x0 = ipm_start(g, IpmOptions())["x"]
    A = lambda x: oracle.acopf._jac_matrix(g, oracle.jacobian(g, x)[0]).toarray()  # noqa: E731
    eq = np.flatnonzero(gl == gu)
    lo = np.flatnonzero(np.isfinite(gl) & (gl != gu))
    hi = np.flatnonzero(np.isfinite(gu) & (gl != gu))
    cons = [dict(type="eq", fun=lambda x: oracle.constraints(g, x)[0][eq], jac=lambda x: A(x)[eq]),
            dict(type="ineq", fun=lambda x: oracle.constraints(g, x)[0][lo] - gl[lo],
                 jac=lambda x: A(x)[lo]),
            dict(type="ineq", fun=lambda x: gu[hi] - oracle.constraints(g, x)[0][hi],
                 jac=lambda x: -A(x)[hi])]
    bnds = [(a if np.isfinite(a) else None, b if np.isfinite(b) else None) for a, b in zip(xl, xu)]
    s = minimize(lambda x: oracle.objective(g, x)[0], x0, jac=lambda x: oracle.gradient(g, x)[0],
                 bounds=bnds, constraints=cons, method="SLSQP",
                 options=dict(maxiter=1000, ftol=1e-12))
    assert s.success
    assert abs(r.objective - s.fun) <= 1e-4 * abs(s.fun), (r.objective, s.fun)


def test_solution_is_interior_and_nearly_feasible():
    g = synth.workload_grid("30bus-opf")
    opts = IpmOptions()
    r = oracle.ipm_solve(g, opts)
    assert r.status == "converged" and r.residual <= opts.tol
    xl, xu, gl, gu = oracle.bounds(g)
    fx, fu = np.isfinite(xl), np.isfinite(xu)
    assert np.all(r.x[fx] > xl[fx]) and np.all(r.x[fu] < xu[fu])
    c = oracle.constraints(g, r.x)[0]
    sl, su = oracle.relaxed_bounds(gl, gu, opts.tol)
    viol = np.maximum(0.0, np.maximum(sl - c, c - su))
    assert viol.max() <= opts.tol


def test_initial_point_and_step_rules_by_hand():
    # push: one-sided bound moves by k1 max(1,|b|); a narrow box by k2 of its width
    assert push_interior(np.array([0.0]), np.array([0.0]), np.array([np.inf]), 1e-2, 1e-2)[0] == 1e-2
    assert push_interior(np.array([5.0]), np.array([-np.inf]), np.array([2.0]), 1e-2, 1e-2)[0] == 2.0 - 2e-2
    v = push_interior(np.array([0.0]), np.array([0.0]), np.array([1e-3]), 1e-2, 1e-2)[0]
    assert v == 1e-5
    # fraction to boundary: x = 1 in [0, 2], dx = -2, tau = 0.99 -> alpha = 0.495
    a = fraction_to_boundary(np.array([1.0]), np.array([-2.0]), np.array([0.0]), np.array([2.0]),
                             0.99)
    assert abs(a - 0.495) < 1e-15
    assert fraction_to_boundary(np.array([1.0]), np.array([0.1]), np.array([0.0]),
                                np.array([2.0]), 0.99) == 1.0


def _scaled_30bus(scale):
    g = synth.workload_grid("30bus")
    return dataclasses.replace(g, Pd=g.Pd * scale, Qd=g.Qd * scale)


def _violation_l1(g, x, tol=1e-4):
    from oracle.ipm import relaxed_bounds
    _, _, gl, gu = oracle.bounds(g)
    sl, su = relaxed_bounds(gl, gu, tol)
    c = oracle.constraints(g, x)[0]
    return float(np.sum(np.abs(c - np.clip(c, sl, su))))


def _least_violation(g, starts=2, tol=1e-4):
    """The smallest L1 constraint violation (against the relaxed bounds, x
    within its bounds) scipy's least_squares reaches from random starts."""
    from scipy.optimize import least_squares

    from oracle.ipm import relaxed_bounds
    L = oracle.layout(g)
    xl, xu, gl, gu = oracle.bounds(g)
    sl, su = relaxed_bounds(gl, gu, tol)
    jr, jc = oracle.jac_structure(g)

    def resid(x):
        c = oracle.constraints(g, x)[0]
        return c - np.clip(c, sl, su)

    def jac(x):
        c = oracle.constraints(g, x)[0]
        outside = ((c < sl) | (c > su)).astype(float)
        A = sp.csr_matrix((oracle.jacobian(g, x)[0], (jr, jc)), shape=(L.m, L.n))
        return (sp.diags(outside) @ A).toarray()

    lb = np.where(np.isfinite(xl), xl, -np.inf)
    ub = np.where(np.isfinite(xu), xu, np.inf)
    best = np.inf
    for t in range(starts):
        x0 = np.clip(synth.make_point(g, 200 + t).x, lb + 1e-9, ub - 1e-9)
        r = least_squares(resid, x0, jac=jac, bounds=(lb, ub), method="trf", max_nfev=500,
                          xtol=1e-15, ftol=1e-15, gtol=1e-15)
        best = min(best, float(np.sum(np.abs(resid(r.x)))))
    return best


@pytest.mark.parametrize("scale", [0.8, 1.0])
def test_restoration_stops_at_the_least_violation_when_infeasible(scale):
    g = _scaled_30bus(scale)
    r = oracle.ipm_solve(g, IpmOptions())
    assert r.status == "infeasible", r.status
    assert any(h.get("restoration") for h in r.history)
    least = _least_violation(g)
    assert least > 0.1  # no feasible point: the pin's premise
    assert abs(_violation_l1(g, r.x) - least) <= 5e-3 * least, (_violation_l1(g, r.x), least)


def test_feasible_load_converges():
    g = _scaled_30bus(0.6)
    assert _least_violation(g, starts=1) < 1e-8  # a feasible point exists
    r = oracle.ipm_solve(g, IpmOptions())
    assert r.status == "converged"


def test_pin_catches_restoration_that_gives_up_early(monkeypatch):
    """A restoration stopping at its first stall (no smaller barrier) leaves
    a larger violation than the least one: the pin above fails."""
    import oracle.ipm as ipm_mod
    real = ipm_mod.restoration

    def early(grid, x, b, mu, accept, opts):
        return real(grid, x, b, mu, accept, dataclasses.replace(opts, resto_mu_min=1e30))

    monkeypatch.setattr(ipm_mod, "restoration", early)
    g = _scaled_30bus(1.0)
    r = oracle.ipm_solve(g, IpmOptions())
    least = _least_violation(g)
    assert r.status != "infeasible" or abs(_violation_l1(g, r.x) - least) > 5e-3 * least
