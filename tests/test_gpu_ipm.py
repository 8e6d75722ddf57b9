"""GPU interior-point method (acopf_ipm_solve) against the oracle's
(oracle.ipm_solve): the same algorithm, the same decisions.

At tol = 1e-4 (the paper's default for the condensed method) on networks
both solve: the same status and iteration count, per-iteration objective,
residual, barrier parameter, violation and step sizes within 1e-4
relative, the final objective within 1e-8 relative and x within 1e-4; on
networks without a feasible point (the 30-bus network at 0.8 and 1.0 times
its loads), the same restorations and the same "infeasible" stop at the same
iteration, at a point of the same violation.  The half-loaded edge case
and the 0.8 and 1.0 loads take second-order corrections (asserted on the
oracle's history), so the same decisions cover them too.  The 1e-4: the slack boxes of the equality rows are 2e-4 wide
and the gaps shrink with mu, so Sigma reaches 1e8-1e10 late in a solve;
M_cond's condition number times the double-precision unit roundoff then
bounds the relative difference of two correct steps computed in different
summation orders at 1e-6-1e-5 (measured up to 1.1e-5); the step sizes and
the next iterates inherit it.  At tol = 1e-6 the equality rows' slack boxes are 2e-6 wide, so
Sigma_s reaches 1e8 and M_cond's condition number amplifies rounding-level
differences of the two implementations (a different summation order) into
relative step differences of about 1e-4: there the two must converge to the
same point (objective within 1e-7 relative, x within 1e-4) in iteration
counts at most 2 apart."""
import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def _scaled(g, scale):
    import dataclasses
    return dataclasses.replace(g, Pd=g.Pd * scale, Qd=g.Qd * scale)


def _half_load(g):
    return _scaled(g, 0.5)


STATUS = {"converged": 0, "max_iter": 1, "line search failed": 2, "inertia correction failed": 3,
          "infeasible": 4}


@pytest.fixture(scope="module")
def acopf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_16830_gb300 import acopf as lib
    return lib


CASES = [("30bus-opf", lambda: synth.workload_grid("30bus-opf"), 1e-4),
         ("edge7", lambda: _half_load(synth.make_edge_case_grid(7)), 1e-4),
         ("random500", lambda: synth.make_grid(500, 675, 100, seed=21, load_scale=0.1), 1e-4),
         ("geo300", lambda: synth.make_grid(300, 405, 60, seed=1011, topology="geometric",
                                            load_scale=0.1), 1e-4),
         ("30bus 0.8 load", lambda: _scaled(synth.workload_grid("30bus"), 0.8), 1e-4),
         ("30bus full load", lambda: synth.workload_grid("30bus"), 1e-4)]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_ipm_matches_oracle(acopf, idx):
    name, make, tol = CASES[idx]
    g = make()
    ref = oracle.ipm_solve(g, oracle.IpmOptions(tol=tol))
    with acopf.model_create(g, 0) as m:
        res, x, hist = acopf.ipm_solve(m, tol=tol, max_iter=200)
    assert res["status"] == STATUS[ref.status], (name, res, ref.status)
    assert res["iterations"] == ref.iterations, (name, res["iterations"], ref.iterations)
    if name in ("edge7", "30bus 0.8 load", "30bus full load"):  # cases that take corrected steps
        assert sum(h.get("soc", 0) for h in ref.history) >= 1, name
    for k, h in enumerate(ref.history):
        for j, key in enumerate(("f", "residual", "mu", "theta", "alpha", "alpha_z", "delta_w")):
            if key not in h:
                continue
            a, b = hist[k, j], h[key]
            assert abs(a - b) <= 1e-4 * max(1.0, abs(b)), (name, k, key, a, b)
    if ref.status == "converged":
        assert abs(res["objective"] - ref.objective) <= 1e-8 * abs(ref.objective)
        assert np.max(np.abs(x - ref.x)) <= 1e-4
        assert res["residual"] <= tol
    if ref.status == "infeasible":  # stopped at a point of the same violation
        from oracle.ipm import relaxed_bounds
        _, _, gl, gu = oracle.bounds(g)
        sl, su = relaxed_bounds(gl, gu, tol)
        viol = lambda v: float(np.sum(np.abs(v - np.clip(v, sl, su))))  # noqa: E731
        a, b = viol(oracle.constraints(g, x)[0]), viol(oracle.constraints(g, ref.x)[0])
        assert abs(a - b) <= 1e-3 * b, (name, a, b)


def test_ipm_tight_tolerance_reaches_the_same_point(acopf):
    g = synth.workload_grid("30bus-opf")
    ref = oracle.ipm_solve(g, oracle.IpmOptions(tol=1e-6))
    with acopf.model_create(g, 0) as m:
        res, x, _ = acopf.ipm_solve(m, tol=1e-6, max_iter=200)
    assert ref.status == "converged" and res["status"] == acopf.IPM_CONVERGED
    assert abs(res["iterations"] - ref.iterations) <= 2
    assert abs(res["objective"] - ref.objective) <= 1e-7 * abs(ref.objective)
    assert np.max(np.abs(x - ref.x)) <= 1e-4


def test_ipm_rejects_bad_arguments(acopf):
    g = synth.workload_grid("30bus-opf")
    with acopf.model_create(g, 0) as m:
        for kw in (dict(tol=0.0), dict(mu_init=-1.0), dict(max_iter=-1)):
            with pytest.raises(acopf.AcopfError) as e:
                acopf.ipm_solve(m, **kw)
            assert e.value.status == acopf.E_INVALID_ARG


def test_ipm_with_a_kept_cholesky_object_reproduces_the_solve(acopf):
    """acopf_ipm_solve_chol: the caller's Cholesky object, kept over two
    solves, gives the plain solve's iterates bit for bit, without the
    symbolic phase in the setup; another model's object is refused."""
    g = synth.workload_grid("10kbus-geo-opf")
    with acopf.model_create(g, 0) as m:
        r0, x0, h0 = acopf.ipm_solve(m, tol=1e-4, max_iter=200)
        ch = acopf.chol_create(m)
        try:
            runs = [acopf.ipm_solve(m, tol=1e-4, max_iter=200, chol=ch) for _ in range(2)]
        finally:
            ch.close()
    assert r0["status"] == acopf.IPM_CONVERGED
    for r, x, h in runs:
        assert (r["status"], r["iterations"]) == (r0["status"], r0["iterations"])
        assert np.array_equal(x, x0)
        assert np.array_equal(np.nan_to_num(h, nan=-1.0), np.nan_to_num(h0, nan=-1.0))
        assert r["objective"] == r0["objective"]
    assert runs[1][0]["setup_seconds"] < r0["setup_seconds"], (runs[1][0], r0)
    g30 = synth.workload_grid("30bus-opf")
    with acopf.model_create(g30, 0) as a, acopf.model_create(g30, 0) as b:
        ch = acopf.chol_create(a)
        try:
            with pytest.raises(acopf.AcopfError) as e:
                acopf.ipm_solve(b, chol=ch)
            assert e.value.status == acopf.E_INVALID_ARG
        finally:
            ch.close()


def test_ipm_10k_near_planar_matches_oracle(acopf):
    """The 10,000-bus near-planar short-line network: both converge to the
    same point (objective within 1e-7 relative, x within 1e-4) in iteration
    counts at most 2 apart."""
    g = synth.workload_grid("10kbus-geo-opf")
    ref = oracle.ipm_solve(g)
    with acopf.model_create(g, 0) as m:
        res, x, _ = acopf.ipm_solve(m)
    assert ref.status == "converged" and res["status"] == acopf.IPM_CONVERGED, res
    assert abs(res["iterations"] - ref.iterations) <= 2
    assert abs(res["objective"] - ref.objective) <= 1e-7 * abs(ref.objective)
    assert np.max(np.abs(x - ref.x)) <= 1e-4


def test_ipm_80k_solution_properties(acopf):
    """The 80,000-bus near-planar short-line network (too large for the
    oracle's solve): the returned point is converged, strictly inside its
    bounds, within tol of the relaxed constraints, and the oracle's objective
    there equals the reported one."""
    g = synth.workload_grid("80kbus-geo-opf")
    tol = 1e-4
    with acopf.model_create(g, 0) as m:
        res, x, _ = acopf.ipm_solve(m, tol=tol)
    assert res["status"] == acopf.IPM_CONVERGED and res["residual"] <= tol, res
    xl, xu, gl, gu = oracle.bounds(g)
    fx, fu = np.isfinite(xl), np.isfinite(xu)
    assert np.all(x[fx] > xl[fx]) and np.all(x[fu] < xu[fu])
    c = oracle.constraints(g, x)[0]
    sl, su = oracle.relaxed_bounds(gl, gu, tol)
    assert np.max(np.maximum(0.0, np.maximum(sl - c, c - su))) <= tol
    f = oracle.objective(g, x)[0]
    assert abs(f - res["objective"]) <= 1e-10 * abs(f)
