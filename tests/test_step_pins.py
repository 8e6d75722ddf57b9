"""Pins of the condensation / step-recovery oracle (oracle/step.py) against
the Newton system the paper prints (Sec. IV.C), solved directly.

The 7x7 block system M_full [dx, ds, dy, dzl_x, dzu_x, dzl_s, dzu_s] = p is
assembled densely, block by block as printed, on a small network (rows and
columns of bound duals only where the bound is finite) and solved with a
dense LU.  The oracle's route (Sigma, q and the condensed right-hand side,
a solve with the condensed matrix M_cond from the callbacks' oracle, then
the recovery formulas) must give the same step.  The paper's printed
formula for ds, with the opposite sign of A dx, must not.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2307_16830_gb300 import synth


def _dense_w(grid, hvals):
    L = oracle.layout(grid)
    r, c = oracle.hess_structure(grid)
    Wl = sp.coo_matrix((hvals, (r, c)), shape=(L.n, L.n)).toarray()
    return Wl + Wl.T - np.diag(np.diag(Wl))


def _dense_a(grid, jvals):
    L = oracle.layout(grid)
    r, c = oracle.jac_structure(grid)
    return sp.coo_matrix((jvals, (r, c)), shape=(L.m, L.n)).toarray()


def _solve_full(W, A, it, dw, dc):
    """Dense solve of the printed Newton system; returns the step blocks."""
    n, m = A.shape[1], A.shape[0]
    fl_x, fu_x = np.flatnonzero(np.isfinite(it.xl)), np.flatnonzero(np.isfinite(it.xu))
    fl_s, fu_s = np.flatnonzero(np.isfinite(it.sl)), np.flatnonzero(np.isfinite(it.su))
    sizes = [n, m, m, fl_x.size, fu_x.size, fl_s.size, fu_s.size]
    off = np.concatenate([[0], np.cumsum(sizes)])
    N = off[-1]
    M = np.zeros((N, N))
    X, S, Y, ZLX, ZUX, ZLS, ZUS = range(7)

    def blk(i, j):
        return slice(off[i], off[i + 1]), slice(off[j], off[j + 1])

    # row block 1: (W + dw I) dx + A' dy - dzl_x + dzu_x = p_x
    M[blk(X, X)] = W + dw * np.eye(n)
    M[blk(X, Y)] = A.T
    M[off[X] + fl_x, off[ZLX] + np.arange(fl_x.size)] = -1.0
    M[off[X] + fu_x, off[ZUX] + np.arange(fu_x.size)] = 1.0
    # row block 2: dw ds - dy - dzl_s + dzu_s = p_s
    M[blk(S, S)] = dw * np.eye(m)
    M[blk(S, Y)] = -np.eye(m)
    M[off[S] + fl_s, off[ZLS] + np.arange(fl_s.size)] = -1.0
    M[off[S] + fu_s, off[ZUS] + np.arange(fu_s.size)] = 1.0
    # row block 3: A dx - ds - dc dy = p_y
    M[blk(Y, X)] = A
    M[blk(Y, S)] = -np.eye(m)
    M[blk(Y, Y)] = -dc * np.eye(m)
    # complementarity rows
    for blkrow, idx, z, gap, col0, sign in (
            (ZLX, fl_x, it.zl_x, it.x - it.xl, off[X], 1.0),
            (ZUX, fu_x, it.zu_x, it.xu - it.x, off[X], -1.0),
            (ZLS, fl_s, it.zl_s, it.s - it.sl, off[S], 1.0),
            (ZUS, fu_s, it.zu_s, it.su - it.s, off[S], -1.0)):
        rows = off[blkrow] + np.arange(idx.size)
        M[rows, col0 + idx] = sign * z[idx]
        M[rows, rows] = gap[idx]
    rhs = np.concatenate([it.p_x, it.p_s, it.p_y, it.p_zl_x[fl_x], it.p_zu_x[fu_x],
                          it.p_zl_s[fl_s], it.p_zu_s[fu_s]])
    sol = np.linalg.solve(M, rhs)
    parts = [sol[off[i]:off[i + 1]] for i in range(7)]
    full = {}
    full["dx"], full["ds"], full["dy"] = parts[0], parts[1], parts[2]
    for name, idx, k, size in (("dzl_x", fl_x, 3, n), ("dzu_x", fu_x, 4, n),
                               ("dzl_s", fl_s, 5, m), ("dzu_s", fu_s, 6, m)):
        v = np.zeros(size)
        v[idx] = parts[k]
        full[name] = v
    return full


def _condensed_route(grid, W_h, J, it, dw, dc):
    """Oracle route: condense, solve M_cond (dense, from its CSR values), recover."""
    L = oracle.layout(grid)
    c = oracle.condense(grid, J, it, dw, dc)
    kv, _ = oracle.condensed_kkt(grid, W_h, J, c["sigma_x"][0], c["sigma_s"][0], dw, dc)
    rp, ci = oracle.kkt_structure(grid)
    rows = np.repeat(np.arange(L.n), np.diff(rp))
    Kl = sp.coo_matrix((kv, (rows, ci)), shape=(L.n, L.n)).toarray()
    K = Kl + Kl.T - np.diag(np.diag(Kl))
    dx = np.linalg.solve(K, c["rhs"][0])
    r = oracle.recover(grid, J, it, dx, dw, dc)
    out = {k: v[0] for k, v in r.items()}
    out["dx"] = dx
    return out, c


def _case(seed):
    g = synth.workload_grid("30bus")
    pt = synth.make_point(g, seed)
    J = oracle.jacobian(g, pt.x)[0]
    H = oracle.hessian(g, pt.x, pt.y, 1.0)[0]
    xl, xu, gl, gu = oracle.bounds(g)
    it = oracle.Iterate(**synth.make_iterate(xl, xu, gl, gu, seed, z_range=(-1.0, 0.5),
                                             gap_floor=0.05))
    return g, J, H, it


@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (0.3, 0.0), (0.5, 0.02)])
def test_condensed_route_solves_the_printed_newton_system(dw, dc):
    g, J, H, it = _case(11)
    full = _solve_full(_dense_w(g, H), _dense_a(g, J), it, dw, dc)
    route, _ = _condensed_route(g, H, J, it, dw, dc)
    for k in ("dx", "ds", "dy", "dzl_x", "dzu_x", "dzl_s", "dzu_s"):
        a, b = route[k], full[k]
        scale = np.max(np.abs(b)) + 1e-300
        assert np.max(np.abs(a - b)) <= 1e-7 * scale, (k, np.max(np.abs(a - b)) / scale)


def test_printed_ds_sign_does_not_solve_the_system():
    """Sec. IV.C prints ds = C (delta_c q_s - (q_y + A dx)); with the printed
    M_aug the recovered ds must carry +A dx (the oracle's reading)."""
    dw, dc = 0.3, 0.02
    g, J, H, it = _case(12)
    full = _solve_full(_dense_w(g, H), _dense_a(g, J), it, dw, dc)
    route, c = _condensed_route(g, H, J, it, dw, dc)
    A = _dense_a(g, J)
    ss, qs = c["sigma_s"][0], c["q_s"][0]
    C = 1.0 / (dc * ss + 1.0 + dc * dw)
    printed = C * (dc * qs - (it.p_y + A @ route["dx"]))
    scale = np.max(np.abs(full["ds"]))
    assert np.max(np.abs(route["ds"] - full["ds"])) <= 1e-7 * scale
    assert np.max(np.abs(printed - full["ds"])) > 1e-3 * scale


def test_infinite_bounds_carry_no_terms():
    """A component whose bounds are both infinite has Sigma = 0, q = p and
    zero bound-dual steps (va is free in the model)."""
    g, J, H, it = _case(13)
    L = oracle.layout(g)
    c = oracle.condense(g, J, it)
    free = np.arange(L.VA, L.VA + L.nb)
    assert np.all(c["sigma_x"][0][free] == 0.0)
    r = oracle.recover(g, J, it, np.ones(L.n))
    assert np.all(r["dzl_x"][0][free] == 0.0) and np.all(r["dzu_x"][0][free] == 0.0)


def test_pin_catches_planted_mistakes(monkeypatch):
    """The direct-solve pin fails when the oracle carries a plausible mistake:
    a wrong sign of the upper-bound term of q, or of a bound-dual step."""
    import oracle.step as st
    orig_block, orig_recover = st._block, st.recover

    def bad_block(v, lo, hi, zl, zu, p, pl, pu):
        il, iu = st.inv_gap(v, lo, hi)
        sig = zl * il + zu * iu
        q = p + il * pl + iu * pu
        return sig, np.abs(sig), q, np.abs(q)

    monkeypatch.setattr(st, "_block", bad_block)
    with pytest.raises(AssertionError):
        test_condensed_route_solves_the_printed_newton_system(0.3, 0.0)
    monkeypatch.setattr(st, "_block", orig_block)

    def bad_recover(*a, **k):
        r = dict(orig_recover(*a, **k))
        r["dzu_s"] = (-r["dzu_s"][0], r["dzu_s"][1])
        return r

    monkeypatch.setattr(oracle, "recover", bad_recover)
    with pytest.raises(AssertionError):
        test_condensed_route_solves_the_printed_newton_system(0.3, 0.0)


def test_dual_residual_is_the_gradient_of_the_lagrangian():
    """r_d = [grad f - A'y - zl_x + zu_x ; y - zl_s + zu_s] is the gradient in
    (x, s) of L = f(x) - y'(g(x) - s) - zl_x'(x - xl) - zu_x'(xu - x)
    - zl_s'(s - sl) - zu_s'(su - s) (finite bounds only), checked by central
    differences of L built from the objective and constraint values alone."""
    g = synth.workload_grid("30bus")
    L = oracle.layout(g)
    xl, xu, gl, gu = oracle.bounds(g)
    it = oracle.Iterate(**synth.make_iterate(xl, xu, gl, gu, 21))
    y = np.random.default_rng(22).standard_normal(L.m)
    fx = lambda v: np.where(np.isfinite(v), v, 0.0)  # noqa: E731

    def lagr(x, s):
        val = oracle.objective(g, x)[0] - y @ (oracle.constraints(g, x)[0] - s)
        val -= it.zl_x @ (fx(x - it.xl)) + it.zu_x @ (fx(it.xu - x))
        val -= it.zl_s @ (fx(s - it.sl)) + it.zu_s @ (fx(it.su - s))
        return val

    rdx, rds, _, _, _ = oracle.kkt_parts(g, oracle.gradient(g, it.x)[0],
                                         oracle.constraints(g, it.x)[0],
                                         oracle.jacobian(g, it.x)[0], it, y, 0.1)
    h = 1e-6
    for j in np.random.default_rng(23).choice(L.n, 40, replace=False):
        e = np.zeros(L.n)
        e[j] = h * max(1.0, abs(it.x[j]))
        fd = (lagr(it.x + e, it.s) - lagr(it.x - e, it.s)) / (2 * e[j])
        assert abs(fd - rdx[j]) <= 1e-5 * max(1.0, abs(rdx[j])), (j, fd, rdx[j])
    for r in np.random.default_rng(24).choice(L.m, 40, replace=False):
        e = np.zeros(L.m)
        e[r] = h * max(1.0, abs(it.s[r]))
        fd = (lagr(it.x, it.s + e) - lagr(it.x, it.s - e)) / (2 * e[r])
        assert abs(fd - rds[r]) <= 1e-5 * max(1.0, abs(rds[r])), (r, fd, rds[r])


def test_residual_scaling_golden():
    """s_d, s_c by hand (s_max = 100): small multipliers leave the residual
    unscaled; large ones divide it by their mean magnitude / 100."""
    assert oracle.residual_scaling(3.0, 7.0, 2, 2) == (1.0, 1.0)
    s_d, s_c = oracle.residual_scaling(3e4, 7e4, 2, 2)
    assert s_d == 250.0 and s_c == 350.0
