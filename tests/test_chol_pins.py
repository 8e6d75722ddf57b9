"""Pins of the M_cond solve / positive-definiteness oracle (oracle/chol.py).

* Sylvester's law of inertia (Sec. IV.C): the printed M_aug, assembled
  densely block by block, has the inertia (n + m, 0, m) exactly when M_cond
  is positive definite, and in general M_aug has m more negative eigenvalues
  than M_cond.  Checked on a convex case (no constraint multipliers, so W is
  the objective's Hessian, positive semidefinite, and delta_w > 0) and on a
  nonconvex one.
* The solve equals a dense solve of W + delta_w I + Sigma_x + A' D A built
  from the dense Hessian and Jacobian, not from the assembled values.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
from paper_2307_16830_gb300 import synth


def _dense(grid, hvals, jvals):
    L = oracle.layout(grid)
    r, c = oracle.hess_structure(grid)
    Wl = sp.coo_matrix((hvals, (r, c)), shape=(L.n, L.n)).toarray()
    W = Wl + Wl.T - np.diag(np.diag(Wl))
    r, c = oracle.jac_structure(grid)
    A = sp.coo_matrix((jvals, (r, c)), shape=(L.m, L.n)).toarray()
    return W, A


def _inertia(M, tol=1e-13):
    """(positive, zero, negative) counts of a symmetric matrix: the
    eigenvalues of the block-diagonal factor of a Bunch-Kaufman LDL'
    (Sylvester: congruent matrices share their inertia)."""
    _, d, _ = scipy.linalg.ldl(M)
    ev = np.linalg.eigvalsh(d)
    t = tol * np.max(np.abs(ev))
    return int(np.sum(ev > t)), int(np.sum(np.abs(ev) <= t)), int(np.sum(ev < -t))


def _case(y_scale, dw, dc, seed):
    g = synth.workload_grid("30bus")
    L = oracle.layout(g)
    pt = synth.make_point(g, seed)
    y = pt.y * y_scale
    J = oracle.jacobian(g, pt.x)[0]
    H = oracle.hessian(g, pt.x, y, 1.0)[0]
    xl, xu, gl, gu = oracle.bounds(g)
    it = oracle.Iterate(**synth.make_iterate(xl, xu, gl, gu, seed))
    c = oracle.condense(g, J, it, dw, dc)
    sx, ss = c["sigma_x"][0], c["sigma_s"][0]
    kv, _ = oracle.condensed_kkt(g, H, J, sx, ss, dw, dc)
    W, A = _dense(g, H, J)
    M_aug = np.block([
        [W + np.diag(sx) + dw * np.eye(L.n), np.zeros((L.n, L.m)), A.T],
        [np.zeros((L.m, L.n)), np.diag(ss) + dw * np.eye(L.m), -np.eye(L.m)],
        [A, -np.eye(L.m), -dc * np.eye(L.m)]])
    D = (ss + dw) / (dc * ss + 1.0 + dc * dw)
    M_cond = W + np.diag(sx) + dw * np.eye(L.n) + A.T @ (D[:, None] * A)
    return g, L, kv, M_aug, M_cond


@pytest.mark.parametrize("dc", [0.0, 1e-2])
def test_convex_case_has_the_inertia_of_a_positive_definite_m_cond(dc):
    g, L, kv, M_aug, M_cond = _case(0.0, 1e-3, dc, 31)
    assert _inertia(M_aug) == (L.n + L.m, 0, L.m)
    assert oracle.is_positive_definite(g, kv)
    assert np.linalg.eigvalsh(M_cond)[0] > 0.0


@pytest.mark.parametrize("dc", [0.0, 1e-2])
def test_nonconvex_case_sylvester(dc):
    g, L, kv, M_aug, M_cond = _case(50.0, 0.0, dc, 32)
    pa, za, na = _inertia(M_aug)
    pc, zc, nc = _inertia(M_cond)
    assert nc > 0, "the case must be indefinite"
    assert (pa, za, na) != (L.n + L.m, 0, L.m)
    assert na - L.m == nc and pa - L.m == pc
    assert not oracle.is_positive_definite(g, kv)


def test_solve_matches_a_dense_solve_of_the_printed_matrix():
    g, L, kv, _, M_cond = _case(1.0, 1e-2, 1e-3, 33)
    b = np.random.default_rng(34).standard_normal(L.n)
    x = oracle.solve_condensed(g, kv, b)
    ref = np.linalg.solve(M_cond, b)
    assert np.max(np.abs(x - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert oracle.backward_error(g, kv, x, b) < 1e-14


def test_pin_catches_a_matrix_without_its_upper_triangle(monkeypatch):
    """A plausible mistake (the lower triangle taken as the whole matrix)
    fails the dense-solve pin."""
    import oracle.chol as oc
    orig = oc.condensed_matrix

    def low_only(grid, kvals):
        K = orig(grid, kvals)
        return sp.tril(K).tocsr()

    monkeypatch.setattr(oc, "condensed_matrix", low_only)
    with pytest.raises(AssertionError):
        test_solve_matches_a_dense_solve_of_the_printed_matrix()
