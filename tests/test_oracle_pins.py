"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

None of these retype the oracle's own formulas: flows are checked against the
complex-phasor form of the textbook pi-model, derivatives against central
finite differences, the condensed matrix against a dense Schur complement of
the augmented system of Sec. IV.C, sizes against Table II, and the 2-bus case
against hand-derived closed forms (tests/golden/).  The mutation tests at the
end plant typical mistakes in the oracle and check that a pin catches them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2307_16830_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def small_grids():
    return [synth.workload_grid("30bus"), synth.make_edge_case_grid(7)]


def two_bus_grid():
    g = synth.Grid(
        bus_type=np.array([3, 1], np.int32), Pd=np.array([0.5, 0.8]),
        Qd=np.array([0.15, 0.24]), Gs=np.array([0.1, 0.0]), Bs=np.array([0.0, 0.2]),
        Vmin=np.array([0.9, 0.9]), Vmax=np.array([1.1, 1.1]),
        f=np.array([0], np.int32), t=np.array([1], np.int32), r=np.array([0.0]),
        x=np.array([0.5]), b=np.array([0.2]), tap=np.array([1.0]), shift=np.array([0.0]),
        rate_a=np.array([3.0]), angmin=np.array([-math.pi / 6]), angmax=np.array([math.pi / 6]),
        gen_bus=np.array([0], np.int32), Pmin=np.array([0.0]), Pmax=np.array([3.0]),
        Qmin=np.array([-1.5]), Qmax=np.array([1.5]), c2=np.array([0.5]),
        c1=np.array([10.0]), c0=np.array([1.0]), name="two-bus")
    x = np.array([math.pi / 6, 0.0, 1.0, 1.0, 2.0, 0.5, 0.9, -1.1, 0.2, 0.3])
    return g, x


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    return out


def dense_jac(grid, x):
    L = oracle.layout(grid)
    r, c = oracle.jac_structure(grid)
    v, _ = oracle.jacobian(grid, x)
    return sp.csr_matrix((v, (r, c)), shape=(L.m, L.n)).toarray()


def dense_hess(grid, x, y, sigma):
    L = oracle.layout(grid)
    r, c = oracle.hess_structure(grid)
    v, _ = oracle.hessian(grid, x, y, sigma)
    H = sp.csr_matrix((v, (r, c)), shape=(L.n, L.n)).toarray()
    return H + H.T - np.diag(np.diag(H))


def fd_jacobian(grid, x):
    """Central differences of the oracle's constraint function, column by column."""
    L = oracle.layout(grid)
    Jfd = np.zeros((L.m, L.n))
    for j in range(L.n):
        h = 1e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        Jfd[:, j] = (oracle.constraints(grid, xp)[0] - oracle.constraints(grid, xm)[0]) / (2 * h)
    return Jfd


def lagrangian_gradient(grid, x, y, sigma):
    return sigma * oracle.gradient(grid, x)[0] + dense_jac(grid, x).T @ y


def fd_hessian(grid, x, y, sigma):
    L = oracle.layout(grid)
    Hfd = np.zeros((L.n, L.n))
    for j in range(L.n):
        h = 1e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        Hfd[:, j] = (lagrangian_gradient(grid, xp, y, sigma)
                     - lagrangian_gradient(grid, xm, y, sigma)) / (2 * h)
    return Hfd


def phasor_flows(grid, x):
    """P_f, Q_f, P_t, Q_t from complex arithmetic: S_f = V_f conj(I_f),
    I_f = Y_ff V_f + Y_ft V_t, I_t = Y_tf V_f + Y_tt V_t with the pi-model
    Y_ff = (y + jb/2)/|T|^2, Y_ft = -y/conj(T), Y_tf = -y/T, Y_tt = y + jb/2."""
    L = oracle.layout(grid)
    va = x[L.VA:L.VA + L.nb]
    vm = x[L.VM:L.VM + L.nb]
    V = vm * np.exp(1j * va)
    y = 1.0 / (grid.r + 1j * grid.x)
    tau = np.where(grid.tap == 0, 1.0, grid.tap)
    T = tau * np.exp(1j * grid.shift)
    Yff = (y + 0.5j * grid.b) / np.abs(T) ** 2
    Yft = -y / np.conj(T)
    Ytf = -y / T
    Ytt = y + 0.5j * grid.b
    Vf, Vt = V[grid.f], V[grid.t]
    Sf = Vf * np.conj(Yff * Vf + Yft * Vt)
    St = Vt * np.conj(Ytf * Vf + Ytt * Vt)
    return Sf.real, Sf.imag, St.real, St.imag


def oracle_flows(grid, x):
    L = oracle.layout(grid)
    g, _ = oracle.constraints(grid, x)
    nl = L.nl
    p, q = x[L.P:L.P + 2 * nl], x[L.Q:L.Q + 2 * nl]
    return (p[:nl] - g[L.PF:L.PF + nl], q[:nl] - g[L.QF:L.QF + nl],
            p[nl:] - g[L.PT:L.PT + nl], q[nl:] - g[L.QT:L.QT + nl])


def flows_vs_phasor_err(grid, x):
    err = 0.0
    for a, b in zip(oracle_flows(grid, x), phasor_flows(grid, x)):
        err = max(err, float(np.max(np.abs(a - b) / (1.0 + np.abs(b)))))
    return err


def jac_vs_fd_err(grid, x):
    J = dense_jac(grid, x)
    Jfd = fd_jacobian(grid, x)
    return float(np.max(np.abs(J - Jfd) / (1.0 + np.abs(Jfd))))


def hess_vs_fd_err(grid, x, y, sigma):
    H = dense_hess(grid, x, y, sigma)
    Hfd = fd_hessian(grid, x, y, sigma)
    Hfd = 0.5 * (Hfd + Hfd.T)
    return float(np.max(np.abs(H - Hfd) / (1.0 + np.abs(Hfd))))


def schur_condensed(grid, x, y, sigma, sig_x, sig_s, dw, dc):
    """Eliminate (ds, dy) from the dense augmented matrix of Sec. IV.C,
    M_aug = [[W + Sx + dw I, 0, A'], [0, Ss + dw I, -I], [A, -I, -dc I]],
    by a dense linear solve (Schur complement onto the x block)."""
    L = oracle.layout(grid)
    n, m = L.n, L.m
    W = dense_hess(grid, x, y, sigma)
    A = dense_jac(grid, x)
    M11 = W + np.diag(sig_x + dw)
    M12 = np.zeros((n, 2 * m))
    M12[:, m:] = A.T
    M22 = np.zeros((2 * m, 2 * m))
    M22[:m, :m] = np.diag(sig_s + dw)
    M22[:m, m:] = -np.eye(m)
    M22[m:, :m] = -np.eye(m)
    M22[m:, m:] = -dc * np.eye(m)
    return M11 - M12 @ np.linalg.solve(M22, M12.T)


def kkt_dense_from_oracle(grid, x, y, sigma, sig_x, sig_s, dw, dc):
    L = oracle.layout(grid)
    hv, hm = oracle.hessian(grid, x, y, sigma)
    jv, jm = oracle.jacobian(grid, x)
    kv, km = oracle.condensed_kkt(grid, hv, jv, sig_x, sig_s, dw, dc, hmag=hm, jmag=jm)
    rowptr, colind = oracle.kkt_structure(grid)
    rows = np.repeat(np.arange(L.n), np.diff(rowptr))
    K = np.zeros((L.n, L.n))
    KM = np.zeros((L.n, L.n))
    K[rows, colind] = kv
    KM[rows, colind] = km
    K = K + K.T - np.diag(np.diag(K))
    KM = KM + KM.T - np.diag(np.diag(KM))
    return K, KM


def kkt_vs_schur_err(grid, pt, dw, dc):
    x, y = pt.x, pt.y
    K, KM = kkt_dense_from_oracle(grid, x, y, 1.0, pt.sigma_x, pt.sigma_s, dw, dc)
    S = schur_condensed(grid, x, y, 1.0, pt.sigma_x, pt.sigma_s, dw, dc)
    return float(np.max(np.abs(K - S) / (KM + 1e-300)))


def moderate_point(grid, seed):
    pt = synth.make_point(grid, seed)
    rng = np.random.default_rng(seed + 1)
    pt.sigma_x = 10.0 ** rng.uniform(-2, 2, pt.sigma_x.size)
    pt.sigma_s = 10.0 ** rng.uniform(-2, 2, pt.sigma_s.size)
    return pt


# ---------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------
def test_layout_sizes_match_formulas():
    for g in small_grids():
        L = oracle.layout(g)
        assert L.n == 2 * g.n_bus + 2 * g.n_gen + 4 * g.n_branch
        assert L.m == g.n_ref + 7 * g.n_branch + 2 * g.n_bus
        r, c = oracle.jac_structure(g)
        assert r.size == g.n_ref + 30 * g.n_branch + 2 * g.n_bus + 2 * g.n_gen
        hr, hc = oracle.hess_structure(g)
        assert hr.size == 14 * g.n_branch + g.n_gen + g.n_bus
        assert np.all(hr >= hc)


def _table2_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table2_sizes.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, nb, nv, nc = line.split()
                rows.append((name, int(nb), float(nv) * 1e3, float(nc) * 1e3))
    return rows


def _table2_feasible(nb, nv, nc, n_of, m_of):
    """Is there (N_branch, N_gen) reproducing both printed sizes to +-50?"""
    for nl in range(nb - 1, 6 * nb):
        if abs(m_of(nb, nl) - nc) > 50:
            continue
        for ng in range(1, nb + 1):
            if abs(n_of(nb, ng, nl) - nv) <= 50:
                return True
    return False


def test_table2_sizes_consistent_with_formulation():
    """Table II: every case's nvars/ncons admit integer branch/generator counts
    under this formulation's size formulas (n = 2Nb + 2Ng + 4Nl,
    m = 1 + 7Nl + 2Nb), while a formulation without branch-flow variables
    (n = 2Nb + 2Ng, m = 1 + 2Nl(thermal) + Nl(angle) + 2Nb) does not."""
    rows = _table2_rows()
    assert len(rows) == 25

    def n_of(nb, ng, nl):
        return 2 * nb + 2 * ng + 4 * nl

    def m_of(nb, nl):
        return 1 + 7 * nl + 2 * nb

    for name, nb, nv, nc in rows:
        assert _table2_feasible(nb, nv, nc, n_of, m_of), name

    def n_alt(nb, ng, nl):
        return 2 * nb + 2 * ng

    def m_alt(nb, nl):
        return 1 + 3 * nl + 2 * nb

    assert not all(_table2_feasible(nb, nv, nc, n_alt, m_alt) for _, nb, nv, nc in rows[:17])


def test_flows_match_complex_phasor_form():
    for g in small_grids():
        for seed in range(3):
            x = synth.make_point(g, seed).x
            assert flows_vs_phasor_err(g, x) < 1e-13


def test_dc_flow_limit():
    """Lossless, uncharged, untapped line at flat voltage: P_f -> th / x as th -> 0."""
    g = synth.workload_grid("30bus").copy()
    g.r[:] = 0.0
    g.b[:] = 0.0
    g.tap[:] = 1.0
    L = oracle.layout(g)
    x = synth.make_point(g, 0).x
    x[L.VM:L.VM + L.nb] = 1.0
    th_scale = 1e-4
    x[L.VA:L.VA + L.nb] *= th_scale
    Pf = oracle_flows(g, x)[0]
    th = x[L.VA + g.f] - x[L.VA + g.t]
    dc = th / g.x
    assert np.max(np.abs(Pf - dc)) <= np.max(np.abs(th) ** 3 / g.x)


def test_lossless_invariant():
    """r = 0 and no phase shift: each line is lossless, P_f + P_t = 0, for any tap
    and charging; summed over all arcs the active flows vanish."""
    g = synth.make_edge_case_grid(3)
    g.r[:] = 0.0
    g.shift[:] = 0.0
    for seed in range(3):
        x = synth.make_point(g, seed).x
        Pf, _, Pt, _ = oracle_flows(g, x)
        scale = np.abs(Pf) + np.abs(Pt)
        assert np.all(np.abs(Pf + Pt) <= 1e-14 * (1 + scale))
        assert abs(np.sum(Pf) + np.sum(Pt)) <= 1e-13 * np.sum(scale)


def test_balance_rows_telescope():
    """sum_i Pbal_i = sum Pd + sum Gs vm^2 - sum pg + sum over all arcs p_a."""
    for g in small_grids():
        L = oracle.layout(g)
        x = synth.make_point(g, 1).x
        c, _ = oracle.constraints(g, x)
        vm = x[L.VM:L.VM + L.nb]
        lhs = np.sum(c[L.PB:L.PB + L.nb])
        rhs = (np.sum(g.Pd) + np.sum(g.Gs * vm ** 2) - np.sum(x[L.PG:L.PG + L.ng])
               + np.sum(x[L.P:L.P + 2 * L.nl]))
        assert abs(lhs - rhs) < 1e-12
        lhs = np.sum(c[L.QB:L.QB + L.nb])
        rhs = (np.sum(g.Qd) - np.sum(g.Bs * vm ** 2) - np.sum(x[L.QG:L.QG + L.ng])
               + np.sum(x[L.Q:L.Q + 2 * L.nl]))
        assert abs(lhs - rhs) < 1e-12


def test_two_bus_closed_form():
    g, x = two_bus_grid()
    gold = read_golden("two_bus_lossless.txt")
    L = oracle.layout(g)
    f, _ = oracle.objective(g, x)
    assert abs(f - gold["f"][0]) < 1e-13
    gr, _ = oracle.gradient(g, x)
    assert abs(gr[L.PG] - gold["grad_pg"][0]) < 1e-13
    c, _ = oracle.constraints(g, x)
    np.testing.assert_allclose(c, gold["cons"], rtol=0, atol=1e-14)
    jv, _ = oracle.jacobian(g, x)
    np.testing.assert_allclose(jv, gold["jac"], rtol=0, atol=1e-14)
    y = np.zeros(L.m)
    y[L.PF] = 1.0
    y[L.QT] = 2.0
    y[L.SF] = 0.5
    y[L.ST] = -0.25
    y[L.PB + 0] = 3.0
    y[L.QB + 1] = -1.0
    hv, _ = oracle.hessian(g, x, y, 1.0)
    np.testing.assert_allclose(hv, gold["hess"], rtol=0, atol=1e-14)


def test_objective_and_gradient_closed_form():
    g = synth.workload_grid("30bus")
    L = oracle.layout(g)
    x = synth.make_point(g, 4).x
    pg = x[L.PG:L.PG + L.ng]
    f, _ = oracle.objective(g, x)
    expect = sum(float(g.c2[k]) * pg[k] ** 2 + float(g.c1[k]) * pg[k] + float(g.c0[k])
                 for k in range(L.ng))
    assert abs(f - expect) < 1e-12 * abs(expect)
    gr, _ = oracle.gradient(g, x)
    assert np.count_nonzero(gr) == L.ng
    h = 1e-5
    for k in range(L.ng):
        xp, xm = x.copy(), x.copy()
        xp[L.PG + k] += h
        xm[L.PG + k] -= h
        fd = (oracle.objective(g, xp)[0] - oracle.objective(g, xm)[0]) / (2 * h)
        assert abs(fd - gr[L.PG + k]) < 1e-6 * (1 + abs(fd))


@pytest.mark.parametrize("which", [0, 1])
def test_jacobian_central_differences(which):
    g = small_grids()[which]
    x = synth.make_point(g, 11).x
    assert jac_vs_fd_err(g, x) < 1e-6
    # every nonzero of the FD Jacobian lies on the COO pattern
    L = oracle.layout(g)
    r, c = oracle.jac_structure(g)
    on = np.zeros((L.m, L.n), bool)
    on[r, c] = True
    assert not np.any((np.abs(fd_jacobian(g, x)) > 1e-8) & ~on)


@pytest.mark.parametrize("which", [0, 1])
def test_hessian_central_differences_and_symmetry(which):
    g = small_grids()[which]
    pt = synth.make_point(g, 12)
    sigma = 0.7
    Hfd = fd_hessian(g, pt.x, pt.y, sigma)
    # the FD Hessian of the Lagrangian is symmetric ...
    assert np.max(np.abs(Hfd - Hfd.T)) < 1e-5 * (1 + np.max(np.abs(Hfd)))
    # ... and equals the oracle's lower-stored Hessian, symmetrised
    assert hess_vs_fd_err(g, pt.x, pt.y, sigma) < 1e-6
    L = oracle.layout(g)
    r, c = oracle.hess_structure(g)
    on = np.zeros((L.n, L.n), bool)
    on[r, c] = True
    on |= on.T
    assert not np.any((np.abs(Hfd) > 1e-6) & ~on)


def test_hessian_linear_in_multipliers():
    g = synth.make_edge_case_grid(5)
    p1, p2 = synth.make_point(g, 1), synth.make_point(g, 2)
    x = p1.x
    h1, _ = oracle.hessian(g, x, p1.y, 0.3)
    h2, _ = oracle.hessian(g, x, p2.y, 1.1)
    h12, m12 = oracle.hessian(g, x, p1.y + p2.y, 1.4)
    assert np.all(np.abs(h1 + h2 - h12) <= 1e-14 * (1 + m12))


@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (0.3, 0.0), (0.25, 0.7), (0.0, 2.0)])
def test_condensed_kkt_equals_schur_complement(dw, dc):
    """Sec. IV.C: eliminating (ds, dy) from M_aug gives M_cond with
    D = (Ss + dw)(dc Ss + (1 + dc dw))^-1; checked for zero and nonzero
    regularisation on the 30-bus and edge-case grids, with Sigma over
    [1e-2, 1e2] (dense elimination stays accurate) and over the full
    [1e-8, 1e8] range."""
    for g in small_grids():
        assert kkt_vs_schur_err(g, moderate_point(g, 3), dw, dc) < 1e-10
        assert kkt_vs_schur_err(g, synth.make_point(g, 3), dw, dc) < 1e-8


def test_condensed_kkt_is_spd_without_multipliers():
    """With y = 0 and sigma = 1, W = diag(2 c2) >= 0, Sigma_x > 0 and A'DA >= 0,
    so M_cond is positive definite (dense Cholesky succeeds)."""
    for g in small_grids():
        pt = moderate_point(g, 5)
        K, _ = kkt_dense_from_oracle(g, pt.x, np.zeros_like(pt.y), 1.0,
                                     pt.sigma_x, pt.sigma_s, 0.0, 0.0)
        np.linalg.cholesky(K)
        assert np.all(np.linalg.eigvalsh(K) > 0)


def test_kkt_pattern_is_structural_union():
    """Brute force over dense 0/1 matrices: the CSR pattern is exactly the lower
    triangle of (|A|'|A| + |W| + I) > 0 with every diagonal present, sorted,
    without duplicates."""
    for g in small_grids():
        L = oracle.layout(g)
        rowptr, colind = oracle.kkt_structure(g)
        jr, jc = oracle.jac_structure(g)
        hr, hc = oracle.hess_structure(g)
        A = np.zeros((L.m, L.n))
        A[jr, jc] = 1
        H = np.zeros((L.n, L.n))
        H[hr, hc] = 1
        S = (A.T @ A + H + H.T + np.eye(L.n)) > 0
        S = np.tril(S)
        assert rowptr[0] == 0 and rowptr[-1] == colind.size
        got = np.zeros_like(S)
        for i in range(L.n):
            cols = colind[rowptr[i]:rowptr[i + 1]]
            assert np.all(np.diff(cols) > 0)
            assert cols[-1] == i
            got[i, cols] = True
        assert np.array_equal(got, S)


# ---------------------------------------------------------------------------
# planted mistakes: each pin must notice a plausible error in the oracle
# ---------------------------------------------------------------------------
def test_pin_catches_sign_error_in_admittance(monkeypatch):
    g = synth.make_edge_case_grid(7)
    x = synth.make_point(g, 0).x
    real = oracle.acopf.branch_admittance

    def wrong(grid):
        g_ff, b_ff, g_ft, b_ft, g_tf, b_tf, g_tt, b_tt = real(grid)
        return g_ff, b_ff, g_ft, -b_ft, g_tf, b_tf, g_tt, b_tt

    monkeypatch.setattr(oracle.acopf, "branch_admittance", wrong)
    assert flows_vs_phasor_err(g, x) > 1e-3


def test_pin_catches_dropped_shift_term(monkeypatch):
    g = synth.make_edge_case_grid(7)
    x = synth.make_point(g, 0).x
    real = oracle.acopf.branch_admittance

    def wrong(grid):
        g2 = grid.copy()
        g2.shift[:] = 0.0
        return real(g2)

    monkeypatch.setattr(oracle.acopf, "branch_admittance", wrong)
    assert flows_vs_phasor_err(g, x) > 1e-4


def test_pin_catches_dropped_jacobian_term(monkeypatch):
    g = synth.workload_grid("30bus")
    x = synth.make_point(g, 0).x
    real = oracle.acopf._flow_value_and_derivs

    def wrong(form, vm_f, vm_t, c, s):
        out = real(form, vm_f, vm_t, c, s)
        a, d, u, w = form
        out["vmf"] = (out["vmf"][0] - 2 * a * vm_f, out["vmf"][1])   # drop 2 a vm_f
        return out

    monkeypatch.setattr(oracle.acopf, "_flow_value_and_derivs", wrong)
    assert jac_vs_fd_err(g, x) > 1e-3


def test_pin_catches_hessian_index_swap(monkeypatch):
    g = synth.workload_grid("30bus")
    pt = synth.make_point(g, 0)
    real = oracle.acopf.hessian

    def wrong(grid, x, y, obj_weight=1.0):
        v, m = real(grid, x, y, obj_weight)
        v = v.copy()
        nl = grid.n_branch
        blk = v[:10 * nl].reshape(10, nl)
        blk[[6, 4], :] = blk[[4, 6], :]          # (vm_t,va_f) <-> (vm_f,va_t)
        return v, m

    monkeypatch.setattr(oracle, "hessian", wrong)
    assert hess_vs_fd_err(g, pt.x, pt.y, 1.0) > 1e-3


def test_pin_catches_transposed_condensation(monkeypatch):
    g = synth.workload_grid("30bus")
    pt = moderate_point(g, 2)
    real = oracle.acopf.condensation_diag

    def wrong(sigma_s, delta_w=0.0, delta_c=0.0):
        # C and D swapped: D := C
        C = 1.0 / (delta_c * np.asarray(sigma_s) + (1.0 + delta_c * delta_w))
        return C, np.abs(C)

    monkeypatch.setattr(oracle.acopf, "condensation_diag", wrong)
    assert kkt_vs_schur_err(g, pt, 0.25, 0.7) > 1e-3
