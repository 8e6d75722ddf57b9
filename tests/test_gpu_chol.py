"""GPU sparse Cholesky of M_cond (acopf_chol_*) against the oracle
(oracle/chol.py).

* Small networks, M_cond from the oracle's own callbacks: a convex case
  (no constraint multipliers and delta_w > 0, positive definite by
  construction, and so by the oracle's dense test) must factor with every
  pivot passing; a nonconvex case the oracle finds indefinite must fail the
  test.  Solves: the normwise backward error (computed by the oracle) at
  most 1e-13, and the forward error against the oracle's solve within
  10 n kappa eps (kappa the 2-norm condition number, computed densely).
* The chain at full size (the near-planar 10,000- and 80,000-bus
  workloads): the library assembles M_cond, factors it and solves; backward
  error against the oracle's M_cond; a planted negative diagonal entry fails
  the pivot test, and the original values factor again.
"""
import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def acopf():
    from paper_2307_16830_gb300 import acopf as lib
    return lib


def _sigmas(L, seed):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-2, 2, L.n), 10.0 ** rng.uniform(-2, 2, L.m)


def _oracle_kvals(g, seed, y_scale, dw, dc):
    L = oracle.layout(g)
    pt = synth.make_point(g, seed)
    sx, ss = _sigmas(L, seed + 1)
    H = oracle.hessian(g, pt.x, pt.y * y_scale, 1.0)[0]
    J = oracle.jacobian(g, pt.x)[0]
    kv, _ = oracle.condensed_kkt(g, H, J, sx, ss, dw, dc)
    return kv


CASES = [("30bus", lambda: synth.workload_grid("30bus")),
         ("edge7", lambda: synth.make_edge_case_grid(7)),
         ("star", lambda: synth.make_star_grid()),
         ("ragged", lambda: synth.make_grid(517, 777, 61, seed=3))]


@pytest.mark.parametrize("idx", range(len(CASES)))
@pytest.mark.parametrize("dc", [0.0, 1e-3])
def test_convex_case_factors_and_solves(dev, acopf, idx, dc):
    name, make = CASES[idx]
    g = make()
    L = oracle.layout(g)
    kv = _oracle_kvals(g, 40 + idx, 0.0, 1e-4, dc)
    if L.n <= 1500:
        assert oracle.is_positive_definite(g, kv)
    b = np.random.default_rng(50 + idx).standard_normal(L.n)
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        kd = gu.t64(torch, kv, dev)
        assert ch.factor(kd) == -1, name
        bd = gu.t64(torch, b, dev)
        xd = torch.full((L.n,), float("nan"), dtype=torch.float64, device=dev)
        ch.solve(bd, xd)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        assert oracle.backward_error(g, kv, x, b) <= 1e-13, name
        if L.n <= 1500:
            ref = oracle.solve_condensed(g, kv, b)
            kappa = np.linalg.cond(oracle.condensed_matrix(g, kv).toarray())
            err = np.max(np.abs(x - ref)) / np.max(np.abs(ref))
            assert err <= 10 * L.n * kappa * EPS, (name, err, kappa)
        # a second factorization and solve of the same values is bit-identical
        assert ch.factor(kd) == -1
        x2 = torch.full_like(xd, float("nan"))
        ch.solve(bd, x2)
        torch.cuda.synchronize()
        assert np.array_equal(x.view(np.uint64), x2.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("idx", [0, 1, 3])
def test_nonconvex_case_fails_the_pivot_test(dev, acopf, idx):
    name, make = CASES[idx]
    g = make()
    kv = _oracle_kvals(g, 60 + idx, 50.0, 0.0, 0.0)
    assert not oracle.is_positive_definite(g, kv), "the case must be indefinite"
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        assert ch.factor(gu.t64(torch, kv, dev)) >= 0, name
        z = torch.zeros(m.n, dtype=torch.float64, device=dev)
        with pytest.raises(acopf.AcopfError) as e:
            ch.solve(z, torch.empty_like(z))
        assert e.value.status == acopf.E_INVALID_ARG


@pytest.mark.parametrize("workload", ["10kbus-geo", "80kbus-geo"])
def test_chain_at_full_size(dev, acopf, workload):
    g = synth.workload_grid(workload)
    L = oracle.layout(g)
    pt = synth.make_point(g, 70)
    sx, ss = _sigmas(L, 71)
    dw = 1e-4
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        out = gu.alloc_outputs(torch, m, dev)
        acopf.eval_assemble(m, gu.t64(torch, pt.x, dev), torch.zeros(L.m, dtype=torch.float64,
                                                                      device=dev),
                            1.0, gu.t64(torch, sx, dev), gu.t64(torch, ss, dev), dw, 0.0,
                            out["f"], out["grad"], out["cons"], out["jac"], out["hess"],
                            out["kkt"])
        assert ch.factor(out["kkt"]) == -1
        b = np.random.default_rng(72).standard_normal(L.n)
        xd = torch.full((L.n,), float("nan"), dtype=torch.float64, device=dev)
        ch.solve(gu.t64(torch, b, dev), xd)
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        H = oracle.hessian(g, pt.x, np.zeros(L.m), 1.0)[0]
        J = oracle.jacobian(g, pt.x)[0]
        kv, _ = oracle.condensed_kkt(g, H, J, sx, ss, dw, 0.0)
        assert oracle.backward_error(g, kv, x, b) <= 1e-13
        # a negative diagonal entry: never positive definite
        rp, _ = m.kkt_structure()
        bad = out["kkt"].clone()
        bad[int(rp[L.n // 2 + 1]) - 1] = -1.0
        assert ch.factor(bad) >= 0
        assert ch.factor(out["kkt"]) == -1
        info = ch.info()
        assert info["nnz_full"] == 2 * int(rp[-1]) - L.n and info["device_bytes"] > 0
        assert info["nnz_factor"] >= L.n and 1 <= info["max_col"] <= L.n


def test_chol_rejects_bad_arguments(dev, acopf):
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        z = torch.zeros(m.nnz_kkt, dtype=torch.float64, device=dev)
        with pytest.raises(acopf.AcopfError) as e:
            ch.factor(z, pivot_tol=-1.0)
        assert e.value.status == acopf.E_INVALID_ARG
        with pytest.raises(acopf.AcopfError) as e:
            ch.factor(None)
        assert e.value.status == acopf.E_INVALID_ARG
        with pytest.raises(acopf.AcopfError) as e:  # nothing factored yet
            ch.solve(z, z)
        assert e.value.status == acopf.E_INVALID_ARG


def test_object_order_is_the_symbolic_order(dev, acopf):
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        stats, p = acopf.chol_analyze(m, with_perm=True)
        assert np.array_equal(ch.permutation(), p)
        info = ch.info()
        assert stats == {k: info[k] for k in stats}


def test_graph_path_matches_direct_path(dev, acopf):
    """On a created stream the factorization and the solve run as captured
    CUDA graphs (re-captured when their arguments change); the results are
    bit-identical to the direct launches on the default stream."""
    g = synth.make_grid(3000, 4050, 600, seed=4, topology="geometric")
    L = oracle.layout(g)
    kv1 = _oracle_kvals(g, 90, 0.0, 1e-4, 0.0)
    kv2 = _oracle_kvals(g, 91, 0.0, 1e-3, 0.0)
    b = gu.t64(torch, np.random.default_rng(92).standard_normal(L.n), dev)
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        ref = []
        for kv in (kv1, kv2):
            assert ch.factor(gu.t64(torch, kv, dev)) == -1
            x = torch.empty(L.n, dtype=torch.float64, device=dev)
            ch.solve(b, x)
            torch.cuda.synchronize()
            ref.append(x.cpu().numpy())
        st = torch.cuda.Stream(device=dev)
        k1, k2 = gu.t64(torch, kv1, dev), gu.t64(torch, kv2, dev)
        x = torch.empty(L.n, dtype=torch.float64, device=dev)
        for rep in range(2):  # capture, then replay
            for kd, r in ((k1, ref[0]), (k2, ref[1])):
                assert ch.factor(kd, stream=st) == -1
                ch.solve(b, x, stream=st)
                st.synchronize()
                assert np.array_equal(x.cpu().numpy().view(np.uint64), r.view(np.uint64)), rep
        bad = k1.clone()
        bad[0] = -1.0  # row 0's only entry is its diagonal
        assert ch.factor(bad, stream=st) >= 0
        assert ch.factor(k1, stream=st) == -1


def test_solve_captured_in_a_caller_graph(dev, acopf):
    """A solve recorded inside the caller's own CUDA graph capture becomes part
    of that graph; its replay gives the bits of a direct solve."""
    g = synth.workload_grid("30bus")
    L = oracle.layout(g)
    kv = _oracle_kvals(g, 95, 0.0, 1e-4, 0.0)
    with acopf.model_create(g, 0) as m, acopf.chol_create(m) as ch:
        assert ch.factor(gu.t64(torch, kv, dev)) == -1
        b = gu.t64(torch, np.random.default_rng(96).standard_normal(L.n), dev)
        ref = torch.empty(L.n, dtype=torch.float64, device=dev)
        ch.solve(b, ref)
        torch.cuda.synchronize()
        st = torch.cuda.Stream(device=dev)
        x = torch.full((L.n,), float("nan"), dtype=torch.float64, device=dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            ch.solve(b, x, stream=st)
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy().view(np.uint64), ref.cpu().numpy().view(np.uint64))
