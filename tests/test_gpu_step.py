"""GPU parity of the condensation around M_cond and the step recovery
(acopf_condense, acopf_recover_step) against the oracle (oracle/step.py).

Inputs are seeded: an interior iterate inside the model's bounds (with the
free and one-sided bounds of the model, so infinite bounds are exercised),
Jacobian values either arbitrary (the operations are linear in them) or
evaluated at a point by the library and by the oracle, and an arbitrary dx.
Every entry must satisfy |v - o| <= 1e-12 M + 1e-14 (M the oracle's
magnitude); repeated calls are bit-identical.
"""
import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def acopf():
    from paper_2307_16830_gb300 import acopf as lib
    return lib


def _iterate(m, seed, dev):
    xl, xu, gl, gu_ = m.bounds()
    d = synth.make_iterate(xl, xu, gl, gu_, seed)
    return d, {k: gu.t64(torch, v, dev) for k, v in d.items()}


def _run(acopf, m, it_dev, jv, dx, dw, dc, dev):
    e = lambda n: torch.full((n,), float("nan"), dtype=torch.float64, device=dev)  # noqa: E731
    out = {"sigma_x": e(m.n), "sigma_s": e(m.m), "q_s": e(m.m), "rhs": e(m.n)}
    acopf.condense(m, it_dev, jv, dw, dc, out["sigma_x"], out["sigma_s"], out["q_s"], out["rhs"])
    rec = {k: e(n) for k, n in (("ds", m.m), ("dy", m.m), ("dzl_x", m.n), ("dzu_x", m.n),
                                ("dzl_s", m.m), ("dzu_s", m.m))}
    acopf.recover_step(m, it_dev, jv, dw, dc, out["sigma_s"], out["q_s"], dx, rec["ds"],
                       rec["dy"], rec["dzl_x"], rec["dzu_x"], rec["dzl_s"], rec["dzu_s"])
    torch.cuda.synchronize()
    out.update(rec)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check(got, ref, keys, label):
    for k in keys:
        val, mag = ref[k]
        ok = oracle.within_tol(got[k], val, mag)
        if not ok.all():
            i = np.flatnonzero(~ok)[0]
            raise AssertionError(f"{label} {k}: {int((~ok).sum())} entries out of tolerance; "
                                 f"first {i}: gpu={got[k][i]!r} oracle={val[i]!r} mag={mag[i]!r}")


CASES = [("30bus", lambda: synth.workload_grid("30bus")),
         ("edge7", lambda: synth.make_edge_case_grid(7)),
         ("star", lambda: synth.make_star_grid()),
         ("ragged", lambda: synth.make_grid(517, 777, 61, seed=3))]


@pytest.mark.parametrize("idx", range(len(CASES)))
@pytest.mark.parametrize("dw,dc", [(0.0, 0.0), (0.1, 0.01)])
def test_condense_and_recover_on_arbitrary_jacobian(dev, acopf, idx, dw, dc):
    name, make = CASES[idx]
    g = make()
    with acopf.model_create(g, 0) as m:
        d, it_dev = _iterate(m, 100 + idx, dev)
        rng = np.random.default_rng(200 + idx)
        jv = rng.standard_normal(m.nnz_jac) * 10.0 ** rng.uniform(-2, 2, m.nnz_jac)
        dx = rng.standard_normal(m.n)
        got = _run(acopf, m, it_dev, gu.t64(torch, jv, dev), gu.t64(torch, dx, dev), dw, dc, dev)
        it = oracle.Iterate(**d)
        ref = oracle.condense(g, jv, it, dw, dc)
        ref.update(oracle.recover(g, jv, it, dx, dw, dc))
        _check(got, ref, ("sigma_x", "sigma_s", "q_s", "rhs", "ds", "dy", "dzl_x", "dzu_x",
                          "dzl_s", "dzu_s"), f"{name} dw={dw} dc={dc}")
        again = _run(acopf, m, it_dev, gu.t64(torch, jv, dev), gu.t64(torch, dx, dev), dw, dc, dev)
        for k in got:
            assert np.array_equal(got[k].view(np.uint64), again[k].view(np.uint64)), k


@pytest.mark.parametrize("workload", ["10kbus", "80kbus"])
def test_condense_chain_at_full_size(dev, acopf, workload):
    """The library's own Jacobian at a point feeds the condensation; the
    oracle's Jacobian at the same point feeds the oracle's."""
    g = synth.workload_grid(workload)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 7)
        d, it_dev = _iterate(m, 300, dev)
        jv_dev = torch.empty(m.nnz_jac, dtype=torch.float64, device=dev)
        acopf.eval_jac_coo(m, gu.t64(torch, pt.x, dev), jv_dev)
        dx = np.random.default_rng(301).standard_normal(m.n)
        got = _run(acopf, m, it_dev, jv_dev, gu.t64(torch, dx, dev), 0.0, 0.0, dev)
        jv, jm = oracle.jacobian(g, pt.x)
        it = oracle.Iterate(**d)
        ref = oracle.condense(g, jv, it, 0.0, 0.0, jmag=jm)
        ref.update(oracle.recover(g, jv, it, dx, 0.0, 0.0, jmag=jm))
        _check(got, ref, ("sigma_x", "sigma_s", "q_s", "rhs", "ds", "dy", "dzl_x", "dzu_x",
                          "dzl_s", "dzu_s"), workload)


def test_condense_rejects_bad_arguments(dev, acopf):
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, 0) as m:
        d, it_dev = _iterate(m, 1, dev)
        z = torch.zeros(max(m.n, m.m, m.nnz_jac), dtype=torch.float64, device=dev)
        bad = dict(it_dev)
        bad["p_y"] = None
        with pytest.raises(acopf.AcopfError) as e:
            acopf.condense(m, bad, z, 0.0, 0.0, z, z, z, z)
        assert e.value.status == acopf.E_INVALID_ARG
        with pytest.raises(acopf.AcopfError) as e:
            acopf.condense(m, it_dev, z, -1.0, 0.0, z, z, z, z)
        assert e.value.status == acopf.E_INVALID_ARG


@pytest.mark.parametrize("name,make,scale", [
    ("30bus", lambda: synth.workload_grid("30bus"), 1.0),
    ("edge7", lambda: synth.make_edge_case_grid(7), 1.0),
    ("ragged", lambda: synth.make_grid(517, 777, 61, seed=3), 1e4),
    ("10kbus", lambda: synth.workload_grid("10kbus"), 1.0)])
def test_kkt_residual_matches_oracle(dev, acopf, name, make, scale):
    """The scaled residual from the library's own callbacks at x equals the
    oracle's from its callbacks (norms to 1e-10 relative, the bound count
    exactly); scale multiplies y and the duals, so the scaling engages."""
    g = make()
    with acopf.model_create(g, 0) as m:
        d, _ = _iterate(m, 700, dev)
        for k in ("zl_x", "zu_x", "zl_s", "zu_s"):
            d[k] = d[k] * scale
        it_dev = {k: gu.t64(torch, v, dev) for k, v in d.items()}
        y = np.random.default_rng(701).standard_normal(m.m) * scale
        xd = it_dev["x"]
        grad = torch.empty(m.n, dtype=torch.float64, device=dev)
        cons = torch.empty(m.m, dtype=torch.float64, device=dev)
        jv = torch.empty(m.nnz_jac, dtype=torch.float64, device=dev)
        acopf.eval_grad(m, xd, grad)
        acopf.eval_cons(m, xd, cons)
        acopf.eval_jac_coo(m, xd, jv)
        out = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
        yd = gu.t64(torch, y, dev)
        acopf.kkt_residual(m, it_dev, yd, grad, cons, jv, 0.1, out)
        torch.cuda.synchronize()
        got = dict(zip(acopf.RESIDUAL_FIELDS, out.cpu().numpy()))
        it = oracle.Iterate(**d)
        ref = oracle.kkt_residual(g, oracle.gradient(g, it.x)[0], oracle.constraints(g, it.x)[0],
                                  oracle.jacobian(g, it.x)[0], it, y, 0.1)
        assert got["n_z"] == ref["n_z"]
        for k in acopf.RESIDUAL_FIELDS:
            if k == "n_z":
                continue
            assert abs(got[k] - ref[k]) <= 1e-10 * max(1.0, abs(ref[k])), (name, k, got[k], ref[k])
        if scale > 1.0:
            assert got["s_d"] > 1.0 and got["s_c"] > 1.0
        again = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
        acopf.kkt_residual(m, it_dev, yd, grad, cons, jv, 0.1, again)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint64), again.cpu().numpy().view(np.uint64))
