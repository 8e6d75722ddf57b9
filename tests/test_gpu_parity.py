"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Indices are compared bit for bit (CPU tests cover the host symbolic phase);
values must satisfy |v - o| <= 1e-12 M + 1e-14 entrywise, M being the oracle's
sum of absolute terms.  Cases span several thread blocks with a ragged tail,
every structural corner of the formulation, regularised condensation, the
separate callbacks, the array-fed assembly, the host-buffer entry point, and
the full 10k and 80k-bus workloads in the launch configuration the benchmark
times.
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


def small_cases():
    return [
        ("30bus", synth.workload_grid("30bus")),
        ("edge7", synth.make_edge_case_grid(7)),
        ("edge11", synth.make_edge_case_grid(11)),
        ("ragged", synth.make_grid(517, 777, 61, seed=3)),   # 7 branch blocks, ragged tail
        ("tree", synth.make_grid(200, 199, 20, seed=4)),      # radial: every bus a tree node
        ("star", synth.make_star_grid()),                      # hub with 300 arcs, 260 generators
    ]


@pytest.mark.parametrize("idx", range(6))
def test_fused_matches_oracle(dev, acopf, idx):
    name, g = small_cases()[idx]
    with acopf.model_create(g, 0) as m:
        for seed in (1, 2):
            pt = synth.make_point(g, seed, obj_weight=0.7)
            got = gu.run_fused(torch, acopf, m, pt, dev)
            gu.assert_parity(got, gu.oracle_all(g, pt), label=f"{name}/seed{seed}")


@pytest.mark.parametrize("dw,dc", [(1e-4, 0.0), (0.3, 0.7), (0.0, 1e-3)])
def test_fused_regularised(dev, acopf, dw, dc):
    g = synth.make_edge_case_grid(7)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 5, delta_w=dw, delta_c=dc)
        got = gu.run_fused(torch, acopf, m, pt, dev)
        gu.assert_parity(got, gu.oracle_all(g, pt), label=f"dw={dw} dc={dc}")


@pytest.mark.parametrize("idx", range(6))
def test_separate_callbacks_match_oracle(dev, acopf, idx):
    name, g = small_cases()[idx]
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 3, obj_weight=1.3, delta_w=0.01, delta_c=0.02)
        got = gu.run_separate(torch, acopf, m, pt, dev)
        gu.assert_parity(got, gu.oracle_all(g, pt), label=name)


def test_array_fed_assembly_on_arbitrary_values(dev, acopf):
    """assemble_condensed_kkt_csr is W + dI + Sx + A'DA for ANY given H and J
    values, including entries the callbacks would fill with constants."""
    g = synth.make_edge_case_grid(11)
    rng = np.random.default_rng(42)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 9)
        hv = rng.standard_normal(m.nnz_hess)
        jv = rng.standard_normal(m.nnz_jac)
        for dw, dc in ((0.0, 0.0), (0.2, 0.5)):
            kv, km = oracle.condensed_kkt(g, hv, jv, pt.sigma_x, pt.sigma_s, dw, dc)
            out = torch.full((m.nnz_kkt,), float("nan"), dtype=torch.float64, device=dev)
            acopf.assemble_condensed_kkt_csr(
                m, gu.t64(torch, hv, dev), gu.t64(torch, jv, dev), gu.t64(torch, pt.sigma_x, dev),
                gu.t64(torch, pt.sigma_s, dev), dw, dc, out)
            torch.cuda.synchronize()
            gu.assert_parity({"kkt": out.cpu().numpy()}, {"kkt": (kv, km)}, keys=("kkt",))


def test_deterministic_bitwise(dev, acopf):
    g = synth.make_grid(2000, 2700, 300, seed=8)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 1)
        a = gu.run_fused(torch, acopf, m, pt, dev)
        b = gu.run_fused(torch, acopf, m, pt, dev)
        for k in gu.KEYS:
            assert np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)), k


def test_host_buffer_entry_point_equals_device_path(dev, acopf):
    g = synth.make_edge_case_grid(7)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 4)
        d = gu.run_fused(torch, acopf, m, pt, dev)
        h = {"f": np.empty(1), "grad": np.empty(m.n), "cons": np.empty(m.m),
             "jac": np.empty(m.nnz_jac), "hess": np.empty(m.nnz_hess), "kkt": np.empty(m.nnz_kkt)}
        for _ in range(2):
            acopf.eval_assemble_host(m, pt.x, pt.y, pt.obj_weight, pt.sigma_x, pt.sigma_s,
                                     pt.delta_w, pt.delta_c, h["f"], h["grad"], h["cons"],
                                     h["jac"], h["hess"], h["kkt"], stream=0)
            for k in gu.KEYS:
                assert np.array_equal(d[k], h[k]), k


def test_degenerate_networks(dev, acopf):
    """One bus with no branch and no generator; two buses without generators."""
    one = synth.Grid(
        bus_type=np.array([3], np.int32), Pd=np.array([0.3]), Qd=np.array([0.1]),
        Gs=np.array([0.05]), Bs=np.array([0.02]), Vmin=np.array([0.9]), Vmax=np.array([1.1]),
        f=np.zeros(0, np.int32), t=np.zeros(0, np.int32), r=np.zeros(0), x=np.zeros(0),
        b=np.zeros(0), tap=np.zeros(0), shift=np.zeros(0), rate_a=np.zeros(0),
        angmin=np.zeros(0), angmax=np.zeros(0), gen_bus=np.zeros(0, np.int32),
        Pmin=np.zeros(0), Pmax=np.zeros(0), Qmin=np.zeros(0), Qmax=np.zeros(0),
        c2=np.zeros(0), c1=np.zeros(0), c0=np.zeros(0), name="one-bus")
    g2 = synth.workload_grid("30bus")
    two = synth.Grid(
        bus_type=np.array([1, 3], np.int32), Pd=np.array([0.3, 0.2]), Qd=np.array([0.1, 0.0]),
        Gs=np.zeros(2), Bs=np.zeros(2), Vmin=np.full(2, 0.9), Vmax=np.full(2, 1.1),
        f=np.array([1], np.int32), t=np.array([0], np.int32), r=g2.r[:1], x=g2.x[:1],
        b=g2.b[:1], tap=np.array([0.0]), shift=np.array([0.1]), rate_a=np.array([0.0]),
        angmin=g2.angmin[:1], angmax=g2.angmax[:1], gen_bus=np.zeros(0, np.int32),
        Pmin=np.zeros(0), Pmax=np.zeros(0), Qmin=np.zeros(0), Qmax=np.zeros(0),
        c2=np.zeros(0), c1=np.zeros(0), c0=np.zeros(0), name="two-bus-no-gen")
    for g in (one, two):
        with acopf.model_create(g, 0) as m:
            pt = synth.make_point(g, 2)
            got = gu.run_fused(torch, acopf, m, pt, dev)
            gu.assert_parity(got, gu.oracle_all(g, pt), label=g.name)
            assert got["f"][0] == 0.0


@pytest.mark.parametrize("name", ["10kbus", "80kbus"])
def test_full_size_workloads(dev, acopf, name):
    """Every output of the 10k and 80k-bus workloads against the oracle, at
    two fresh points, in the launch configuration bench.py times."""
    g = synth.workload_grid(name)
    with acopf.model_create(g, 0) as m:
        for call in (0, 1):
            pt = synth.make_point(g, synth.point_seed(synth.WORKLOADS[name]["seed"], call))
            got = gu.run_fused(torch, acopf, m, pt, dev)
            gu.assert_parity(got, gu.oracle_all(g, pt), label=f"{name}/call{call}")


def test_streams_and_profiling(dev, acopf):
    g = synth.make_grid(3000, 4100, 400, seed=12)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 6)
        ref = gu.run_fused(torch, acopf, m, pt, dev)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            got = gu.run_fused(torch, acopf, m, pt, dev, stream=s)
        for k in gu.KEYS:
            assert np.array_equal(ref[k], got[k]), k
        acopf.profile_begin(m, 3)
        for _ in range(3):
            got = gu.run_fused(torch, acopf, m, pt, dev)
        calls, p1, p2, tot = acopf.profile_end(m)
        assert calls == 3 and p1 > 0 and p2 > 0 and tot >= p1
        for k in gu.KEYS:
            assert np.array_equal(ref[k], got[k]), k


def test_pdl_option_does_not_change_results(dev, acopf):
    g = synth.make_edge_case_grid(7)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 13)
        a = gu.run_fused(torch, acopf, m, pt, dev)
        acopf.model_set_option(m, acopf.OPT_PDL, 0)
        b = gu.run_fused(torch, acopf, m, pt, dev)
        for k in gu.KEYS:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("spread", [20.0, 3e5])
def test_fused_at_wide_angles(dev, acopf, spread):
    """Branch angles far outside the operating range (every quadrant, up to
    hundreds of thousands of radians) still match the oracle."""
    g = synth.make_grid(517, 777, 61, seed=3)
    rng = np.random.default_rng(77)
    with acopf.model_create(g, 0) as m:
        pt = synth.make_point(g, 9, obj_weight=1.1)
        pt.x = pt.x.copy()
        pt.x[:g.n_bus] = rng.uniform(-spread, spread, g.n_bus)
        got = gu.run_fused(torch, acopf, m, pt, dev)
        gu.assert_parity(got, gu.oracle_all(g, pt), label=f"spread {spread}")



@pytest.mark.parametrize("depth", [2, 3])
def test_pipeline_matches_single_calls(dev, acopf, depth):
    """Pipelined host-buffer calls (copies and kernels of consecutive calls
    overlapping) give each call's single-call results bit for bit."""
    g = synth.make_grid(517, 777, 61, seed=3)
    with acopf.model_create(g, 0) as m:
        pts = [synth.make_point(g, 40 + k, obj_weight=0.9 + 0.05 * k,
                                delta_w=0.02 if k == 3 else 0.0) for k in range(5)]
        ref = [gu.run_fused(torch, acopf, m, pt, dev) for pt in pts]
        outs = []
        with acopf.pipeline_create(m, depth) as p:
            for pt in pts:
                o = {k: np.full(n, np.nan) for k, n in (("f", 1), ("grad", m.n), ("cons", m.m),
                                                         ("jac", m.nnz_jac), ("hess", m.nnz_hess),
                                                         ("kkt", m.nnz_kkt))}
                p.submit(pt.x, pt.y, pt.obj_weight, pt.sigma_x, pt.sigma_s, pt.delta_w,
                         pt.delta_c, o["f"], o["grad"], o["cons"], o["jac"], o["hess"], o["kkt"])
                outs.append(o)
            p.wait()
        for k in range(len(pts)):
            for key in gu.KEYS:
                assert np.array_equal(outs[k][key].view(np.uint64), ref[k][key].view(np.uint64)), \
                    (k, key)
        for bad in (1, 9):
            with pytest.raises(acopf.AcopfError) as e:
                acopf.pipeline_create(m, bad)
            assert e.value.status == acopf.E_INVALID_ARG
