"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host symbolic phase reproduces the oracle's index arrays bit for bit.

No compute call runs here (models are created host-only, device = -1)."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

acopf = pytest.importorskip("paper_2307_16830_gb300.acopf",
                            reason="libacopf.so not built (run __graft_entry__.build())")

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "acopf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(acopf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    lib = acopf._lib
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(acopf.EXPORTED) == names


def test_status_strings():
    assert acopf.status_string(acopf.OK) == "ACOPF_OK"
    assert acopf.status_string(acopf.E_BAD_MODEL) == "ACOPF_E_BAD_MODEL"
    assert acopf.status_string(12345) == "ACOPF_E_UNKNOWN"


def grids():
    return [synth.workload_grid("30bus"), synth.make_edge_case_grid(7),
            synth.make_edge_case_grid(11), synth.make_grid(300, 420, 40, seed=5),
            synth.make_star_grid()]


@pytest.mark.parametrize("k", range(5))
def test_host_structures_match_oracle_bit_exactly(k):
    g = grids()[k]
    with acopf.model_create(g, device=-1) as m:
        L = oracle.layout(g)
        assert (m.n, m.m) == (L.n, L.m)
        assert (m.n_bus, m.n_branch, m.n_gen, m.n_ref) == (g.n_bus, g.n_branch, g.n_gen, g.n_ref)
        jr, jc = oracle.jac_structure(g)
        r, c = m.jac_structure()
        assert np.array_equal(r, jr) and np.array_equal(c, jc)
        hr, hc = oracle.hess_structure(g)
        r, c = m.hess_structure()
        assert np.array_equal(r, hr) and np.array_equal(c, hc)
        rp, ci = oracle.kkt_structure(g)
        r, c = m.kkt_structure()
        assert m.nnz_kkt == ci.size
        assert np.array_equal(r, rp) and np.array_equal(c, ci)
        xl, xu, gl, gu = oracle.bounds(g)
        bl = m.bounds()
        for got, want in zip(bl, (xl, xu, gl, gu)):
            assert np.array_equal(got, want)


def test_host_structures_10k_grid():
    g = synth.workload_grid("10kbus")
    with acopf.model_create(g, device=-1) as m:
        rp, ci = oracle.kkt_structure(g)
        r, c = m.kkt_structure()
        assert np.array_equal(r, rp) and np.array_equal(c, ci)
        jr, jc = oracle.jac_structure(g)
        r, c = m.jac_structure()
        assert np.array_equal(r, jr) and np.array_equal(c, jc)


def test_sizes_match_formulas():
    g = synth.workload_grid("10kbus")
    with acopf.model_create(g, device=-1) as m:
        nb, nl, ng = g.n_bus, g.n_branch, g.n_gen
        assert m.n == 2 * nb + 2 * ng + 4 * nl == 78_000
        assert m.m == 1 + 7 * nl + 2 * nb == 114_501
        assert m.nnz_jac == 1 + 30 * nl + 2 * nb + 2 * ng == 429_001
        assert m.nnz_hess == 14 * nl + ng + nb == 201_000


def _bad(g, **changes):
    g = g.copy()
    for k, v in changes.items():
        getattr(g, k)[...] = v
    return g


def test_validation_rejects_bad_networks():
    g = synth.workload_grid("30bus")
    cases = []
    h = g.copy()
    h.t[0] = h.f[0]
    cases.append(("self-loop", h))
    h = g.copy()
    h.f[3] = g.n_bus
    cases.append(("bus out of range", h))
    h = g.copy()
    h.r[2] = 0.0
    h.x[2] = 0.0
    cases.append(("zero impedance", h))
    h = g.copy()
    h.gen_bus[1] = -1
    cases.append(("generator bus", h))
    h = g.copy()
    h.Pd[4] = math.nan
    cases.append(("nan load", h))
    for name, bad in cases:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.model_create(bad, device=-1)
        assert ei.value.status == acopf.E_BAD_MODEL, name
        assert acopf.last_error()


def test_host_only_model_refuses_compute_calls():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, device=-1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.eval_cons(m, 1, 2, stream=0)
        assert ei.value.status == acopf.E_NO_DEVICE
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.eval_assemble(m, 1, 1, 1.0, 1, 1, 0.0, 0.0, 1, 1, 1, 1, 1, 1, stream=0)
        assert ei.value.status == acopf.E_NO_DEVICE


def test_null_arguments_rejected():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, device=-1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.eval_cons(m, None, None, stream=0)
        assert ei.value.status == acopf.E_INVALID_ARG
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.assemble_condensed_kkt_csr(m, 1, 1, 1, 1, -1.0, 0.0, 1, stream=0)
        assert ei.value.status == acopf.E_INVALID_ARG


def test_launch_accounting():
    for kind in range(7):
        assert acopf.launches_per_call(kind) == (2 if kind in (0, 1) else 1)
    assert acopf.launches_per_call(99) == -1


def test_batch_create_rejects_without_device_work():
    """Argument checks of acopf_batch_create that come before any CUDA call."""
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, device=-1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.batch_create([m])
        assert ei.value.status == acopf.E_NO_DEVICE
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.batch_create([])
        assert ei.value.status == acopf.E_INVALID_ARG



def test_server_create_rejects_without_device_work():
    """Argument checks of acopf_server_create that come before any CUDA call."""
    with pytest.raises(acopf.AcopfError) as ei:
        acopf.server_create(-1, 1 << 30)
    assert ei.value.status == acopf.E_NO_DEVICE
    for budget, mode, max_active in ((0, acopf.SERVE_CONTINUOUS, 4), (1 << 30, 7, 4),
                                     (1 << 30, acopf.SERVE_FIFO, 0)):
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.server_create(0, budget, mode, max_active)
        assert ei.value.status == acopf.E_INVALID_ARG


@pytest.mark.parametrize("k", range(3))
def test_arc_rows_tile_contiguous_ranges(k):
    """The kernels stage the arc rows of a warp's 32 consecutive branches in
    shared memory and write them as one range: row p_l of M_cond must hold
    exactly 5 + (generators at the from bus) + (earlier arcs at that bus)
    entries and row q_l one more, and consecutive branches' rows must be
    consecutive CSR rows (likewise p_{nl+l}, q_{nl+l} at the to bus)."""
    g = [synth.make_edge_case_grid(7), synth.make_grid(517, 777, 61, seed=3),
         synth.make_star_grid()][k]
    with acopf.model_create(g, device=-1) as m:
        rp, _ = m.kkt_structure()
        nb, nl, ng = m.n_bus, m.n_branch, m.n_gen
        P, Q = 2 * nb + 2 * ng, 2 * nb + 2 * ng + 2 * nl
        gens = np.bincount(np.asarray(g.gen_bus), minlength=nb)
        bus_of_arc = np.concatenate([np.asarray(g.f), np.asarray(g.t)])
        seen = np.zeros(nb, dtype=np.int64)
        rank = np.zeros(2 * nl, dtype=np.int64)
        for a in range(2 * nl):  # earlier arcs (smaller arc index) at the same bus
            rank[a] = seen[bus_of_arc[a]]
            seen[bus_of_arc[a]] += 1
        ln = np.diff(rp)
        for a in range(2 * nl):
            i = bus_of_arc[a]
            assert ln[P + a] == 5 + gens[i] + rank[a], (a, ln[P + a])
            assert ln[Q + a] == 6 + gens[i] + rank[a], (a, ln[Q + a])


def test_pipeline_create_rejects_without_device_work():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, device=-1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.pipeline_create(m, 2)
        assert ei.value.status == acopf.E_NO_DEVICE


def test_chol_create_rejects_without_device_work():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, -1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.chol_create(m)
        assert ei.value.status == acopf.E_NO_DEVICE


def test_chol_analyze_runs_on_host_only_models():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, -1) as m:
        st = acopf.chol_analyze(m)
        assert st["n"] == m.n and st["nnz_factor"] >= st["n"]


def test_ipm_solve_rejects_without_device_work():
    g = synth.workload_grid("30bus-opf")
    with acopf.model_create(g, -1) as m:
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.ipm_solve(m)
        assert ei.value.status == acopf.E_NO_DEVICE
