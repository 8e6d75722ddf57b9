"""The symbolic phase of the sparse Cholesky factorization of M_cond (host
code, run through acopf_chol_analyze on host-only models), checked against
a dense structural elimination of the reordered pattern."""
import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import acopf, synth


def _dense_counts(S):
    """Column counts of the Cholesky factor of the boolean pattern S
    (structural elimination: column j's pattern joins every later column it
    touches)."""
    S = S.copy()
    n = S.shape[0]
    counts = np.zeros(n, dtype=np.int64)
    for j in range(n):
        rows = np.flatnonzero(S[j + 1:, j]) + j + 1
        counts[j] = rows.size
        if rows.size:
            S[np.ix_(rows, rows)] = True
    return counts


def _pattern(g):
    L = oracle.layout(g)
    rp, ci = oracle.kkt_structure(g)
    kv = np.ones(ci.size)
    return L, oracle.condensed_matrix(g, kv).toarray() != 0


CASES = [("30bus", lambda: synth.workload_grid("30bus")),
         ("edge7", lambda: synth.make_edge_case_grid(7)),
         ("star", lambda: synth.make_star_grid()),
         ("ragged", lambda: synth.make_grid(517, 777, 61, seed=3)),
         ("geo", lambda: synth.make_grid(400, 540, 80, seed=9, topology="geometric"))]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_counts_match_a_dense_elimination(idx):
    name, make = CASES[idx]
    g = make()
    L, S = _pattern(g)
    with acopf.model_create(g, -1) as m:
        st, p = acopf.chol_analyze(m, with_perm=True)
    assert np.array_equal(np.sort(p), np.arange(L.n)), name
    c = _dense_counts(S[np.ix_(p, p)])
    assert st["n"] == L.n and st["nnz_full"] == int(S.sum())
    assert st["nnz_factor"] == L.n + int(c.sum()), name
    assert st["max_col"] == int(c.max()) + 1
    flops = float(np.sum(1.0 + c + c * (c + 1.0)))
    assert abs(st["factor_flops"] - flops) <= 1e-12 * flops
    assert 1 <= st["n_levels"] <= st["n_supernodes"] <= L.n
    # the blocks hold every entry of L (and the upper triangles of their
    # diagonal blocks)
    assert st["storage"] >= st["nnz_factor"]


def test_order_reduces_fill():
    """Minimum degree beats the natural order of the variables by a wide
    margin on a meshed network."""
    g = synth.make_grid(400, 540, 80, seed=9, topology="geometric")
    L, S = _pattern(g)
    with acopf.model_create(g, -1) as m:
        st = acopf.chol_analyze(m)
    natural = L.n + int(_dense_counts(S).sum())
    assert st["nnz_factor"] < 0.5 * natural


def test_order_is_deterministic():
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, -1) as m:
        a = acopf.chol_analyze(m, with_perm=True)
        b = acopf.chol_analyze(m, with_perm=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_geometric_workload_has_a_small_factor():
    """The near-planar 10,000-bus workload's factor stays within a few times
    the size of M_cond (the random-chord workloads' does not)."""
    g = synth.workload_grid("10kbus-geo")
    with acopf.model_create(g, -1) as m:
        st = acopf.chol_analyze(m)
    assert st["nnz_factor"] < 2 * st["nnz_full"]
    assert st["n_levels"] < 200
    # the task plan: after the assembly and the bottom levels (one launch
    # each), one warp-task and one block-task launch; the solve: permutation,
    # bottom levels, warp and block tasks both ways, permutation back
    assert st["factor_tasks"] >= 1
    bottom = st["factor_launches"] - 3
    assert bottom >= 0 and st["solve_launches"] == 2 * bottom + 6
