"""The seeded input generators: counts, connectivity and the two topology
recipes."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_2307_16830_gb300 import synth


def _check_network(g, n_bus, n_branch):
    assert g.bus_type.size == n_bus and g.f.size == n_branch
    assert np.all(g.f != g.t)
    lo, hi = np.minimum(g.f, g.t), np.maximum(g.f, g.t)
    assert np.unique(lo.astype(np.int64) * n_bus + hi).size == n_branch  # no parallel lines
    A = sp.coo_matrix((np.ones(n_branch), (g.f, g.t)), shape=(n_bus, n_bus))
    assert connected_components(A, directed=False)[0] == 1


@pytest.mark.parametrize("topology", ["random", "geometric"])
def test_counts_and_connectivity(topology):
    g = synth.make_grid(3000, 4050, 600, seed=5, topology=topology)
    _check_network(g, 3000, 4050)
    again = synth.make_grid(3000, 4050, 600, seed=5, topology=topology)
    assert np.array_equal(g.f, again.f) and np.array_equal(g.t, again.t)


def test_geometric_recipe_is_local():
    """The geometric recipe joins near neighbours: the branches' endpoints
    are, on average, far closer in the plane than random pairs (recomputed
    here from the generator's own draw of the points)."""
    n = 3000
    g = synth.make_grid(n, 4050, 600, seed=6, topology="geometric")
    pts = np.random.default_rng(6).random((n, 2))  # the generator's first draw
    d_branch = np.hypot(*(pts[g.f] - pts[g.t]).T).mean()
    rng = np.random.default_rng(0)
    a, b = rng.integers(0, n, 4000), rng.integers(0, n, 4000)
    d_random = np.hypot(*(pts[a] - pts[b]).T).mean()
    assert d_branch < 0.1 * d_random


def test_geometric_workloads():
    for name in ("10kbus-geo",):
        spec = synth.WORKLOADS[name]
        g = synth.workload_grid(name)
        _check_network(g, spec["n_bus"], spec["n_branch"])


def test_unknown_topology_rejected():
    with pytest.raises(ValueError):
        synth.make_grid(30, 41, 6, seed=1, topology="ring")
