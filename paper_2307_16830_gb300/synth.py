"""Seeded synthetic power grids and evaluation points.

This module only draws data: network topology, line and bus parameters,
generator costs, and random primal/dual/barrier points at which the NLP
callbacks are evaluated.  It holds none of the method's arithmetic (no power
flow, no derivatives, no assembly), so both the CUDA library and the CPU
oracle may take their inputs from it.

The recipe stands in for the pglib-opf ``goc``/``pegase`` cases the paper
benchmarks (Section V.A), which are not available here:

* topology: a uniformly random recursive spanning tree over a random bus
  permutation, then unique random extra edges (no self-loops, no parallel
  lines) up to the requested branch count; or, for the workloads of the
  sparse factorization ("-geo"), a near-planar network: buses at random
  points of the unit square joined by their Euclidean minimum spanning tree
  and then by random pairs of near neighbours (real transmission networks
  are near-planar, with small separators; the random chords of the first
  recipe give separators of linear size);
* branches: r ~ U(0.001, 0.05), x ~ U(0.01, 0.3), total charging b ~ U(0, 0.1)
  (r, x and b times the workload's impedance and charging scales, 1 unless stated),
  tap 1 except U(0.95, 1.05) on 10 % of branches, shift 0,
  rate_a ~ U(1, 5) p.u., angle-difference limits +-30 degrees;
* buses: Pd ~ U(0, 1) (times the workload's load scale, 1 unless stated),
  Qd = 0.3 Pd, Gs = Bs = 0, Vm in [0.9, 1.1];
* generators at distinct random buses: c2 ~ U(0, 0.1), c1 ~ U(10, 40), c0 = 0,
  Pg in [0, Pmax] with Pmax ~ U(1, 5), Qg in [-Pmax/2, Pmax/2];
  the bus of generator 0 is the (single) reference bus;
* points: x uniform within its bounds (voltage angles, which are unbounded,
  uniform in +-30 degrees; flows of unrated lines uniform in +-1), multipliers
  y ~ N(0, 1), and the barrier diagonals Sigma_x, Sigma_s log-uniform in
  [1e-8, 1e8].

All draws use numpy's PCG64 through ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

REF_BUS_TYPE = 3


@dataclasses.dataclass
class Grid:
    """Raw network data in per-unit, structure-of-arrays form.

    Buses, branches and generators are numbered from 0.  A branch connects
    its from-bus ``f`` to its to-bus ``t``; the tap ratio (0 read as 1) and
    phase shift sit on the from side.
    """

    bus_type: np.ndarray
    Pd: np.ndarray
    Qd: np.ndarray
    Gs: np.ndarray
    Bs: np.ndarray
    Vmin: np.ndarray
    Vmax: np.ndarray
    f: np.ndarray
    t: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    tap: np.ndarray
    shift: np.ndarray
    rate_a: np.ndarray
    angmin: np.ndarray
    angmax: np.ndarray
    gen_bus: np.ndarray
    Pmin: np.ndarray
    Pmax: np.ndarray
    Qmin: np.ndarray
    Qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray
    c0: np.ndarray
    name: str = "grid"

    @property
    def n_bus(self) -> int:
        return int(self.Pd.shape[0])

    @property
    def n_branch(self) -> int:
        return int(self.f.shape[0])

    @property
    def n_gen(self) -> int:
        return int(self.gen_bus.shape[0])

    @property
    def n_ref(self) -> int:
        return int(np.count_nonzero(self.bus_type == REF_BUS_TYPE))

    @property
    def n_var(self) -> int:
        """Length of x: va, vm per bus; pg, qg per generator; p, q per arc."""
        return 2 * self.n_bus + 2 * self.n_gen + 4 * self.n_branch

    @property
    def n_con(self) -> int:
        """Length of g: reference rows, 7 rows per branch, 2 balance rows per bus."""
        return self.n_ref + 7 * self.n_branch + 2 * self.n_bus

    def copy(self) -> "Grid":
        return dataclasses.replace(
            self, **{fl.name: np.array(getattr(self, fl.name), copy=True)
                     for fl in dataclasses.fields(self) if fl.name != "name"})

    def nbytes(self) -> int:
        return sum(getattr(self, fl.name).nbytes
                   for fl in dataclasses.fields(self) if fl.name != "name")


@dataclasses.dataclass
class Point:
    """One evaluation point: primal x, multipliers y, barrier diagonals."""

    x: np.ndarray
    y: np.ndarray
    sigma_x: np.ndarray
    sigma_s: np.ndarray
    obj_weight: float = 1.0
    delta_w: float = 0.0
    delta_c: float = 0.0


def _random_topology(rng: np.random.Generator, n_bus: int, n_branch: int):
    if n_bus < 2:
        raise ValueError("need at least 2 buses")
    if n_branch < n_bus - 1:
        raise ValueError("need at least n_bus - 1 branches for a spanning tree")
    max_edges = n_bus * (n_bus - 1) // 2
    if n_branch > max_edges:
        raise ValueError("more branches than distinct bus pairs")
    perm = rng.permutation(n_bus)
    k = np.arange(1, n_bus, dtype=np.float64)
    parent_pos = np.minimum(np.floor(rng.random(n_bus - 1) * k).astype(np.int64),
                            np.arange(0, n_bus - 1))
    a = perm[1:].astype(np.int64)
    b = perm[parent_pos].astype(np.int64)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keys = lo * n_bus + hi
    need = n_branch - (n_bus - 1)
    while need > 0:
        cand_a = rng.integers(0, n_bus, size=2 * need + 16)
        cand_b = rng.integers(0, n_bus, size=2 * need + 16)
        ok = cand_a != cand_b
        clo = np.minimum(cand_a, cand_b)[ok]
        chi = np.maximum(cand_a, cand_b)[ok]
        ck = clo * n_bus + chi
        _, first = np.unique(ck, return_index=True)
        ck = ck[np.sort(first)]
        ck = ck[~np.isin(ck, keys)][:need]
        keys = np.concatenate([keys, ck])
        need -= ck.shape[0]
    lo = keys // n_bus
    hi = keys % n_bus
    swap = rng.random(keys.shape[0]) < 0.5
    f = np.where(swap, hi, lo)
    t = np.where(swap, lo, hi)
    order = rng.permutation(keys.shape[0])
    return f[order].astype(np.int32), t[order].astype(np.int32)


def _geometric_topology(rng: np.random.Generator, n_bus: int, n_branch: int):
    """Buses at uniform random points of the unit square; the Euclidean
    minimum spanning tree of their 8-nearest-neighbour graph, then extra
    branches drawn uniformly among the remaining pairs of 4-nearest
    neighbours, up to the requested branch count.  Bus numbers carry no
    geometry (the points are drawn in random order)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
    from scipy.spatial import cKDTree

    if n_bus < 10:
        raise ValueError("the geometric recipe needs at least 10 buses")
    if n_branch < n_bus - 1:
        raise ValueError("need at least n_bus - 1 branches for a spanning tree")
    pts = rng.random((n_bus, 2))
    d, nbr = cKDTree(pts).query(pts, k=9)
    rank = np.tile(np.arange(1, 9), n_bus)
    a = np.repeat(np.arange(n_bus), 8)
    b = nbr[:, 1:].ravel()
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keys, first = np.unique(lo.astype(np.int64) * n_bus + hi, return_index=True)
    w, rank = d[:, 1:].ravel()[first], rank[first]
    G = coo_matrix((w + 1e-300, (keys // n_bus, keys % n_bus)), shape=(n_bus, n_bus)).tocsr()
    if connected_components(G, directed=False)[0] != 1:
        raise ValueError("the 8-nearest-neighbour graph of the points is not connected")
    mst = minimum_spanning_tree(G).tocoo()
    tkeys = (np.minimum(mst.row, mst.col).astype(np.int64) * n_bus
             + np.maximum(mst.row, mst.col))
    rest = keys[~np.isin(keys, tkeys) & (rank <= 4)]
    need = n_branch - tkeys.size
    if need > rest.size:
        raise ValueError("more branches than neighbour pairs")
    keys = np.concatenate([tkeys, rng.choice(rest, size=need, replace=False)])
    lo, hi = keys // n_bus, keys % n_bus
    swap = rng.random(keys.shape[0]) < 0.5
    f = np.where(swap, hi, lo)
    t = np.where(swap, lo, hi)
    order = rng.permutation(keys.shape[0])
    return f[order].astype(np.int32), t[order].astype(np.int32)


def make_grid(n_bus: int, n_branch: int, n_gen: int, seed: int,
              name: str | None = None, topology: str = "random",
              load_scale: float = 1.0, impedance_scale: float = 1.0,
              charging_scale: float = 1.0) -> Grid:
    """Synthetic grid with the recipe of the module docstring (topology
    "random", or "geometric": see _geometric_topology); load_scale,
    impedance_scale (r and x) and charging_scale (b) scale the drawn values
    (the same draws)."""
    if not 1 <= n_gen <= n_bus:
        raise ValueError("need 1 <= n_gen <= n_bus")
    rng = np.random.default_rng(seed)
    if topology == "random":
        f, t = _random_topology(rng, n_bus, n_branch)
    elif topology == "geometric":
        f, t = _geometric_topology(rng, n_bus, n_branch)
    else:
        raise ValueError(f"unknown topology {topology!r}")
    nl = f.shape[0]
    r = rng.uniform(0.001, 0.05, nl) * impedance_scale
    x = rng.uniform(0.01, 0.3, nl) * impedance_scale
    b = rng.uniform(0.0, 0.1, nl) * charging_scale
    tap = np.ones(nl)
    tapped = rng.random(nl) < 0.1
    tap[tapped] = rng.uniform(0.95, 1.05, int(tapped.sum()))
    shift = np.zeros(nl)
    rate_a = rng.uniform(1.0, 5.0, nl)
    ang = math.pi / 6.0
    angmin = np.full(nl, -ang)
    angmax = np.full(nl, ang)

    Pd = rng.uniform(0.0, 1.0, n_bus) * load_scale
    Qd = 0.3 * Pd
    Gs = np.zeros(n_bus)
    Bs = np.zeros(n_bus)
    Vmin = np.full(n_bus, 0.9)
    Vmax = np.full(n_bus, 1.1)

    gen_bus = rng.choice(n_bus, size=n_gen, replace=False).astype(np.int32)
    Pmax = rng.uniform(1.0, 5.0, n_gen)
    Pmin = np.zeros(n_gen)
    Qmax = 0.5 * Pmax
    Qmin = -0.5 * Pmax
    c2 = rng.uniform(0.0, 0.1, n_gen)
    c1 = rng.uniform(10.0, 40.0, n_gen)
    c0 = np.zeros(n_gen)

    bus_type = np.ones(n_bus, dtype=np.int32)
    bus_type[gen_bus] = 2
    bus_type[gen_bus[0]] = REF_BUS_TYPE
    return Grid(bus_type=bus_type, Pd=Pd, Qd=Qd, Gs=Gs, Bs=Bs, Vmin=Vmin, Vmax=Vmax,
                f=f, t=t, r=r, x=x, b=b, tap=tap, shift=shift, rate_a=rate_a,
                angmin=angmin, angmax=angmax, gen_bus=gen_bus, Pmin=Pmin, Pmax=Pmax,
                Qmin=Qmin, Qmax=Qmax, c2=c2, c1=c1, c0=c0,
                name=name or f"synthetic-{n_bus}bus-seed{seed}")


def make_edge_case_grid(seed: int = 7) -> Grid:
    """Small grid carrying every structural corner the formulation has.

    Starting from a 24-bus synthetic grid it adds: parallel branches (two and
    three lines between the same buses, in both orientations), a bus with
    three generators, an isolated bus (no branches, one generator), a second
    reference bus, nonzero phase shifts, a tap given as 0 (meaning 1),
    unrated lines (rate_a = 0), and nonzero bus shunts Gs, Bs.
    """
    rng = np.random.default_rng(seed)
    g = make_grid(24, 34, 5, seed)
    nb = g.n_bus + 1                      # bus 24 is isolated
    iso = nb - 1

    def ext(a, v):
        return np.concatenate([a, np.asarray(v, dtype=a.dtype)])

    bus_type = ext(g.bus_type, [1])
    other_ref = int(np.flatnonzero(bus_type != REF_BUS_TYPE)[3])
    bus_type[other_ref] = REF_BUS_TYPE
    Pd = ext(g.Pd, [0.4])
    Qd = ext(g.Qd, [0.1])
    Gs = rng.uniform(-0.05, 0.05, nb)
    Bs = rng.uniform(-0.2, 0.2, nb)
    Vmin = ext(g.Vmin, [0.9])
    Vmax = ext(g.Vmax, [1.1])

    # parallel lines: duplicate branches 0, 1 (reversed) and 2 (twice)
    dup = [0, 1, 2, 2]
    f = ext(g.f, [g.f[0], g.t[1], g.f[2], g.t[2]])
    t = ext(g.t, [g.t[0], g.f[1], g.t[2], g.f[2]])
    nl = f.shape[0]
    r = ext(g.r, rng.uniform(0.001, 0.05, len(dup)))
    x = ext(g.x, rng.uniform(0.01, 0.3, len(dup)))
    b = ext(g.b, rng.uniform(0.0, 0.1, len(dup)))
    tap = ext(g.tap, [1.02, 0.97, 1.0, 0.0])
    tap[5] = 0.0
    tap[6] = 1.04
    shift = np.zeros(nl)
    shift[[3, 6, nl - 2]] = [0.05, -0.08, 0.03]
    rate_a = ext(g.rate_a, rng.uniform(1.0, 5.0, len(dup)))
    rate_a[[4, 9]] = 0.0
    angmin = ext(g.angmin, [-math.pi / 6] * len(dup))
    angmax = ext(g.angmax, [math.pi / 6] * len(dup))

    bus3 = int(g.gen_bus[1])
    gen_bus = ext(g.gen_bus, [bus3, bus3, iso])
    ng = gen_bus.shape[0]
    Pmax = ext(g.Pmax, rng.uniform(1.0, 5.0, 3))
    Pmin = np.zeros(ng)
    Qmax = 0.5 * Pmax
    Qmin = -0.5 * Pmax
    c2 = ext(g.c2, rng.uniform(0.0, 0.1, 3))
    c1 = ext(g.c1, rng.uniform(10.0, 40.0, 3))
    c0 = ext(g.c0, rng.uniform(0.0, 5.0, 3))
    return Grid(bus_type=bus_type, Pd=Pd, Qd=Qd, Gs=Gs, Bs=Bs, Vmin=Vmin, Vmax=Vmax,
                f=f, t=t, r=r, x=x, b=b, tap=tap, shift=shift, rate_a=rate_a,
                angmin=angmin, angmax=angmax, gen_bus=gen_bus, Pmin=Pmin, Pmax=Pmax,
                Qmin=Qmin, Qmax=Qmax, c2=c2, c1=c1, c0=c0,
                name=f"edge-cases-seed{seed}")


def make_star_grid(n_leaves: int = 300, gens_at_hub: int = 260, seed: int = 5) -> Grid:
    """A hub bus joined to every other bus, carrying most generators: one bus
    with hundreds of arcs and generators (wide rows of the KKT matrix)."""
    rng = np.random.default_rng(seed)
    nb = n_leaves + 1
    leaves = np.arange(1, nb, dtype=np.int32)
    flip = rng.random(n_leaves) < 0.5
    f = np.where(flip, leaves, 0).astype(np.int32)
    t = np.where(flip, 0, leaves).astype(np.int32)
    nl = n_leaves
    gen_bus = np.concatenate([np.zeros(gens_at_hub, np.int32),
                              rng.choice(np.arange(1, nb), size=5, replace=False).astype(np.int32)])
    ng = gen_bus.shape[0]
    Pmax = rng.uniform(1.0, 5.0, ng)
    bus_type = np.ones(nb, dtype=np.int32)
    bus_type[0] = REF_BUS_TYPE
    Pd = rng.uniform(0.0, 1.0, nb)
    return Grid(bus_type=bus_type, Pd=Pd, Qd=0.3 * Pd, Gs=np.zeros(nb), Bs=np.zeros(nb),
                Vmin=np.full(nb, 0.9), Vmax=np.full(nb, 1.1), f=f, t=t,
                r=rng.uniform(0.001, 0.05, nl), x=rng.uniform(0.01, 0.3, nl),
                b=rng.uniform(0.0, 0.1, nl), tap=np.ones(nl), shift=np.zeros(nl),
                rate_a=rng.uniform(1.0, 5.0, nl), angmin=np.full(nl, -math.pi / 6),
                angmax=np.full(nl, math.pi / 6), gen_bus=gen_bus, Pmin=np.zeros(ng), Pmax=Pmax,
                Qmin=-0.5 * Pmax, Qmax=0.5 * Pmax, c2=rng.uniform(0.0, 0.1, ng),
                c1=rng.uniform(10.0, 40.0, ng), c0=np.zeros(ng), name=f"star-{n_leaves}")


def scale_loads(grid: Grid, seed: int, lo: float = 0.9, hi: float = 1.1) -> Grid:
    """Load scenario: every bus's Pd (and Qd) scaled by its own U(lo, hi) draw."""
    rng = np.random.default_rng(seed)
    out = grid.copy()
    s = rng.uniform(lo, hi, grid.n_bus)
    out.Pd = grid.Pd * s
    out.Qd = grid.Qd * s
    out.name = f"{grid.name}-load{seed}"
    return out


def make_point(grid: Grid, seed: int, *, obj_weight: float = 1.0,
               delta_w: float = 0.0, delta_c: float = 0.0) -> Point:
    """Random evaluation point.

    x is laid out as [va (n_bus), vm (n_bus), pg (n_gen), qg (n_gen),
    p (2 n_branch), q (2 n_branch)], arcs 0..n_branch-1 being the from ends
    and n_branch..2 n_branch-1 the to ends of the branches.
    """
    rng = np.random.default_rng(seed)
    nb, ng, nl = grid.n_bus, grid.n_gen, grid.n_branch
    ang = math.pi / 6.0
    va = rng.uniform(-ang, ang, nb)
    vm = rng.uniform(grid.Vmin, grid.Vmax)
    pg = rng.uniform(grid.Pmin, grid.Pmax)
    qg = rng.uniform(grid.Qmin, grid.Qmax)
    rate = np.where(grid.rate_a > 0, grid.rate_a, 1.0)
    rate2 = np.concatenate([rate, rate])
    p = rng.uniform(-rate2, rate2)
    q = rng.uniform(-rate2, rate2)
    x = np.concatenate([va, vm, pg, qg, p, q])
    y = rng.standard_normal(grid.n_con)
    sigma_x = 10.0 ** rng.uniform(-8.0, 8.0, grid.n_var)
    sigma_s = 10.0 ** rng.uniform(-8.0, 8.0, grid.n_con)
    return Point(x=x, y=y, sigma_x=sigma_x, sigma_s=sigma_s,
                 obj_weight=obj_weight, delta_w=delta_w, delta_c=delta_c)


# The workloads used by the tests and the benchmark, by size.
WORKLOADS = {
    "30bus": dict(n_bus=30, n_branch=41, n_gen=6, seed=1000),
    "10kbus": dict(n_bus=10_000, n_branch=13_500, n_gen=2_000, seed=1001),
    "80kbus": dict(n_bus=80_000, n_branch=110_000, n_gen=12_000, seed=1002),
    # near-planar networks of the same counts: the workloads of the sparse
    # factorization, whose cost is set by the network's separators
    "10kbus-geo": dict(n_bus=10_000, n_branch=13_500, n_gen=2_000, seed=1011,
                       topology="geometric"),
    "80kbus-geo": dict(n_bus=80_000, n_branch=110_000, n_gen=12_000, seed=1012,
                       topology="geometric"),
    # lightly loaded networks, solvable from the flat start: the workloads of
    # the full interior-point method (at full load the recipe's networks
    # have no feasible point the method finds)
    "30bus-opf": dict(n_bus=30, n_branch=41, n_gen=6, seed=1000, load_scale=0.5),
    "2kbus-opf": dict(n_bus=2000, n_branch=2700, n_gen=400, seed=1011, load_scale=0.1),
    # near-planar networks of short lines (impedance x0.3, charging x0.1):
    # the recipe's draws make every local line electrically long, and those
    # networks have no feasible point at these sizes
    "10kbus-geo-opf": dict(n_bus=10_000, n_branch=13_500, n_gen=2_000, seed=1011,
                           topology="geometric", load_scale=0.1, impedance_scale=0.3,
                           charging_scale=0.1),
    "80kbus-geo-opf": dict(n_bus=80_000, n_branch=110_000, n_gen=12_000, seed=1012,
                           topology="geometric", load_scale=0.1, impedance_scale=0.3,
                           charging_scale=0.1),
}


def workload_grid(name: str) -> Grid:
    spec = WORKLOADS[name]
    return make_grid(spec["n_bus"], spec["n_branch"], spec["n_gen"], spec["seed"],
                     name=f"synthetic-{name}", topology=spec.get("topology", "random"),
                     load_scale=spec.get("load_scale", 1.0),
                     impedance_scale=spec.get("impedance_scale", 1.0),
                     charging_scale=spec.get("charging_scale", 1.0))


def point_seed(grid_seed: int, call_index: int) -> int:
    return grid_seed * 7919 + call_index


def grid_for_size(n_bus: int, seed: int, name: str | None = None) -> Grid:
    """Grid of n_bus buses with the proportions of the workloads above: 1.35
    branches and 0.2 generators per bus (at least a spanning tree, at least
    one generator, at most one branch per bus pair)."""
    n_bus = int(n_bus)
    n_branch = max(n_bus - 1, int(round(1.35 * n_bus)))
    n_branch = min(n_branch, n_bus * (n_bus - 1) // 2)
    n_gen = max(1, int(round(0.2 * n_bus)))
    return make_grid(n_bus, n_branch, n_gen, seed, name=name)


def log_uniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Bus counts drawn log-uniformly in [lo, hi]."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


def stratified_log_uniform_sizes(count: int, lo: int, hi: int) -> np.ndarray:
    """count bus counts at the midpoint quantiles of the log-uniform
    distribution on [lo, hi] (a deterministic, evenly spread sample)."""
    q = (np.arange(count) + 0.5) / count
    return np.rint(np.exp(math.log(lo) + q * (math.log(hi) - math.log(lo)))).astype(np.int64)


# The batch workload: load scenarios of one network plus networks of mixed size.
BATCH_WORKLOAD = dict(n_scenarios=128, scenario_bus=2000, scenario_branch=2700, scenario_gen=400,
                      n_mixed=128, mixed_lo=30, mixed_hi=20000, seed=1003)


def batch_workload(n_scenarios: int = 128, n_mixed: int = 128, seed: int = 1003,
                   scenario_bus: int = 2000, scenario_branch: int = 2700,
                   scenario_gen: int = 400, mixed_lo: int = 30, mixed_hi: int = 20000):
    """Returns (base, scenarios, mixed): the base network, n_scenarios load
    scenarios of it (every bus's Pd and Qd scaled by its own U(0.9, 1.1)) and
    n_mixed networks with log-uniform bus counts in [mixed_lo, mixed_hi]."""
    base = make_grid(scenario_bus, scenario_branch, scenario_gen, seed,
                     name=f"synthetic-{scenario_bus}bus-seed{seed}")
    scenarios = [scale_loads(base, seed * 1000 + k) for k in range(n_scenarios)]
    rng = np.random.default_rng(seed + 1)
    sizes = log_uniform_sizes(rng, n_mixed, mixed_lo, mixed_hi)
    mixed = [grid_for_size(int(nb), seed + 10 + k) for k, nb in enumerate(sizes)]
    return base, scenarios, mixed


def make_iterate(xl, xu, gl, gu, seed: int, *, z_range=(-4.0, 2.0), gap_floor=0.0):
    """Interior iterate of the barrier problem with the right-hand sides of
    its Newton system (random data, the model's bounds given): slack bounds
    sl = gl - r, su = gu + r with r ~ U(1e-4, 1e-2) (the solver's relaxation
    of the constraint bounds, so every equality row has an interior), x and s
    strictly inside their bounds (free components ~ N(0, 1), one-sided ones
    at 10^U(-3, 1) from the bound, boxed ones at U(0.01, 0.99) of the box,
    at least gap_floor from each bound), bound duals 10^U(z_range) at finite
    bounds and 0 at infinite ones, right-hand sides ~ N(0, 1) (0 for absent
    bounds).  Returns a dict keyed like the oracle's Iterate."""
    rng = np.random.default_rng(seed)
    xl, xu, gl, gu = (np.asarray(a, dtype=np.float64) for a in (xl, xu, gl, gu))
    m = gl.shape[0]
    sl = np.where(np.isfinite(gl), gl - rng.uniform(1e-4, 1e-2, m), -np.inf)
    su = np.where(np.isfinite(gu), gu + rng.uniform(1e-4, 1e-2, m), np.inf)

    def inside(lo, hi):
        k = lo.shape[0]
        v = rng.standard_normal(k)
        lf, hf = np.isfinite(lo), np.isfinite(hi)
        off = 10.0 ** rng.uniform(-3.0, 1.0, k) + gap_floor
        t = rng.uniform(0.01, 0.99, k)
        both = lf & hf
        lo0, hi0 = np.where(lf, lo, 0.0), np.where(hf, hi, 0.0)
        v = np.where(lf & ~hf, lo0 + off, v)
        v = np.where(hf & ~lf, hi0 - off, v)
        v = np.where(both, lo0 + t * (hi0 - lo0), v)
        return v

    def duals(b):
        return np.where(np.isfinite(b), 10.0 ** rng.uniform(*z_range, b.shape[0]), 0.0)

    def rhs(b):
        return np.where(np.isfinite(b), rng.standard_normal(b.shape[0]), 0.0)

    x = inside(xl, xu)
    s = inside(sl, su)
    n = xl.shape[0]
    return dict(x=x, s=s, xl=xl, xu=xu, sl=sl, su=su,
                zl_x=duals(xl), zu_x=duals(xu), zl_s=duals(sl), zu_s=duals(su),
                p_x=rng.standard_normal(n), p_s=rng.standard_normal(m),
                p_y=rng.standard_normal(m), p_zl_x=rhs(xl), p_zu_x=rhs(xu),
                p_zl_s=rhs(sl), p_zu_s=rhs(su))
