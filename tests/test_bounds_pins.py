"""Pins of the variable and constraint bounds against hand-derived values.

The bounds are the box constraints of the NLP (Sec. II.A) for the polar
branch-flow AC-OPF model: free voltage angles, data boxes on voltage
magnitudes and generation, +-rate_a on every arc flow, rate_a^2 above the
apparent-power rows, [angmin, angmax] on the angle-difference rows, zero on
the reference, flow-definition and balance rows, and no limit at all where a
line has rate_a <= 0.  The expected values in tests/golden/bounds_*.txt were
written out by hand from those rules (each file shows its derivation); the
mutation tests plant the plausible mistakes in the oracle and check that a
golden file catches each one.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def two_bus_grid():
    """The network of two_bus_lossless.txt."""
    return synth.Grid(
        bus_type=np.array([3, 1], np.int32), Pd=np.array([0.5, 0.8]),
        Qd=np.array([0.15, 0.24]), Gs=np.array([0.1, 0.0]), Bs=np.array([0.0, 0.2]),
        Vmin=np.array([0.9, 0.9]), Vmax=np.array([1.1, 1.1]),
        f=np.array([0], np.int32), t=np.array([1], np.int32), r=np.array([0.0]),
        x=np.array([0.5]), b=np.array([0.2]), tap=np.array([1.0]), shift=np.array([0.0]),
        rate_a=np.array([3.0]), angmin=np.array([-math.pi / 6]), angmax=np.array([math.pi / 6]),
        gen_bus=np.array([0], np.int32), Pmin=np.array([0.0]), Pmax=np.array([3.0]),
        Qmin=np.array([-1.5]), Qmax=np.array([1.5]), c2=np.array([0.5]),
        c1=np.array([10.0]), c0=np.array([1.0]), name="two-bus")


def edge_three_bus_grid():
    """The network of bounds_edge_three_bus.txt: its data rows decide the
    bounds; the electrical data (which the bounds do not depend on) is filled
    with ordinary line and load values."""
    d = read_golden("bounds_edge_three_bus.txt")
    nb, nl, ng = d["bus_type"].size, d["f"].size, d["gen_bus"].size
    i32 = lambda a: a.astype(np.int32)  # noqa: E731
    return synth.Grid(
        bus_type=i32(d["bus_type"]), Pd=np.full(nb, 0.3), Qd=np.full(nb, 0.09),
        Gs=np.zeros(nb), Bs=np.zeros(nb), Vmin=d["Vmin"], Vmax=d["Vmax"],
        f=i32(d["f"]), t=i32(d["t"]), r=np.full(nl, 0.01), x=np.full(nl, 0.1),
        b=np.full(nl, 0.02), tap=d["tap"], shift=np.zeros(nl), rate_a=d["rate_a"],
        angmin=d["angmin"], angmax=d["angmax"], gen_bus=i32(d["gen_bus"]),
        Pmin=d["Pmin"], Pmax=d["Pmax"], Qmin=d["Qmin"], Qmax=d["Qmax"],
        c2=np.full(ng, 0.01), c1=np.full(ng, 20.0), c0=np.zeros(ng), name="edge-three-bus")


CASES = [("bounds_two_bus.txt", two_bus_grid), ("bounds_edge_three_bus.txt", edge_three_bus_grid)]


def same_bounds(got, want):
    """Equal as written, up to the last bit of a squared rating (0.8 * 0.8 in
    FP64 is one ulp above the decimal 0.64); infinities must match in sign."""
    got = np.asarray(got, dtype=np.float64)
    return got.shape == want.shape and bool(np.all(np.isclose(got, want, rtol=4e-16, atol=0.0)))


def golden_mismatches(grid_fn, name):
    """Names of the bound vectors where the oracle disagrees with the file."""
    want = read_golden(name)
    got = oracle.acopf.bounds(grid_fn())
    return [k for k, v in zip(("xl", "xu", "gl", "gu"), got) if not same_bounds(v, want[k])]


@pytest.mark.parametrize("name,grid_fn", CASES, ids=[c[0] for c in CASES])
def test_oracle_bounds_match_hand_derived_values(name, grid_fn):
    assert golden_mismatches(grid_fn, name) == []


def test_golden_sizes_follow_the_layout():
    for name, grid_fn in CASES:
        g = grid_fn()
        L = oracle.layout(g)
        d = read_golden(name)
        assert d["xl"].size == d["xu"].size == L.n == 2 * g.n_bus + 2 * g.n_gen + 4 * g.n_branch
        assert d["gl"].size == d["gu"].size == L.m == g.n_ref + 7 * g.n_branch + 2 * g.n_bus


@pytest.mark.parametrize("name,grid_fn", CASES, ids=[c[0] for c in CASES])
def test_library_bounds_match_hand_derived_values(name, grid_fn):
    acopf = pytest.importorskip("paper_2307_16830_gb300.acopf",
                                reason="libacopf.so not built (run __graft_entry__.build())")
    want = read_golden(name)
    with acopf.model_create(grid_fn(), device=-1) as m:
        got = m.bounds()
    for k, v in zip(("xl", "xu", "gl", "gu"), got):
        assert same_bounds(v, want[k]), k


# ---------------------------------------------------------------------------
# planted mistakes: each must make a golden file disagree
# ---------------------------------------------------------------------------
def _planted(monkeypatch, edit):
    real = oracle.acopf.bounds

    def wrong(grid):
        xl, xu, gl, gu = (np.array(v, copy=True) for v in real(grid))
        edit(grid, oracle.layout(grid), xl, xu, gl, gu)
        return xl, xu, gl, gu

    monkeypatch.setattr(oracle.acopf, "bounds", wrong)


def _caught():
    return any(golden_mismatches(fn, name) for name, fn in CASES)


def test_pin_catches_rating_instead_of_its_square(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        rate = np.where(grid.rate_a > 0, grid.rate_a, np.inf)
        gu[L.SF:L.SF + L.nl] = rate
        gu[L.ST:L.ST + L.nl] = rate
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_finite_limit_on_an_unrated_line(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        rate = np.asarray(grid.rate_a, dtype=np.float64)    # rate_a <= 0 kept as is
        for k in range(4):
            xl[L.P + k * L.nl:L.P + (k + 1) * L.nl] = -np.abs(rate)
            xu[L.P + k * L.nl:L.P + (k + 1) * L.nl] = np.abs(rate)
    _planted(monkeypatch, edit)
    assert golden_mismatches(edge_three_bus_grid, "bounds_edge_three_bus.txt") == ["xl", "xu"]


def test_pin_catches_thermal_square_left_on_an_unrated_line(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        rate = np.asarray(grid.rate_a, dtype=np.float64)
        gu[L.SF:L.SF + L.nl] = rate * rate
        gu[L.ST:L.ST + L.nl] = rate * rate
    _planted(monkeypatch, edit)
    assert golden_mismatches(edge_three_bus_grid, "bounds_edge_three_bus.txt") == ["gu"]


def test_pin_catches_zero_lower_bound_on_thermal_rows(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        gl[L.SF:L.ST + L.nl] = 0.0
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_swapped_angle_limits(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        gl[L.ANG:L.ANG + L.nl] = grid.angmax
        gu[L.ANG:L.ANG + L.nl] = grid.angmin
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_bounded_angles(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        xl[L.VA:L.VA + L.nb] = -math.pi
        xu[L.VA:L.VA + L.nb] = math.pi
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_generator_boxes_swapped_p_for_q(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        xl[L.PG:L.PG + L.ng], xl[L.QG:L.QG + L.ng] = grid.Qmin, grid.Pmin
        xu[L.PG:L.PG + L.ng], xu[L.QG:L.QG + L.ng] = grid.Qmax, grid.Pmax
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_only_from_arcs_limited(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        for base in (L.P, L.Q):
            xl[base + L.nl:base + 2 * L.nl] = -np.inf
            xu[base + L.nl:base + 2 * L.nl] = np.inf
    _planted(monkeypatch, edit)
    assert _caught()


def test_pin_catches_angle_limits_on_the_reference_rows(monkeypatch):
    def edit(grid, L, xl, xu, gl, gu):
        nref = L.PF - L.REF
        gl[L.REF:L.PF] = grid.angmin[:nref]
        gu[L.REF:L.PF] = grid.angmax[:nref]
    _planted(monkeypatch, edit)
    assert _caught()
