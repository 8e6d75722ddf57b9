"""GPU tests of the batched form: many instances of the fused evaluation in
one pair of launches.

Every instance's outputs in a batch must be bit-identical to those of its
own single-instance acopf_eval_assemble call (same device code, same data),
under every schedule the autotuner may pick, and within the parity
tolerance of the oracle.  Load scenarios share one model and differ only in
the Pd / Qd they pass; their single-instance reference is a model built from
the scaled network.
"""
import numpy as np
import pytest

from paper_2307_16830_gb300 import synth

import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT_KEYS = ("f", "grad", "cons", "jvals", "hvals", "kvals")
KEY_MAP = {"f": "f", "grad": "grad", "cons": "cons", "jvals": "jac", "hvals": "hess",
           "kvals": "kkt"}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def acopf():
    from paper_2307_16830_gb300 import acopf as lib
    return lib


class Inst:
    """One batch instance: its network (for the oracle and the alone run),
    the model the batch evaluates, an optional load override, a point and
    device buffers."""

    def __init__(self, grid, model, point, load_override=False):
        self.grid, self.model, self.pt = grid, model, point
        self.load_override = load_override

    def alloc(self, dev):
        m, t = self.model, lambda a: gu.t64(torch, a, dev)
        self.inp = {"x": t(self.pt.x), "y": t(self.pt.y), "sigma_x": t(self.pt.sigma_x),
                    "sigma_s": t(self.pt.sigma_s)}
        if self.load_override:
            self.inp["Pd"], self.inp["Qd"] = t(self.grid.Pd), t(self.grid.Qd)
        sizes = {"f": 1, "grad": m.n, "cons": m.m, "jvals": m.nnz_jac, "hvals": m.nnz_hess,
                 "kvals": m.nnz_kkt}
        self.out = {k: torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
                    for k, n in sizes.items()}

    def set_point(self, point, dev):
        self.pt = point
        for k in ("x", "y", "sigma_x", "sigma_s"):
            self.inp[k].copy_(gu.t64(torch, getattr(point, k), dev))

    def io(self):
        d = dict(self.inp)
        d.update(self.out)
        d.update(obj_weight=self.pt.obj_weight, delta_w=self.pt.delta_w, delta_c=self.pt.delta_c)
        return d

    def clear(self):
        for v in self.out.values():
            v.fill_(float("nan"))

    def result(self):
        return {KEY_MAP[k]: v.cpu().numpy() for k, v in self.out.items()}


def bits_equal(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def assert_same_bits(got, alone, label):
    for k in gu.KEYS:
        if not bits_equal(got[k], alone[k]):
            d = np.flatnonzero(got[k].view(np.uint64) != alone[k].view(np.uint64))
            raise AssertionError(f"{label} {k}: {d.size} entries differ from the alone call; "
                                 f"first at {d[0]}: batch={got[k][d[0]]!r} alone={alone[k][d[0]]!r}")


def small_batch(acopf):
    """Mixed instances: 4 uses of one model (base loads and 3 scenarios, one
    regularised), shunts (edge grid, also regularised), a star bus, a
    radial network, a ragged multi-block network, the 30-bus network and a
    2-bus network."""
    base = synth.make_grid(300, 420, 50, seed=21)
    base_m = acopf.model_create(base, 0)
    models = {"base": base_m}
    insts = [Inst(base, base_m, synth.make_point(base, 1))]
    for k in range(3):
        g = synth.scale_loads(base, 100 + k)
        dw, dc = ((0.1, 0.01) if k == 1 else (0.0, 0.0))
        insts.append(Inst(g, base_m, synth.make_point(g, 10 + k, delta_w=dw, delta_c=dc),
                          load_override=True))
    others = [("edge7", synth.make_edge_case_grid(7), 1e-4, 0.0),
              ("star", synth.make_star_grid(), 0.0, 0.0),
              ("tree", synth.make_grid(200, 199, 20, seed=4), 0.0, 0.0),
              ("ragged", synth.make_grid(517, 777, 61, seed=3), 0.0, 0.0),
              ("30bus", synth.workload_grid("30bus"), 0.0, 0.0),
              ("2bus", synth.make_grid(2, 1, 1, seed=9), 0.0, 0.0)]
    for k, (name, g, dw, dc) in enumerate(others):
        m = acopf.model_create(g, 0)
        models[name] = m
        insts.append(Inst(g, m, synth.make_point(g, 20 + k, obj_weight=0.8, delta_w=dw,
                                                 delta_c=dc)))
    return insts, models


def alone_results(acopf, insts, dev):
    """Each instance through its own single-instance call (scenarios on a
    model built from the scaled network)."""
    out = []
    for it in insts:
        if it.load_override:
            with acopf.model_create(it.grid, 0) as m:
                out.append(gu.run_fused(torch, acopf, m, it.pt, dev))
        else:
            out.append(gu.run_fused(torch, acopf, it.model, it.pt, dev))
    return out


def valid_schedules(acopf):
    return [s for s in range(acopf.BATCH_SCHEDULES) if (s & 3) < 3]


def run_batch(acopf, batch, insts):
    for it in insts:
        it.clear()
    acopf.batch_eval_assemble(batch)
    torch.cuda.synchronize()
    return [it.result() for it in insts]


def test_batch_equals_alone_under_every_schedule(dev, acopf):
    insts, models = small_batch(acopf)
    for it in insts:
        it.alloc(dev)
    alone = alone_results(acopf, insts, dev)
    for k, it in enumerate(insts):  # the alone path itself against the oracle
        gu.assert_parity(alone[k], gu.oracle_all(it.grid, it.pt), label=f"alone {k}")
    with acopf.batch_create([it.model for it in insts]) as b:
        acopf.batch_set_io(b, [it.io() for it in insts])
        for s in valid_schedules(acopf):
            acopf.batch_set_schedule(b, s)
            for rep in range(2):  # a graph schedule is captured on the first run, replayed next
                got = run_batch(acopf, b, insts)
                for k in range(len(insts)):
                    assert_same_bits(got[k], alone[k], f"schedule {s} rep {rep} instance {k}")
    for m in models.values():
        m.close()


def test_batch_new_inputs_and_variant_change(dev, acopf):
    """New points through set_io reach a captured graph; a change of code
    variant (delta_w from 0 to nonzero) regroups the work items."""
    insts, models = small_batch(acopf)
    for it in insts:
        it.alloc(dev)
    with acopf.batch_create([it.model for it in insts]) as b:
        acopf.batch_set_io(b, [it.io() for it in insts])
        acopf.batch_set_schedule(b, acopf.SCHED_ORDER_SIZE | acopf.SCHED_PDL | acopf.SCHED_GRAPH)
        run_batch(acopf, b, insts)
        for k, it in enumerate(insts):
            dw = 0.05 if k in (0, 6) else it.pt.delta_w
            it.set_point(synth.make_point(it.grid, 500 + k, obj_weight=1.1, delta_w=dw,
                                          delta_c=it.pt.delta_c), dev)
        acopf.batch_set_io(b, [it.io() for it in insts])
        got = run_batch(acopf, b, insts)
        alone = alone_results(acopf, insts, dev)
        for k, it in enumerate(insts):
            assert_same_bits(got[k], alone[k], f"instance {k}")
            gu.assert_parity(got[k], gu.oracle_all(it.grid, it.pt), label=f"instance {k}")
    for m in models.values():
        m.close()


def test_batch_deterministic_and_autotuned(dev, acopf):
    insts, models = small_batch(acopf)
    for it in insts:
        it.alloc(dev)
    with acopf.batch_create([it.model for it in insts]) as b:
        acopf.batch_set_io(b, [it.io() for it in insts])
        first = run_batch(acopf, b, insts)
        best, times = acopf.batch_autotune(b, reps=3)
        assert best in valid_schedules(acopf)
        assert sorted(times) == valid_schedules(acopf)
        assert all(t > 0 for t in times.values())
        assert times[best] == min(times.values())
        sched, n1, n2, nbytes = acopf.batch_info(b)
        assert sched == best and n1 > 0 and n2 > 0 and nbytes > 0
        again = run_batch(acopf, b, insts)
        for k in range(len(insts)):
            assert_same_bits(again[k], first[k], f"instance {k}")
    for m in models.values():
        m.close()


def test_batch_rejects_bad_arguments(dev, acopf):
    g = synth.workload_grid("30bus")
    with acopf.model_create(g, 0) as m:
        it = Inst(g, m, synth.make_point(g, 1))
        it.alloc(dev)
        with acopf.batch_create([m, m]) as b:
            with pytest.raises(acopf.AcopfError) as e:
                acopf.batch_eval_assemble(b)  # before set_io
            assert e.value.status == acopf.E_INVALID_ARG
            with pytest.raises(acopf.AcopfError) as e:
                acopf.batch_set_io(b, [it.io()])  # count differs
            assert e.value.status == acopf.E_INVALID_ARG
            bad = it.io()
            bad["kvals"] = None
            with pytest.raises(acopf.AcopfError) as e:
                acopf.batch_set_io(b, [it.io(), bad])
            assert e.value.status == acopf.E_INVALID_ARG
            bad = it.io()
            bad["delta_w"] = -1.0
            with pytest.raises(acopf.AcopfError) as e:
                acopf.batch_set_io(b, [it.io(), bad])
            assert e.value.status == acopf.E_INVALID_ARG
            bad = it.io()
            bad["Qd"] = None
            bad["Pd"] = it.inp["x"]
            with pytest.raises(acopf.AcopfError) as e:
                acopf.batch_set_io(b, [it.io(), bad])
            assert e.value.status == acopf.E_INVALID_ARG
            for s in (-1, 3, 7, acopf.BATCH_SCHEDULES):
                with pytest.raises(acopf.AcopfError) as e:
                    acopf.batch_set_schedule(b, s)
                assert e.value.status == acopf.E_INVALID_ARG


def test_batch_workload_256(dev, acopf):
    """The full batch workload (128 load scenarios of a 2,000-bus network on
    one shared model plus 128 networks of 30 to 20,000 buses) under the
    benchmark's autotuned schedule: every instance bit-identical to its alone
    call, sampled instances against the oracle."""
    base, scenarios, mixed = synth.batch_workload()
    base_m = acopf.model_create(base, 0)
    insts = []
    for k, g in enumerate(scenarios):
        insts.append(Inst(g, base_m, synth.make_point(g, synth.point_seed(k, 0)),
                          load_override=True))
    mixed_models = [acopf.model_create(g, 0) for g in mixed]
    for k, (g, m) in enumerate(zip(mixed, mixed_models)):
        insts.append(Inst(g, m, synth.make_point(g, synth.point_seed(1000 + k, 0))))
    for it in insts:
        it.alloc(dev)
    with acopf.batch_create([it.model for it in insts]) as b:
        acopf.batch_set_io(b, [it.io() for it in insts])
        acopf.batch_autotune(b, reps=3)
        got = run_batch(acopf, b, insts)
    # alone calls, one instance at a time
    with acopf.model_create(scenarios[0], 0) as m0:
        for k, it in enumerate(insts):
            model = m0 if k == 0 else None
            if it.load_override and k > 0:
                with acopf.model_create(it.grid, 0) as mk:
                    alone = gu.run_fused(torch, acopf, mk, it.pt, dev)
            else:
                alone = gu.run_fused(torch, acopf, model or it.model, it.pt, dev)
            assert_same_bits(got[k], alone, f"instance {k} ({it.grid.n_bus} buses)")
    sizes = np.array([it.grid.n_bus for it in insts])
    sample = [0, 127] + list(128 + np.argsort(sizes[128:])[:3])
    for k in sample:
        gu.assert_parity(got[k], gu.oracle_all(insts[k].grid, insts[k].pt), label=f"instance {k}")
    for m in mixed_models:
        m.close()
    base_m.close()


def test_one_model_on_two_streams_through_batches(dev, acopf):
    """A model's own calls share its scratch; concurrent evaluations of one
    model on several streams go through batches, each with its own scratch:
    two one-instance batches of the same model, evaluated concurrently on
    two streams, give the results of sequential single-instance calls."""
    g = synth.make_grid(517, 777, 61, seed=3)
    with acopf.model_create(g, 0) as m:
        insts = [Inst(g, m, synth.make_point(g, 300 + k)) for k in range(2)]
        for it in insts:
            it.alloc(dev)
        alone = [gu.run_fused(torch, acopf, m, it.pt, dev) for it in insts]
        streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        batches = [acopf.batch_create([m]) for _ in range(2)]
        for b, it, s in zip(batches, insts, streams):
            acopf.batch_set_io(b, [it.io()], stream=s)
        torch.cuda.synchronize()
        for rep in range(20):
            for b, s in zip(batches, streams):
                acopf.batch_eval_assemble(b, stream=s)
        torch.cuda.synchronize()
        for k, it in enumerate(insts):
            assert_same_bits(it.result(), alone[k], f"stream {k}")
        for b in batches:
            b.close()
