"""GPU tests of the served form: requests over resident models, admitted by
device-memory budget, continuously batched (or run as plain launches in
FIFO mode).

Each request's results must be the same alone and in a mix of co-scheduled
requests, in both modes, and equal to its single-instance calls: the
objective of every call and the last call's gradient, constraints,
Jacobian, Hessian and condensed KKT values, bit for bit; the last call also
within the parity tolerance of the oracle.
"""
import threading
import time

import numpy as np
import pytest

from paper_2307_16830_gb300 import synth

import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIG = 8 << 30


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def acopf():
    from paper_2307_16830_gb300 import acopf as lib
    return lib


class Job:
    """A request: network, model, point sets, load override, outputs."""

    def __init__(self, grid, model, seeds, n_calls, load_override=False, dw=0.0, dc=0.0):
        self.grid, self.model, self.n_calls = grid, model, n_calls
        self.pts = [synth.make_point(grid, s, obj_weight=0.9, delta_w=dw, delta_c=dc)
                    for s in seeds]
        self.load_override, self.dw, self.dc = load_override, dw, dc

    def submit(self, server):
        m = self.model
        stack = lambda k: np.ascontiguousarray(np.stack([getattr(p, k) for p in self.pts]))
        self.out = dict(f_calls=np.full(self.n_calls, np.nan), grad=np.full(m.n, np.nan),
                        cons=np.full(m.m, np.nan), jvals=np.full(m.nnz_jac, np.nan),
                        hvals=np.full(m.nnz_hess, np.nan), kvals=np.full(m.nnz_kkt, np.nan))
        loads = dict(Pd=np.ascontiguousarray(self.grid.Pd), Qd=np.ascontiguousarray(self.grid.Qd)) \
            if self.load_override else {}
        return server.submit(m, self.n_calls, stack("x"), stack("y"), stack("sigma_x"),
                             stack("sigma_s"), obj_weight=0.9, delta_w=self.dw, delta_c=self.dc,
                             **loads, **self.out)

    def result(self):
        return {k: v.copy() for k, v in self.out.items()}


def jobs(acopf):
    base = synth.make_grid(300, 420, 50, seed=21)
    base_m = acopf.model_create(base, 0)
    out = [Job(base, base_m, (1, 2), 5),
           Job(synth.scale_loads(base, 7), base_m, (3,), 4, load_override=True),
           Job(synth.scale_loads(base, 8), base_m, (4, 5, 6), 7, load_override=True, dw=0.05)]
    models = [base_m]
    for k, (g, dw) in enumerate(((synth.make_edge_case_grid(7), 1e-3),
                                 (synth.make_star_grid(), 0.0),
                                 (synth.make_grid(517, 777, 61, seed=3), 0.0),
                                 (synth.workload_grid("30bus"), 0.0))):
        m = acopf.model_create(g, 0)
        models.append(m)
        out.append(Job(g, m, (10 + k, 20 + k), 3 + k, dw=dw))
    return out, models


def single_calls(acopf, job, dev):
    """The request through plain single-instance calls: f of every call and
    the last call's outputs."""
    if job.load_override:
        m = acopf.model_create(job.grid, 0)
    else:
        m = job.model
    fs, last = [], None
    for c in range(job.n_calls):
        last = gu.run_fused(torch, acopf, m, job.pts[c % len(job.pts)], dev)
        fs.append(last["f"][0])
    if job.load_override:
        m.close()
    return np.array(fs), last


def as_keys(r):
    return {"f_calls": r["f_calls"], "grad": r["grad"], "cons": r["cons"], "jac": r["jvals"],
            "hess": r["hvals"], "kkt": r["kvals"]}


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


def assert_request_equal(got, ref, label):
    for k in got:
        assert same_bits(got[k], ref[k]), f"{label}: {k} differs"


def run_alone(acopf, job, mode):
    with acopf.server_create(0, BIG, mode) as s:
        t = job.submit(s)
        assert s.wait(t, 120.0) == acopf.OK
        return job.result()


def run_mix(acopf, js, mode, stagger_s=0.0):
    """All jobs submitted from two client threads, optionally staggered."""
    with acopf.server_create(0, BIG, mode) as s:
        tickets = [None] * len(js)

        def client(idx):
            for k in idx:
                tickets[k] = js[k].submit(s)
                if stagger_s:
                    time.sleep(stagger_s)

        th = [threading.Thread(target=client, args=(range(i, len(js), 2),)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for t in tickets:
            assert s.wait(t, 120.0) == acopf.OK
        st = s.stats()
        assert st["completed"] == len(js) and st["active"] == 0 and st["bytes_in_use"] == 0
        return [j.result() for j in js], st


def test_served_results_same_alone_and_in_mix(dev, acopf):
    js, models = jobs(acopf)
    direct = [single_calls(acopf, j, dev) for j in js]
    for j, (fs, last) in zip(js, direct):  # the plain path against the oracle
        gu.assert_parity(last, gu.oracle_all(j.grid, j.pts[(j.n_calls - 1) % len(j.pts)]),
                         label=j.grid.name)
    ref = [dict(f_calls=fs, grad=last["grad"], cons=last["cons"], jvals=last["jac"],
                hvals=last["hess"], kvals=last["kkt"]) for fs, last in direct]
    for mode in (acopf.SERVE_CONTINUOUS, acopf.SERVE_FIFO):
        for k, j in enumerate(js):
            assert_request_equal(run_alone(acopf, j, mode), ref[k], f"mode {mode} alone {k}")
        for stagger in (0.0, 0.0005):
            mix, st = run_mix(acopf, js, mode, stagger)
            for k in range(len(js)):
                assert_request_equal(mix[k], ref[k], f"mode {mode} stagger {stagger} mix {k}")
            if mode == acopf.SERVE_CONTINUOUS:
                assert st["ticks"] >= max(j.n_calls for j in js)
                assert st["ticks"] < sum(j.n_calls for j in js)  # calls shared launches
            else:
                assert st["ticks"] == 0
                assert st["launches"] == acopf.launches_per_call(0) * sum(j.n_calls for j in js)
    for m in models:
        m.close()


def test_inflight_option_keeps_results(dev, acopf):
    js, models = jobs(acopf)
    ref = [run_alone(acopf, j, acopf.SERVE_CONTINUOUS) for j in js]
    for depth in (1, 16):
        with acopf.server_create(0, BIG, acopf.SERVE_CONTINUOUS) as s:
            s.set_option(acopf.SERVE_OPT_INFLIGHT, depth)
            tickets = [j.submit(s) for j in js]
            for t in tickets:
                assert s.wait(t, 120.0) == acopf.OK
            for k, j in enumerate(js):
                assert_request_equal(j.result(), ref[k], f"inflight {depth} request {k}")
    # a tick budget of 1 work unit: every tick takes only its longest-admitted
    # request, so the requests run one after another, with the same results
    with acopf.server_create(0, BIG, acopf.SERVE_CONTINUOUS) as s:
        s.set_option(acopf.SERVE_OPT_TICK_WORK, 1)
        tickets = [j.submit(s) for j in js]
        for t in tickets:
            assert s.wait(t, 120.0) == acopf.OK
        for k, j in enumerate(js):
            assert_request_equal(j.result(), ref[k], f"tick work 1 request {k}")
        assert s.stats()["ticks"] == sum(j.n_calls for j in js)
    with acopf.server_create(0, BIG, acopf.SERVE_CONTINUOUS) as s:
        for bad_opt, bad_val in ((acopf.SERVE_OPT_INFLIGHT, 0), (acopf.SERVE_OPT_INFLIGHT, 17),
                                 (acopf.SERVE_OPT_TICK_WORK, 0), (99, 1)):
            with pytest.raises(acopf.AcopfError) as e:
                s.set_option(bad_opt, bad_val)
            assert e.value.status == acopf.E_INVALID_ARG
    for m in models:
        m.close()


def test_admission_respects_budget(dev, acopf):
    js, models = jobs(acopf)
    ref = [run_alone(acopf, j, acopf.SERVE_CONTINUOUS) for j in js]
    with acopf.server_create(0, BIG, acopf.SERVE_CONTINUOUS) as s:
        t = js[0].submit(s)
        s.wait(t)
        one = s.stats()["peak_bytes"]
    budget = int(one * 1.5)  # room for one request of the largest kind, not two
    with acopf.server_create(0, budget, acopf.SERVE_CONTINUOUS) as s:
        tickets = []
        for j in js:
            try:
                tickets.append((j, j.submit(s)))
            except acopf.AcopfError as e:
                assert e.status == acopf.E_BUDGET
        for j, t in tickets:
            assert s.wait(t, 120.0) == acopf.OK
        st = s.stats()
        assert 0 < st["peak_bytes"] <= budget
        assert st["completed"] == len(tickets) >= 4
        for k, (j, t) in enumerate(tickets):
            a, d = s.times(t)
            assert 0.0 <= a <= d
            idx = js.index(j)
            assert_request_equal(j.result(), ref[idx], f"budgeted {idx}")
    with acopf.server_create(0, 4096, acopf.SERVE_CONTINUOUS) as s:
        with pytest.raises(acopf.AcopfError) as e:
            js[0].submit(s)
        assert e.value.status == acopf.E_BUDGET
    for m in models:
        m.close()


def test_max_active_and_timeout(dev, acopf):
    g = synth.workload_grid("10kbus")
    with acopf.model_create(g, 0) as m:
        j = Job(g, m, (1,), 400)
        j2 = Job(g, m, (2,), 3)
        with acopf.server_create(0, BIG, acopf.SERVE_CONTINUOUS, max_active=1) as s:
            t = j.submit(s)
            t2 = j2.submit(s)
            with pytest.raises(acopf.AcopfError) as e:
                s.wait(t2, 0.0)  # queued behind the long request
            assert e.value.status == acopf.E_TIMEOUT
            assert s.wait(t, 120.0) == acopf.OK and s.wait(t2, 120.0) == acopf.OK
            assert s.stats()["peak_active"] == 1
            a2, _ = s.times(t2)
            _, d1 = s.times(t)
            assert a2 > 0.0 and d1 > 0.0
            s.release(t)
            with pytest.raises(acopf.AcopfError):
                s.poll(t)
        with acopf.server_create(0, BIG) as s:
            p = j.pts[0]
            with pytest.raises(acopf.AcopfError) as e:
                s.submit(m, 0, p.x, p.y, p.sigma_x, p.sigma_s)  # n_calls < 1
            assert e.value.status == acopf.E_INVALID_ARG
            with pytest.raises(acopf.AcopfError) as e:
                s.submit(m, 2, p.x, p.y, p.sigma_x, p.sigma_s, delta_c=-1.0)
            assert e.value.status == acopf.E_INVALID_ARG
            with pytest.raises(acopf.AcopfError) as e:
                s.submit(m, 2, p.x, p.y, p.sigma_x, p.sigma_s, Pd=np.asarray(g.Pd, float))
            assert e.value.status == acopf.E_INVALID_ARG
