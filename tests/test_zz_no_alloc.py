"""The allocation-free objective entry point, checked on the GPU.

acopf_objective_noalloc serves callers that may not allocate device memory
(a component inside a host application whose allocator owns the device, a
solver loop under a fixed memory budget): its scratch is a static device
array instead of model-owned memory.  It is checked against the oracle's
objective, the model-based entry point and an exactly rounded host sum
(math.fsum), on sizes from 0 terms to its 2^24 limit, each twice in a row
(the static array keeps the last call's state).  This file is collected
last, so that a run stopping at the first failure has run every other test
first; it passes alone in a fresh process as well.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_16830_gb300 import acopf
    return acopf, torch.device("cuda:0")


@pytest.mark.gpu
def test_noalloc_objective_matches_oracle_and_model_twice_in_a_row():
    acopf, dev = _need_gpu()
    g = synth.workload_grid("10kbus")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731
    c2, c1, c0 = t(g.c2), t(g.c1), t(g.c0)
    with acopf.model_create(g, 0) as m:
        pg0 = 2 * g.n_bus
        for call in range(2):
            pt = synth.make_point(g, 40 + call)
            x = t(pt.x)
            f_model = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            f_static = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            acopf.eval_obj(m, x, f_model)
            acopf.objective_noalloc(g.n_gen, x[pg0:pg0 + g.n_gen], c2, c1, c0, f_static)
            torch.cuda.synchronize()
            a, b = float(f_model.item()), float(f_static.item())
            want, mag = oracle.objective(g, pt.x)
            tol = oracle.TOL_REL * mag + oracle.TOL_ABS
            assert abs(b - want) <= tol, (call, b, want)
            assert abs(a - b) <= tol, (call, a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [0, 1, 300_000, 1 << 24])
def test_noalloc_objective_on_random_arrays_against_an_exact_host_sum(n):
    """n = 2^24 runs the full 1,024-block grid with 64 terms per thread and
    the last block summing 1,024 block partials; n = 0 must write 0."""
    acopf, dev = _need_gpu()
    rng = np.random.default_rng(977 + n)
    pg = rng.uniform(0.0, 5.0, n)
    c2 = rng.uniform(0.0, 0.1, n)
    c1 = rng.uniform(10.0, 40.0, n)
    c0 = rng.uniform(-1.0, 1.0, n)
    want = math.fsum((c2 * pg * pg + c1 * pg + c0).tolist()) if n else 0.0
    mag = float(np.sum(np.abs(c2) * pg * pg + np.abs(c1 * pg) + np.abs(c0)))
    t = lambda a: torch.as_tensor(a, device=dev)  # noqa: E731
    args = [t(a) for a in (pg, c2, c1, c0)] if n else [torch.zeros(1, dtype=torch.float64,
                                                                   device=dev)] * 4
    got = []
    for _ in range(2):                     # the arrival counter must be reset between calls
        f = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        acopf.objective_noalloc(n, *args, f)
        torch.cuda.synchronize()
        got.append(float(f.item()))
    for v in got:
        assert abs(v - want) <= oracle.TOL_REL * mag + oracle.TOL_ABS, (n, v, want)
    assert np.array_equal(np.array(got).view(np.uint64), np.array(got[:1] * 2).view(np.uint64))


def test_noalloc_objective_rejects_sizes_beyond_its_scratch():
    """The size check comes before any device work, so it runs without a GPU."""
    acopf = pytest.importorskip("paper_2307_16830_gb300.acopf",
                                reason="libacopf.so not built (run __graft_entry__.build())")
    for bad in ((1 << 24) + 1, -1):
        with pytest.raises(acopf.AcopfError) as ei:
            acopf.objective_noalloc(bad, 1, 1, 1, 1, 1, stream=0)
        assert ei.value.status == acopf.E_INVALID_ARG
