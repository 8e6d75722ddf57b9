"""The allocation-free objective entry point against the model-based one.

acopf_objective_noalloc serves callers that may not allocate device memory:
its scratch is a static device array instead of model-owned memory.  This
file is collected last, so that a run stopping at the first failure has run
every other test first; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
from paper_2307_16830_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_objective_matches_model_objective_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_16830_gb300 import acopf
    dev = torch.device("cuda:0")
    g = synth.workload_grid("10kbus")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731
    c2, c1, c0 = t(g.c2), t(g.c1), t(g.c0)
    with acopf.model_create(g, 0) as m:
        pg0 = 2 * g.n_bus
        for call in range(2):                       # the static array keeps the last call's state
            pt = synth.make_point(g, 40 + call)
            x = t(pt.x)
            f_model = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            f_static = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            acopf.eval_obj(m, x, f_model)
            acopf.objective_noalloc(g.n_gen, x[pg0:pg0 + g.n_gen], c2, c1, c0, f_static)
            torch.cuda.synchronize()
            a, b = float(f_model.item()), float(f_static.item())
            _, mag = oracle.objective(g, pt.x)
            assert abs(a - b) <= oracle.TOL_REL * mag + oracle.TOL_ABS, (call, a, b)


def test_noalloc_objective_rejects_sizes_beyond_its_scratch():
    from paper_2307_16830_gb300 import acopf
    with pytest.raises(acopf.AcopfError) as ei:
        acopf.objective_noalloc((1 << 24) + 1, 1, 1, 1, 1, 1, stream=0)
    assert ei.value.status == acopf.E_INVALID_ARG
