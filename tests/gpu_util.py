"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle under the parity tolerance."""
import numpy as np

import oracle

KEYS = ("f", "grad", "cons", "jac", "hess", "kkt")


def t64(torch, a, dev):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


def alloc_outputs(torch, model, dev, fill=float("nan")):
    """Output buffers pre-filled with NaN, so an entry a kernel forgets to write fails."""
    return {
        "f": torch.full((1,), fill, dtype=torch.float64, device=dev),
        "grad": torch.full((model.n,), fill, dtype=torch.float64, device=dev),
        "cons": torch.full((model.m,), fill, dtype=torch.float64, device=dev),
        "jac": torch.full((model.nnz_jac,), fill, dtype=torch.float64, device=dev),
        "hess": torch.full((model.nnz_hess,), fill, dtype=torch.float64, device=dev),
        "kkt": torch.full((model.nnz_kkt,), fill, dtype=torch.float64, device=dev),
    }


def run_fused(torch, acopf, model, pt, dev, stream=None):
    x, y = t64(torch, pt.x, dev), t64(torch, pt.y, dev)
    sx, ss = t64(torch, pt.sigma_x, dev), t64(torch, pt.sigma_s, dev)
    out = alloc_outputs(torch, model, dev)
    acopf.eval_assemble(model, x, y, pt.obj_weight, sx, ss, pt.delta_w, pt.delta_c,
                        out["f"], out["grad"], out["cons"], out["jac"], out["hess"], out["kkt"],
                        stream=stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def run_separate(torch, acopf, model, pt, dev):
    x, y = t64(torch, pt.x, dev), t64(torch, pt.y, dev)
    sx, ss = t64(torch, pt.sigma_x, dev), t64(torch, pt.sigma_s, dev)
    out = alloc_outputs(torch, model, dev)
    acopf.eval_obj(model, x, out["f"])
    acopf.eval_grad(model, x, out["grad"])
    acopf.eval_cons(model, x, out["cons"])
    acopf.eval_jac_coo(model, x, out["jac"])
    acopf.eval_hess_coo(model, x, y, pt.obj_weight, out["hess"])
    acopf.assemble_condensed_kkt_csr(model, out["hess"], out["jac"], sx, ss, pt.delta_w,
                                     pt.delta_c, out["kkt"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_all(grid, pt):
    ref = oracle.eval_assemble(grid, pt)
    ref["f"] = (np.array([ref["f"][0]]), np.array([ref["f"][1]]))
    return ref


def assert_parity(got, ref, keys=KEYS, label=""):
    """Every entry within |v - o| <= 1e-12 M + 1e-14 (M = oracle magnitude)."""
    for k in keys:
        val, mag = ref[k]
        g = np.asarray(got[k])
        assert g.shape == val.shape, (label, k, g.shape, val.shape)
        ok = oracle.within_tol(g, val, mag)
        if not ok.all():
            bad = np.flatnonzero(~ok)
            i = bad[np.argmax(np.abs(g[bad] - val[bad]) / (mag[bad] + 1e-300))]
            raise AssertionError(
                f"{label} {k}: {bad.size} of {g.size} entries out of tolerance; worst at {i}: "
                f"gpu={g[i]!r} oracle={val[i]!r} magnitude={mag[i]!r}")


def max_rel_err(got, ref, keys=KEYS):
    out = {}
    for k in keys:
        val, mag = ref[k]
        g = np.asarray(got[k])
        out[k] = float(np.max(np.abs(g - val) / (mag + 1e-300))) if g.size else 0.0
    return out
