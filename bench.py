"""Benchmark: ACOPF evaluate-and-assemble calls per second on GB300.

One step is one call of the fused unit of work of an IPM iteration (objective,
gradient, constraints, sparse Jacobian, Lagrangian Hessian and the condensed
KKT matrix W + Sigma_x + A'DA) on the 80,000-bus / 110,000-branch / 12,000-
generator synthetic grid, at a fresh random point, inputs resident in HBM.
Input and output buffers rotate over 4 sets (about 110 MB each, 4 x 110 MB >
the 129 MB L2), so no call finds its data in L2 from the previous one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(instances shard with no collective): the barrier and max-over-ranks timing
bracket the timed steps and `value` counts the calls of all ranks.
`--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_16830_gb300 import synth  # noqa: E402

METRIC = "eval+KKT-assembly calls/s and % HBM roofline; served p50/p99 vs plain launches"
UNIT = "calls/s"
ROTATE = 4
GRAPH_CALLS = 100  # calls captured in one CUDA graph (rotating over the ROTATE sets)

# Counters of the phase-1 kernel on the 80,000-bus workload from one ncu
# capture (profiles/k_phase1_80kbus.md): DRAM read + write bytes per launch,
# and its executed FP64 arithmetic (FMA counted as 2 flops), valid for the
# kernels.cu whose hash is recorded; the traffic is reported as null once the
# kernel source changes.
PHASE1_NCU = {
    "kernels_sha": "6e6919f740c50987",
    "workload": "80kbus",
    "dram_bytes": 40_916_736 + 35_136_768,
    "fp64_dfma": 6_746_000, "fp64_dadd": 6_944_803, "fp64_dmul": 6_220_000,
}
# FP64 flops of phase 1 per branch (the kernel's arithmetic on the fused
# path without regularisation, bus and generator work folded in), from the
# capture above: (2 dfma + dadd + dmul) / n_branch.
FLOPS_PER_BRANCH = (2 * PHASE1_NCU["fp64_dfma"] + PHASE1_NCU["fp64_dadd"]
                    + PHASE1_NCU["fp64_dmul"]) / 110_000


def kernels_sha() -> str:
    p = os.path.join(ROOT, "paper_2307_16830_gb300", "csrc", "kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank value over all ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world: int, steps: int, ms_max: float) -> float:
    """Calls per second of the whole job: every rank runs `steps` calls."""
    return world * steps / (ms_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                parts = [p.strip() for p in out.stdout.strip().split(",")]
                if len(parts) >= 8:
                    self.samples.append((time.time(), parts))
            except Exception:
                pass
            self._stop.wait(0.1)

    def start(self):
        self._t.start()
        return self

    def stop(self):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(p[0]) for _, p in self.samples if p[0].replace(".", "").isdigit()]
        mx = [float(p[1]) for _, p in self.samples if p[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, p in self.samples:
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# algorithmic bytes and FP64 flops
# ---------------------------------------------------------------------------
def workload_sizes(model, grid):
    nb, nl, ng = grid.n_bus, grid.n_branch, grid.n_gen
    return dict(nb=nb, nl=nl, ng=ng, n=model.n, m=model.m, nnzj=model.nnz_jac,
                nnzh=model.nnz_hess, nnzk=model.nnz_kkt)


def workload_config(args, s, world):
    """The `config` object of both arms (sizes from the model or the oracle)."""
    return {"workload": f"{args.workload}: synthetic grid, {s['nb']} buses, {s['nl']} "
                        f"branches, {s['ng']} generators; one call = obj+grad+cons+jac+"
                        f"hess+condensed KKT at a fresh point",
            "n": s["n"], "m": s["m"], "nnz_jac": s["nnzj"], "nnz_hess": s["nnzh"],
            "nnz_kkt": s["nnzk"], "parallelism": f"replicas x{world}",
            "l2": f"inputs/outputs rotate over {ROTATE} sets of "
                  f"{algorithmic_bytes(s) / 1e6:.0f} MB (> 129 MB L2 together)"}


def algorithmic_bytes(s):
    """Compulsory bytes of one call: inputs read once, model data read once,
    outputs written once (index metadata excluded)."""
    inputs = 8 * (2 * s["n"] + 2 * s["m"])
    model = 72 * s["nl"] + 32 * s["nb"] + 28 * s["ng"]
    outputs = 8 * (1 + s["n"] + s["m"] + s["nnzj"] + s["nnzh"] + s["nnzk"])
    return inputs + model + outputs


def phase1_bytes(s, kkt_arc_gen):
    """Compulsory bytes of the phase-1 launch: branch (f, t, 8 coefficients),
    bus (Pd, Qd) and generator (c2, c1, c0, bus) data; x and Sigma_x read once
    (8 n each); y and Sigma_s of the branch rows (13 per branch) and Sigma_s
    of the balance rows (2 per bus); writes of f, the gradient, all
    constraints, Jacobian and Hessian values, the arc and generator rows of
    M_cond, and the bus diagonal terms left for phase 2 (2 per bus).  Index
    metadata and the slot partials (scratch) are excluded."""
    nb, nl, ng, n, m = s["nb"], s["nl"], s["ng"], s["n"], s["m"]
    reads = 72 * nl + 16 * nb + 28 * ng + 8 * (2 * n + 13 * nl + 2 * nb)
    writes = 8 * (1 + n + m + s["nnzj"] + s["nnzh"] + kkt_arc_gen + 2 * nb)
    return reads + writes


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch

    from paper_2307_16830_gb300 import acopf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    grid = synth.workload_grid(args.workload)
    seed = synth.WORKLOADS[args.workload]["seed"]
    model = acopf.model_create(grid, local)
    acopf.model_set_option(model, acopf.OPT_PDL, args.pdl)
    s = workload_sizes(model, grid)
    stream = torch.cuda.Stream(device=dev)

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    sets = []
    for r in range(ROTATE):
        pt = synth.make_point(grid, synth.point_seed(seed, 1000 * rank + r))
        sets.append(dict(
            x=t(pt.x), y=t(pt.y), sx=t(pt.sigma_x), ss=t(pt.sigma_s),
            f=torch.empty(1, dtype=torch.float64, device=dev),
            grad=torch.empty(model.n, dtype=torch.float64, device=dev),
            cons=torch.empty(model.m, dtype=torch.float64, device=dev),
            jac=torch.empty(model.nnz_jac, dtype=torch.float64, device=dev),
            hess=torch.empty(model.nnz_hess, dtype=torch.float64, device=dev),
            kkt=torch.empty(model.nnz_kkt, dtype=torch.float64, device=dev)))

    def step(k):
        b = sets[k % ROTATE]
        acopf.eval_assemble(model, b["x"], b["y"], 1.0, b["sx"], b["ss"], 0.0, 0.0, b["f"],
                            b["grad"], b["cons"], b["jac"], b["hess"], b["kkt"], stream=stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(local).start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        # keep the GPU busy long enough for the clock sampler to see the load
        soak_end = time.time() + args.soak
        k = 0
        while k < args.warmup or time.time() < soak_end:
            step(k)
            k += 1
            if k % 256 == 0:
                stream.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            step(k)
        e1.record(stream)
        barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, world, dev)
    value = throughput(world, args.steps, ms_max)

    # the same calls replayed from a CUDA graph (GRAPH_CALLS calls per replay)
    graph_ms = None
    if args.graph_replays > 0:
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                for k in range(ROTATE):
                    step(k)
            stream.synchronize()
            with torch.cuda.graph(g, stream=stream):
                for k in range(GRAPH_CALLS):
                    step(k)
            with torch.cuda.stream(stream):
                for _ in range(2):
                    g.replay()
                barrier()
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                for _ in range(args.graph_replays):
                    g.replay()
                g1.record(stream)
                barrier()
            graph_ms = (reduce_max(g0.elapsed_time(g1), world, dev)
                        / (args.graph_replays * GRAPH_CALLS))
            del g
        except RuntimeError as exc:  # report, keep the plain-launch result
            print(f"graph replay not timed: {exc}", file=sys.stderr)
            graph_ms = None

    # per-phase durations (separate pass, events between the phases)
    nprof = max(16, min(args.steps, 512))
    with torch.cuda.stream(stream):
        acopf.profile_begin(model, nprof)
        for k in range(nprof):
            step(k)
        calls, p1, p2, tot = acopf.profile_end(model)
    p1_ms, p2_ms, call_ms = p1 / calls, p2 / calls, tot / calls

    # end to end through the host-buffer pipeline (pinned memory): every step
    # copies its inputs in and all its outputs back; consecutive steps overlap
    e2e = None
    if args.e2e_steps > 0:
        hs = []  # one host set per staging slot, so no two calls in flight share buffers
        for r in range(args.e2e_depth):
            pt = synth.make_point(grid, synth.point_seed(seed, 5000 + 1000 * rank + r))
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
            hs.append(dict(x=pin(pt.x), y=pin(pt.y), sx=pin(pt.sigma_x), ss=pin(pt.sigma_s),
                           out=[torch.empty(nn, dtype=torch.float64).pin_memory() for nn in
                                (1, model.n, model.m, model.nnz_jac, model.nnz_hess,
                                 model.nnz_kkt)]))
        hsn = [{k: (v.numpy() if k != "out" else [o.numpy() for o in v]) for k, v in h.items()}
               for h in hs]
        pipe = acopf.pipeline_create(model, args.e2e_depth)

        def hstep(k):
            b = hsn[k % args.e2e_depth]
            pipe.submit(b["x"], b["y"], 1.0, b["sx"], b["ss"], 0.0, 0.0, *b["out"])

        for k in range(3):
            hstep(k)
        pipe.wait()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            hstep(k)
        pipe.wait()
        barrier()
        dt = reduce_max(time.perf_counter() - t0, world, dev)
        pipe.close()
        h2d = 8 * (2 * model.n + 2 * model.m)
        d2h = 8 * (1 + model.n + model.m + model.nnz_jac + model.nnz_hess + model.nnz_kkt)
        e2e = {"value": throughput(world, args.e2e_steps, 1e3 * dt), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": f"acopf_pipeline_submit (depth {args.e2e_depth}), page-locked host buffers"}
        # the host link's own rate for one call's outputs: a plain page-locked
        # device-to-host copy of the same bytes, timed the same way
        hbuf = torch.empty(d2h // 8, dtype=torch.float64).pin_memory()
        dbuf = torch.empty(d2h // 8, dtype=torch.float64, device=dev)
        for _ in range(3):
            hbuf.copy_(dbuf, non_blocking=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(20):
            hbuf.copy_(dbuf, non_blocking=True)
        torch.cuda.synchronize(dev)
        link = 20 * d2h / (time.perf_counter() - t0) / 1e9
        per_rank = e2e["value"] / world
        e2e["copy_bound"] = {"d2h_gbs_plain_copy": link,
                             "d2h_gbs_achieved": per_rank * d2h / 1e9,
                             "frac": per_rank * d2h / 1e9 / link}
        del hbuf, dbuf

    fp64_rates = acopf.measure_fp64_rates(local)  # G lane-ops/s of fma, add, mul
    rp, _ = model.kkt_structure()
    kkt_bus_rows = int(rp[model.n_bus * 2] - rp[0])
    kkt_arc_gen = model.nnz_kkt - kkt_bus_rows
    res = dict(value=value, ms=ms_max, p1_ms=p1_ms, p2_ms=p2_ms, call_ms=call_ms, e2e=e2e,
               graph_ms=graph_ms,
               clocks=clocks.summary(), sizes=s, fp64_rates=fp64_rates,
               kkt_arc_gen=kkt_arc_gen, gpu=torch.cuda.get_device_name(dev))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    model.close()
    return res


def run_small_workloads(local):
    """Per-call time of the 30-bus and 10,000-bus workloads: plain launches
    and the same calls replayed from a CUDA graph (4 rotating point sets;
    both fit in L2, so these are latency and L2 figures, not HBM ones)."""
    import torch

    from paper_2307_16830_gb300 import acopf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    out = {}
    for name, calls in (("30bus", 2000), ("10kbus", 1000)):
        grid = synth.workload_grid(name)
        seed = synth.WORKLOADS[name]["seed"]
        model = acopf.model_create(grid, local)

        def t(a):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

        sets = []
        for r in range(ROTATE):
            pt = synth.make_point(grid, synth.point_seed(seed, r))
            sets.append([t(pt.x), t(pt.y), t(pt.sigma_x), t(pt.sigma_s)] + [
                torch.empty(k, dtype=torch.float64, device=dev) for k in
                (1, model.n, model.m, model.nnz_jac, model.nnz_hess, model.nnz_kkt)])

        def step(k):
            b = sets[k % ROTATE]
            acopf.eval_assemble(model, b[0], b[1], 1.0, b[2], b[3], 0.0, 0.0, *b[4:],
                                stream=stream)

        with torch.cuda.stream(stream):
            for k in range(50):
                step(k)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(calls):
                step(k)
            e1.record(stream)
            stream.synchronize()
        plain_us = 1e3 * e0.elapsed_time(e1) / calls
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for k in range(GRAPH_CALLS):
                step(k)
        with torch.cuda.stream(stream):
            g.replay()
            stream.synchronize()
            e0.record(stream)
            for _ in range(calls // GRAPH_CALLS):
                g.replay()
            e1.record(stream)
            stream.synchronize()
        graph_us = 1e3 * e0.elapsed_time(e1) / (calls // GRAPH_CALLS * GRAPH_CALLS)
        del g
        out[name] = {"buses": grid.n_bus, "branches": grid.n_branch, "generators": grid.n_gen,
                     "plain_us_per_call": plain_us, "graph_us_per_call": graph_us,
                     "calls_per_s_plain": 1e6 / plain_us, "calls_per_s_graph": 1e6 / graph_us}
        model.close()
    return out


def run_step_bench(args, local):
    """Condensation around M_cond (acopf_condense: Sigma_x, Sigma_s, q_s and
    the condensed right-hand side) and step recovery (acopf_recover_step) on
    the 80,000-bus workload, each timed over calls rotating between 2
    iterates (2 x 160 MB of inputs > L2), against the HBM floor of their
    algorithmic bytes (inputs read once, outputs written once; the Jacobian's
    row and column lists and the row scratch excluded, as index metadata)."""
    import torch

    from paper_2307_16830_gb300 import acopf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    grid = synth.workload_grid("80kbus")
    model = acopf.model_create(grid, local)
    n, m, nj = model.n, model.m, model.nnz_jac

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    pt = synth.make_point(grid, 11)
    jv = torch.empty(nj, dtype=torch.float64, device=dev)
    acopf.eval_jac_coo(model, t(pt.x), jv, stream=stream)
    xl, xu, gl, gu = model.bounds()
    sets = []
    for r in range(2):
        it = {k: t(v) for k, v in synth.make_iterate(xl, xu, gl, gu, 400 + r).items()}
        e = lambda k: torch.empty(k, dtype=torch.float64, device=dev)  # noqa: E731
        sets.append(dict(it=it, dx=t(np.random.default_rng(500 + r).standard_normal(n)),
                         sx=e(n), ss=e(m), qs=e(m), rhs=e(n), ds=e(m), dy=e(m), zlx=e(n),
                         zux=e(n), zls=e(m), zus=e(m)))

    def condense(k):
        b = sets[k % 2]
        acopf.condense(model, b["it"], jv, 0.0, 0.0, b["sx"], b["ss"], b["qs"], b["rhs"],
                       stream=stream)

    def recover(k):
        b = sets[k % 2]
        acopf.recover_step(model, b["it"], jv, 0.0, 0.0, b["ss"], b["qs"], b["dx"], b["ds"],
                           b["dy"], b["zlx"], b["zux"], b["zls"], b["zus"], stream=stream)

    def timed(fn, reps=200):
        with torch.cuda.stream(stream):
            for k in range(10):
                fn(k)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(reps):
                fn(k)
            e1.record(stream)
            stream.synchronize()
        return 1e3 * e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        condense(0)
        recover(0)
    c_us = timed(condense)
    r_us = timed(recover)
    y = t(np.random.default_rng(600).standard_normal(m))
    grad = torch.empty(n, dtype=torch.float64, device=dev)
    cons = torch.empty(m, dtype=torch.float64, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        acopf.eval_grad(model, sets[0]["it"]["x"], grad, stream=stream)
        acopf.eval_cons(model, sets[0]["it"]["x"], cons, stream=stream)

    def residual(k):
        b = sets[k % 2]
        acopf.kkt_residual(model, b["it"], y, grad, cons, jv, 0.1, res, stream=stream)

    e_us = timed(residual)
    hbm = 6772.9
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    c_bytes = 8 * (10 * n + 11 * m + nj)
    r_bytes = 8 * (10 * n + 14 * m + nj)
    e_bytes = 8 * (6 * n + 8 * m + nj)  # x, bounds, duals, grad (n); s, bounds, duals, y, g (m); J
    model.close()
    return {
        "workload": "80kbus: condensation (Sigma_x, Sigma_s, q_s, rhs = q_x + A'(C q_s + D q_y)), "
                    "step recovery (ds, dy, 4 bound-dual steps) and the scaled KKT residual "
                    "at an interior iterate",
        "condense_us": c_us, "condense_bytes": c_bytes,
        "condense_gbs": c_bytes / (c_us * 1e-6) / 1e9,
        "condense_frac_hbm": c_bytes / (c_us * 1e-6) / 1e9 / hbm,
        "recover_us": r_us, "recover_bytes": r_bytes,
        "recover_gbs": r_bytes / (r_us * 1e-6) / 1e9,
        "recover_frac_hbm": r_bytes / (r_us * 1e-6) / 1e9 / hbm,
        "residual_us": e_us, "residual_bytes": e_bytes,
        "residual_gbs": e_bytes / (e_us * 1e-6) / 1e9,
        "residual_frac_hbm": e_bytes / (e_us * 1e-6) / 1e9 / hbm,
        "launches": {"condense": 2, "recover": 1, "residual": 1},
    }


def run_chol_bench(args, local):
    """Sparse Cholesky of M_cond (acopf_chol_*) on the near-planar 10,000- and
    80,000-bus workloads: the host symbolic phase once, then the numeric
    factorization (zeroing and assembly of the supernodal blocks, the bottom
    levels one thread per supernode, then one persistent task-graph launch;
    the pivot test returned to the host) and the solve (permutation, bottom
    levels, warp and block task launches each way, permutation back), M_cond
    assembled by the library at a convex point (no constraint multipliers,
    delta_w = 1e-4: positive definite)."""
    import time

    import torch

    from paper_2307_16830_gb300 import acopf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    out = {}
    reps = max(1, args.chol_reps)
    warm = 3 if reps >= 10 else 1
    for name in args.chol_workloads:
        grid = synth.workload_grid(name)
        model = acopf.model_create(grid, local)
        n, m = model.n, model.m
        pt = synth.make_point(grid, 90)
        rng = np.random.default_rng(91)

        def t(a):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

        bufs = {k: torch.empty(c, dtype=torch.float64, device=dev) for k, c in
                (("f", 1), ("g", n), ("c", m), ("j", model.nnz_jac), ("h", model.nnz_hess),
                 ("k", model.nnz_kkt))}
        with torch.cuda.stream(stream):
            acopf.eval_assemble(model, t(pt.x), torch.zeros(m, dtype=torch.float64, device=dev),
                                1.0, t(10.0 ** rng.uniform(-2, 2, n)),
                                t(10.0 ** rng.uniform(-2, 2, m)), 1e-4, 0.0, bufs["f"],
                                bufs["g"], bufs["c"], bufs["j"], bufs["h"], bufs["k"],
                                stream=stream)
        stream.synchronize()
        t0 = time.perf_counter()
        ch = acopf.chol_create(model)
        create_s = time.perf_counter() - t0
        info = ch.info()
        for _ in range(warm):
            assert ch.factor(bufs["k"], stream=stream) == -1
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            ch.factor(bufs["k"], stream=stream)
        factor_ms = 1e3 * (time.perf_counter() - t0) / reps
        b = t(rng.standard_normal(n))
        x = torch.empty(n, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(warm):
                ch.solve(b, x, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ch.solve(b, x, stream=stream)
            e1.record(stream)
        stream.synchronize()
        solve_ms = e0.elapsed_time(e1) / reps
        ch.close()
        model.close()
        out[name] = {**{k: info[k] for k in ("n", "nnz_factor", "max_col", "n_supernodes",
                                             "n_levels", "storage")},
                     "factor_gflop": info["factor_flops"] / 1e9, "symbolic_s": create_s,
                     "factor_ms": factor_ms,
                     "factor_gflops": info["factor_flops"] / (factor_ms * 1e-3) / 1e9,
                     "solve_ms": solve_ms, "device_bytes": info["device_bytes"],
                     "factor_tasks": info["factor_tasks"],
                     "launches": {"factor": info["factor_launches"],
                                  "solve": info["solve_launches"]}}
    out["timing"] = (f"factor: host wall clock per call over {reps} calls (each call returns the "
                     f"pivot test to the host); solve: CUDA events over {reps} calls")
    return out


def run_ipm_bench(args, local):
    """The full condensed-space interior-point method (acopf_ipm_solve,
    Algorithm 1, tol 1e-4) on the lightly loaded workloads: the 30- and
    2,000-bus random networks and the 10,000- and 80,000-bus near-planar
    short-line networks (the last at most --ipm-iters iterations).  Host wall
    time of each call, its setup (the symbolic phase of the factorization)
    reported apart."""
    import torch

    from paper_2307_16830_gb300 import acopf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    names = {0: "converged", 1: "max_iter", 2: "line search failed", 3: "inertia correction failed",
             4: "infeasible"}
    out = {}
    for name, max_iter in (("30bus-opf", 200), ("2kbus-opf", 200), ("10kbus-geo-opf", 200),
                           ("80kbus-geo-opf", args.ipm_iters)):
        model = acopf.model_create(synth.workload_grid(name), local)
        res, _, hist = acopf.ipm_solve(model, tol=1e-4, max_iter=max_iter, stream=stream)
        kept = None
        if name == "80kbus-geo-opf":  # a second solve with a Cholesky object the caller keeps
            ch = acopf.chol_create(model)
            try:
                kept, _, _ = acopf.ipm_solve(model, tol=1e-4, max_iter=max_iter, stream=stream,
                                             chol=ch)
            finally:
                ch.close()
        model.close()
        it = max(res["iterations"], 1)
        out[name] = {"status": names.get(res["status"], res["status"]),
                     "iterations": res["iterations"], "seconds": res["seconds"],
                     "setup_seconds": res["setup_seconds"],
                     "ms_per_iteration": 1e3 * (res["seconds"] - res["setup_seconds"]) / it,
                     "factorizations": res["factorizations"], "trial_points": res["trial_points"],
                     "objective": res["objective"], "residual": res["residual"]}
        if kept is not None:
            out[name]["kept_cholesky"] = {"seconds": kept["seconds"],
                                          "setup_seconds": kept["setup_seconds"],
                                          "iterations": kept["iterations"],
                                          "objective": kept["objective"]}
    out["timing"] = ("host wall time of acopf_ipm_solve; ms_per_iteration excludes the setup "
                     "(symbolic phase of the factorization, allocation, initial point); "
                     "kept_cholesky: a repeated solve through acopf_ipm_solve_chol with a "
                     "Cholesky object created once for the network (its symbolic phase outside "
                     "the solve)")
    return out


def _pinned(torch, a):
    """Page-locked host copy of a numpy array (numpy view, torch owner)."""
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t.numpy(), t


def run_batch_bench(args, local):
    """Batched form: the batch workload (128 load scenarios of one 2,000-bus
    network on one shared model + 128 networks of 30..20,000 buses) in one
    autotuned batched evaluation, against the same 256 instances as plain
    single-instance calls on the same stream."""
    import torch

    from paper_2307_16830_gb300 import acopf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    base, scen, mixed = synth.batch_workload()
    base_m = acopf.model_create(base, local)
    mixed_m = [acopf.model_create(g, local) for g in mixed]
    scen_m = [acopf.model_create(g, local) for g in scen]  # the plain path has no load override

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    ios = []
    nb = nl = ng = 0
    for k, g in enumerate(scen + mixed):
        m = base_m if k < len(scen) else mixed_m[k - len(scen)]
        pt = synth.make_point(g, synth.point_seed(1003 * 1000 + k, 0))
        d = dict(x=t(pt.x), y=t(pt.y), sigma_x=t(pt.sigma_x), sigma_s=t(pt.sigma_s),
                 obj_weight=1.0, delta_w=0.0, delta_c=0.0,
                 f=torch.empty(1, dtype=torch.float64, device=dev),
                 grad=torch.empty(m.n, dtype=torch.float64, device=dev),
                 cons=torch.empty(m.m, dtype=torch.float64, device=dev),
                 jvals=torch.empty(m.nnz_jac, dtype=torch.float64, device=dev),
                 hvals=torch.empty(m.nnz_hess, dtype=torch.float64, device=dev),
                 kvals=torch.empty(m.nnz_kkt, dtype=torch.float64, device=dev))
        if k < len(scen):
            d["Pd"], d["Qd"] = t(g.Pd), t(g.Qd)
        ios.append(d)
        nb, nl, ng = nb + g.n_bus, nl + g.n_branch, ng + g.n_gen
    count = len(ios)
    batch = acopf.batch_create([base_m] * len(scen) + mixed_m)
    with torch.cuda.stream(stream):
        acopf.batch_set_io(batch, ios, stream=stream)
        best, times = acopf.batch_autotune(batch, reps=args.batch_tune_reps, stream=stream)
    sched, n1, n2, _ = acopf.batch_info(batch)

    def timed(fn, reps, warm=3):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    ms_batch = timed(lambda: acopf.batch_eval_assemble(batch, stream=stream), args.batch_steps)
    plain_models = scen_m + mixed_m

    def plain():
        for m, d in zip(plain_models, ios):
            acopf.eval_assemble(m, d["x"], d["y"], 1.0, d["sigma_x"], d["sigma_s"], 0.0, 0.0,
                                d["f"], d["grad"], d["cons"], d["jvals"], d["hvals"],
                                d["kvals"], stream=stream)

    ms_plain = timed(plain, max(3, args.batch_steps // 10))
    variants = 1  # no shunts and no regularisation in this workload: one phase-1 launch
    out_bytes = sum(8 * (1 + d[k].numel()) for d in ios for k in ("grad", "cons", "jvals",
                                                                  "hvals", "kvals"))
    in_bytes = sum(8 * d[k].numel() for d in ios for k in ("x", "y", "sigma_x", "sigma_s"))
    batch.close()
    for m in [base_m] + mixed_m + scen_m:
        m.close()
    return {
        "workload": f"{len(scen)} load scenarios of one {base.n_bus}-bus network (one model, "
                    f"Pd/Qd per instance) + {len(mixed)} networks of 30..20,000 buses "
                    f"(log-uniform); {nb} buses, {nl} branches, {ng} generators in total",
        "instances": count, "schedule": sched,
        "autotune_ms": {str(k): round(v, 4) for k, v in sorted(times.items())},
        "work_items": {"phase1": n1, "phase2": n2},
        "launches_per_batch": variants + 1,
        "ms_per_batch": ms_batch, "instances_per_s": count / (ms_batch * 1e-3),
        "plain_ms_per_256_calls": ms_plain, "plain_instances_per_s": count / (ms_plain * 1e-3),
        "plain_launches": 2 * count, "speedup_vs_plain": ms_plain / ms_batch,
        "io_bytes_per_batch": in_bytes + out_bytes,
        "io_gbs": (in_bytes + out_bytes) / (ms_batch * 1e-3) / 1e9,
        "fp64_tflops_est": FLOPS_PER_BRANCH * nl / (ms_batch * 1e-3) / 1e12,
    }


def run_serve_bench(args, local):
    """Served form: a Poisson request stream over resident models (24 networks
    whose bus counts are spaced log-uniformly from 30 to 80,000, both ends
    included; a request picks one uniformly, so request sizes are
    log-uniform), each request 50 evaluate+assemble calls at 50 distinct
    random points (the network's 50 point sets, one per call); continuous
    batching against FIFO plain launches, both under a 40 GB device-memory
    budget, at arrival rates 0.1..1.2 x the measured saturation rate.
    Latency = submission to completion (host steady clock)."""
    import torch

    from paper_2307_16830_gb300 import acopf

    rng = np.random.default_rng(2004)
    calls = 50
    sizes = np.rint(np.geomspace(30, 80_000, args.serve_models)).astype(np.int64)
    pool, hold = [], []
    for k, nbus in enumerate(sizes):
        g = synth.grid_for_size(int(nbus), 3000 + k)
        m = acopf.model_create(g, local)
        pts = [synth.make_point(g, synth.point_seed(3000 + k, c)) for c in range(calls)]
        arrs = {}
        for key in ("x", "y", "sigma_x", "sigma_s"):
            arrs[key], own = _pinned(torch, np.stack([getattr(p, key) for p in pts]))
            hold.append(own)
        pool.append((m, arrs))
    R = args.serve_requests
    pick = rng.integers(0, len(pool), R)
    outs = []
    for _ in range(R):
        a, own = _pinned(torch, np.zeros(calls))
        outs.append(a)
        hold.append(own)
    budget = 40 << 30
    names = {acopf.SERVE_CONTINUOUS: "continuous", acopf.SERVE_FIFO: "fifo_plain"}
    # one long-running server per mode, as in service: its memory pool is grown
    # by the warm-up run and reused by every measured run
    servers = {mode: acopf.server_create(local, budget, mode, 256) for mode in names}

    def run(mode, lam):
        arrive = np.cumsum(rng.exponential(1.0 / lam, R)) if lam else np.zeros(R)
        srv = servers[mode]
        st0 = srv.stats()
        tickets = []
        t0 = time.perf_counter()
        for i in range(R):
            wait = arrive[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            m, a = pool[pick[i]]
            tickets.append(srv.submit(m, calls, a["x"], a["y"], a["sigma_x"], a["sigma_s"],
                                      f_calls=outs[i]))
        for tk in tickets:
            if srv.wait(tk, 600.0) != acopf.OK:
                raise RuntimeError("served request failed")
        t1 = time.perf_counter()
        tm = np.array([srv.times(tk) for tk in tickets])  # (admitted, done) after submission
        st = srv.stats()
        for tk in tickets:
            srv.release(tk)
        # the most requests admitted at once (admission-to-done intervals, with the
        # scheduled arrival times as submission times)
        ev = sorted([(arrive[i] + tm[i, 0], 1) for i in range(R)] +
                    [(arrive[i] + tm[i, 1], -1) for i in range(R)], key=lambda e: (e[0], e[1]))
        active = peak = 0
        for _, d in ev:
            active += d
            peak = max(peak, active)
        lat = tm[:, 1]
        return {"lambda_req_s": lam, "p50_ms": float(1e3 * np.percentile(lat, 50)),
                "p99_ms": float(1e3 * np.percentile(lat, 99)),
                "throughput_req_s": R / (t1 - t0), "calls_per_s": R * calls / (t1 - t0),
                "launches": st["launches"] - st0["launches"], "ticks": st["ticks"] - st0["ticks"],
                "peak_active": int(peak)}

    for mode in names:  # warm-up: grows each server's pool to the saturated working set
        run(mode, 0)
    sat = {names[m]: run(m, 0)["throughput_req_s"] for m in names}
    mu = max(sat.values())
    sweep = {names[m]: [] for m in names}
    for frac in args.serve_fracs:
        for mode in names:
            r = run(mode, frac * mu)
            r["lambda_frac"] = frac
            sweep[names[mode]].append(r)
    for srv in servers.values():
        srv.close()
    for m, _ in pool:
        m.close()
    return {"workload": f"{len(pool)} resident networks of {int(sizes.min())}..{int(sizes.max())} "
                        f"buses (log-uniform, mean {sizes.mean():.0f}); {R} requests per rate, "
                        f"{calls} calls each at {calls} distinct random points; budget 40 GB",
            "saturation_req_s": sat, "sweep": sweep}


def cpu_baseline_sample(workload: str, calls: int):
    import oracle
    grid = synth.workload_grid(workload)
    seed = synth.WORKLOADS[workload]["seed"]
    st = oracle.kkt_structure(grid)
    pts = [synth.make_point(grid, synth.point_seed(seed, 9000 + k)) for k in range(calls)]
    t0 = time.perf_counter()
    for pt in pts:
        oracle.eval_assemble(grid, pt, structure=st)
    dt = time.perf_counter() - t0
    return calls / dt, dt


REF_MAX_CALLS = 60  # full oracle calls at most in one reference run (about a second each)


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm: each step is one full oracle
    evaluate-and-assemble call on the benchmark's own workload (the
    80,000-bus grid by default) at a fresh point, on one host core.  At most
    REF_MAX_CALLS calls are timed (and at most 3 untimed ones run first), so
    the run ends within a few minutes; the line reports the calls timed."""
    if rank != 0:
        return
    import oracle
    full = synth.workload_grid(args.workload)
    seed = synth.WORKLOADS[args.workload]["seed"]
    st_full = oracle.kkt_structure(full)
    steps = min(args.steps, REF_MAX_CALLS)
    warm = min(args.warmup, 3)
    pts = [synth.make_point(full, synth.point_seed(seed, 9000 + k)) for k in range(warm + steps)]
    for k in range(warm):
        oracle.eval_assemble(full, pts[k], structure=st_full)
    t0 = time.perf_counter()
    for k in range(steps):
        oracle.eval_assemble(full, pts[warm + k], structure=st_full)
    dt = time.perf_counter() - t0
    value = steps / dt
    L = oracle.layout(full)
    sizes = dict(nb=full.n_bus, nl=full.n_branch, ng=full.n_gen, n=L.n, m=L.m,
                 nnzj=len(oracle.jac_structure(full)[0]), nnzh=len(oracle.hess_structure(full)[0]),
                 nnzk=int(st_full[0][-1]))
    sample_desc = (f"{steps} full {args.workload} oracle calls at fresh points ({dt:.1f} s"
                   + (f"; {args.steps} requested, capped at {REF_MAX_CALLS}" if steps < args.steps
                      else "") + ")")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(args, sizes, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample_desc + "; numpy/scipy FP64, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="80kbus", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="staging slots of the host-buffer pipeline timed as e2e")
    ap.add_argument("--cpu-calls", type=int, default=3)
    ap.add_argument("--pdl", type=int, default=1, choices=[0, 1],
                    help="chain the two phases with programmatic dependent launch")
    ap.add_argument("--soak", type=float, default=1.0,
                    help="seconds of untimed calls (at least --warmup) before timing")
    ap.add_argument("--graph-replays", type=int, default=20,
                    help="also time the calls replayed from a CUDA graph of 100 calls")
    ap.add_argument("--small-workloads", type=int, default=1, choices=[0, 1],
                    help="also time the 30-bus and 10,000-bus workloads (plain and graph)")
    ap.add_argument("--step", type=int, default=1, choices=[0, 1],
                    help="also time the condensation and step recovery (80k workload)")
    ap.add_argument("--chol", type=int, default=1, choices=[0, 1],
                    help="also time the sparse Cholesky of M_cond (10k and 80k workloads)")
    ap.add_argument("--chol-workloads", nargs="+", default=["10kbus-geo", "80kbus-geo"],
                    choices=sorted(synth.WORKLOADS))
    ap.add_argument("--chol-reps", type=int, default=20)
    ap.add_argument("--ipm", type=int, default=1, choices=[0, 1],
                    help="also run the full interior-point method (2k solve, 80k iterations)")
    ap.add_argument("--ipm-iters", type=int, default=200)
    ap.add_argument("--batch", type=int, default=1, choices=[0, 1],
                    help="also time the batched form (256 instances) against plain calls")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-tune-reps", type=int, default=10)
    ap.add_argument("--serve", type=int, default=1, choices=[0, 1],
                    help="also run the served form (Poisson requests, p50/p99)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-models", type=int, default=24)
    ap.add_argument("--serve-fracs", type=float, nargs="+", default=[0.1, 0.3, 0.6, 0.9, 1.2])
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    r = run_ours(args, rank, world, local)
    def leg(enabled, fn):
        """One extra leg on a clean device: Python garbage and PyTorch's cached
        device memory from the previous legs released first."""
        if not (enabled and world == 1):
            return None
        import gc

        import torch
        gc.collect()
        torch.cuda.synchronize(local)
        torch.cuda.empty_cache()
        return fn()

    # the served form first: its latencies depend on the host and on device
    # memory growth, which the other legs would disturb
    serve = leg(args.serve, lambda: run_serve_bench(args, local))
    small = leg(args.small_workloads, lambda: run_small_workloads(local))
    step = leg(args.step, lambda: run_step_bench(args, local))
    chol = leg(args.chol, lambda: run_chol_bench(args, local))
    ipm = leg(args.ipm, lambda: run_ipm_bench(args, local))
    batch = leg(args.batch, lambda: run_batch_bench(args, local))
    if rank != 0:
        return
    cpu = None
    if world == 1 and args.cpu_calls > 0:
        v, dt = cpu_baseline_sample(args.workload, args.cpu_calls)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_calls} full {args.workload} oracle calls ({dt:.1f} s)"}
    s = r["sizes"]
    # roofline of the dominant kernel (phase 1)
    p1_s = r["p1_ms"] * 1e-3
    measured = NCU_MATCH = (PHASE1_NCU["kernels_sha"] == kernels_sha()
                            and PHASE1_NCU["workload"] == args.workload)
    ops = {k: PHASE1_NCU[k] for k in ("fp64_dfma", "fp64_dadd", "fp64_dmul")}
    if measured:
        traffic = PHASE1_NCU["dram_bytes"]
    else:  # scale the captured counts by the branch count
        ops = {k: v * s["nl"] / 110_000 for k, v in ops.items()}
        traffic = None
    flops = 2 * ops["fp64_dfma"] + ops["fp64_dadd"] + ops["fp64_dmul"]
    by1 = phase1_bytes(s, r["kkt_arc_gen"])
    ach_flops = flops / p1_s / 1e12
    r_fma, r_add, r_mul = r["fp64_rates"]
    peak_flops = 2 * r_fma / 1e3
    # FP64 issue bound of this kernel's operation mix (adds and multiplies
    # are one flop per issue, FMAs two, and each has its own measured rate)
    t_mix = (ops["fp64_dfma"] / r_fma + ops["fp64_dadd"] / r_add + ops["fp64_dmul"] / r_mul) / 1e9
    ach_bw = by1 / p1_s / 1e9
    hbm_peak = 6772.9
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    fp64_frac = ach_flops / peak_flops
    hbm_frac = ach_bw / hbm_peak
    roof_common = {"traffic": traffic, "kernel": "k_phase1 (branch, bus-input and generator blocks)",
                   "launch_ms": r["p1_ms"], "fp64_flops_per_launch": flops,
                   "fp64_flops_source": "ncu capture of this kernel" if NCU_MATCH
                   else "per-branch figure of the last ncu capture x branches",
                   "algorithmic_bytes_per_launch": by1}
    if fp64_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": ach_flops, "peak": peak_flops, "unit": "TFLOP/s",
                "frac": fp64_frac, **roof_common,
                "peak_source": "FP64 FMA throughput measured live (acopf_measure_fp64_rates)",
                "fp64_mix_view": {"issue_bound_us": t_mix * 1e6, "frac": t_mix / p1_s,
                                  "rates_gops": {"fma": r_fma, "add": r_add, "mul": r_mul},
                                  "ops_per_launch": ops},
                "hbm_view": {"achieved_gbs": ach_bw, "peak_gbs": hbm_peak, "frac": hbm_frac}}
    else:
        roof = {"bound": "hbm", "achieved": ach_bw, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_frac, **roof_common, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "fp64_view": {"achieved_tflops": ach_flops, "peak_tflops": peak_flops,
                              "frac": fp64_frac, "issue_bound_us": t_mix * 1e6}}
    call_bytes = algorithmic_bytes(s)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, s, world),
        "hbm_roofline_call": {"algorithmic_bytes": call_bytes,
                              "achieved_gbs": call_bytes / (r["ms"] / args.steps * 1e-3) / 1e9,
                              "frac": call_bytes / (r["ms"] / args.steps * 1e-3) / 1e9 / hbm_peak},
        "phases_ms": {"phase1": r["p1_ms"], "phase2": r["p2_ms"], "call": r["call_ms"]},
        "clocks": r["clocks"], "e2e": r["e2e"],
        "gpu_launches": 2 * args.steps, "roofline": roof, "cpu_baseline": cpu,
        "graph": None if r["graph_ms"] is None else {
            "ms_per_call": r["graph_ms"], "calls_per_s": 1e3 / r["graph_ms"],
            "note": f"{GRAPH_CALLS} calls per CUDA graph, {args.graph_replays} replays"},
        "small_workloads": small, "step": step, "chol": chol, "ipm": ipm,
        "gpu": r["gpu"], "batch": batch, "serve": serve,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
