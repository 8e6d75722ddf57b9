"""Thin ctypes binding of libacopf (include/acopf.h), with the C names.

Argument marshalling only: every computation runs in the CUDA library.
Device arrays are passed as torch tensors (float64, contiguous, on the
model's device) or as raw integer device addresses; streams as
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or None for the
current torch stream.  There is no CPU fallback: if ``libacopf.so`` has not
been built, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libacopf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
        " (the ACOPF kernels have no CPU fallback)")

_lib = C.CDLL(LIB_PATH)

OK = 0
E_INVALID_ARG = -1
E_BAD_MODEL = -2
E_CUDA = -3
E_OOM = -4
E_BUDGET = -5
E_TIMEOUT = -6
E_BUSY = -7
E_NO_DEVICE = -8

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


class Buses(C.Structure):
    _fields_ = [("n", C.c_int32), ("type", _i32p), ("Pd", _f64p), ("Qd", _f64p), ("Gs", _f64p),
                ("Bs", _f64p), ("Vmin", _f64p), ("Vmax", _f64p)]


class Branches(C.Structure):
    _fields_ = [("n", C.c_int32), ("f", _i32p), ("t", _i32p), ("r", _f64p), ("x", _f64p),
                ("b", _f64p), ("tap", _f64p), ("shift", _f64p), ("rate_a", _f64p),
                ("angmin", _f64p), ("angmax", _f64p)]


class Gens(C.Structure):
    _fields_ = [("n", C.c_int32), ("bus", _i32p), ("Pmin", _f64p), ("Pmax", _f64p),
                ("Qmin", _f64p), ("Qmax", _f64p), ("c2", _f64p), ("c1", _f64p), ("c0", _f64p)]


def _sig(name, res, *args):
    fn = getattr(_lib, name)
    fn.restype = res
    fn.argtypes = list(args)
    return fn


_vp = C.c_void_p
_status_string = _sig("acopf_status_string", C.c_char_p, C.c_int32)
_last_error = _sig("acopf_last_error", C.c_char_p)
_model_create = _sig("acopf_model_create", C.c_int32, C.POINTER(Buses), C.POINTER(Branches),
                     C.POINTER(Gens), C.c_int, C.POINTER(_vp))
_model_destroy = _sig("acopf_model_destroy", C.c_int32, _vp)
_model_dims = _sig("acopf_model_dims", C.c_int32, _vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p)
_model_counts = _sig("acopf_model_counts", C.c_int32, _vp, _i32p, _i32p, _i32p, _i32p)
_bounds = _sig("acopf_bounds", C.c_int32, _vp, _vp, _vp, _vp, _vp)
_jac_structure = _sig("acopf_jac_structure", C.c_int32, _vp, _vp, _vp)
_hess_structure = _sig("acopf_hess_structure", C.c_int32, _vp, _vp, _vp)
_kkt_structure = _sig("acopf_kkt_structure", C.c_int32, _vp, _vp, _vp)
_eval_obj = _sig("acopf_eval_obj", C.c_int32, _vp, _vp, _vp, _vp)
_eval_grad = _sig("acopf_eval_grad", C.c_int32, _vp, _vp, _vp, _vp)
_eval_cons = _sig("acopf_eval_cons", C.c_int32, _vp, _vp, _vp, _vp)
_eval_jac_coo = _sig("acopf_eval_jac_coo", C.c_int32, _vp, _vp, _vp, _vp)
_eval_hess_coo = _sig("acopf_eval_hess_coo", C.c_int32, _vp, _vp, _vp, C.c_double, _vp, _vp)
_assemble = _sig("acopf_assemble_condensed_kkt_csr", C.c_int32, _vp, _vp, _vp, _vp, _vp,
                 C.c_double, C.c_double, _vp, _vp)
_eval_assemble = _sig("acopf_eval_assemble", C.c_int32, _vp, _vp, _vp, C.c_double, _vp, _vp,
                      C.c_double, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp)
_eval_assemble_host = _sig("acopf_eval_assemble_host", C.c_int32, _vp, _vp, _vp, C.c_double, _vp,
                           _vp, C.c_double, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp)
_launches_per_call = _sig("acopf_launches_per_call", C.c_int32, C.c_int32)
_model_set_option = _sig("acopf_model_set_option", C.c_int32, _vp, C.c_int32, C.c_int64)
_objective_noalloc = _sig("acopf_objective_noalloc", C.c_int32, C.c_int64, _vp, _vp, _vp, _vp,
                          _vp, _vp)
OPT_PDL = 1
_measure_fp64 = _sig("acopf_measure_fp64_gflops", C.c_int32, C.c_int, _f64p)
_measure_fp64_rates = _sig("acopf_measure_fp64_rates", C.c_int32, C.c_int, _f64p, _f64p, _f64p)
_profile_begin = _sig("acopf_profile_begin", C.c_int32, _vp, C.c_int32)
_profile_end = _sig("acopf_profile_end", C.c_int32, _vp, _i32p, _f64p, _f64p, _f64p)

class BatchIO(C.Structure):
    """One instance's inputs and outputs in a batch (device addresses)."""
    _fields_ = [("x", _vp), ("y", _vp), ("sigma_x", _vp), ("sigma_s", _vp),
                ("obj_weight", C.c_double), ("delta_w", C.c_double), ("delta_c", C.c_double),
                ("Pd", _vp), ("Qd", _vp), ("f", _vp), ("grad", _vp), ("cons", _vp),
                ("jvals", _vp), ("hvals", _vp), ("kvals", _vp)]


SCHED_ORDER_GIVEN = 0
SCHED_ORDER_SIZE = 1
SCHED_ORDER_GROUP = 2
SCHED_PDL = 4
SCHED_GRAPH = 8
SCHED_PERSISTENT = 16
BATCH_SCHEDULES = 32

_batch_create = _sig("acopf_batch_create", C.c_int32, C.POINTER(_vp), C.c_int32, C.POINTER(_vp))
_batch_destroy = _sig("acopf_batch_destroy", C.c_int32, _vp)
_batch_set_io = _sig("acopf_batch_set_io", C.c_int32, _vp, C.POINTER(BatchIO), C.c_int32, _vp)
_batch_eval_assemble = _sig("acopf_batch_eval_assemble", C.c_int32, _vp, _vp)
_batch_set_schedule = _sig("acopf_batch_set_schedule", C.c_int32, _vp, C.c_int32)
_batch_autotune = _sig("acopf_batch_autotune", C.c_int32, _vp, _vp, C.c_int32, _i32p,
                       C.POINTER(C.c_float))
_batch_info = _sig("acopf_batch_info", C.c_int32, _vp, _i32p, _i64p, _i64p, _i64p)

class Request(C.Structure):
    """A served request (host addresses)."""
    _fields_ = [("model", _vp), ("n_calls", C.c_int32), ("n_points", C.c_int32),
                ("x", _vp), ("y", _vp), ("sigma_x", _vp), ("sigma_s", _vp),
                ("obj_weight", C.c_double), ("delta_w", C.c_double), ("delta_c", C.c_double),
                ("Pd", _vp), ("Qd", _vp), ("f_calls", _vp), ("grad", _vp), ("cons", _vp),
                ("jvals", _vp), ("hvals", _vp), ("kvals", _vp)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("ticks", C.c_int64),
                ("launches", C.c_int64), ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64),
                ("active", C.c_int32), ("queued", C.c_int32), ("peak_active", C.c_int32)]


SERVE_CONTINUOUS = 0
SERVE_FIFO = 1

_server_create = _sig("acopf_server_create", C.c_int32, C.c_int, C.c_int64, C.c_int32, C.c_int32,
                      C.POINTER(_vp))
_server_destroy = _sig("acopf_server_destroy", C.c_int32, _vp)
_server_submit = _sig("acopf_server_submit", C.c_int32, _vp, C.POINTER(Request),
                      C.POINTER(C.c_uint64))
_server_poll = _sig("acopf_server_poll", C.c_int32, _vp, C.c_uint64, _i32p, _i32p)
_server_wait = _sig("acopf_server_wait", C.c_int32, _vp, C.c_uint64, C.c_double, _i32p)
_server_times = _sig("acopf_server_request_times", C.c_int32, _vp, C.c_uint64, _f64p, _f64p)
_server_release = _sig("acopf_server_release", C.c_int32, _vp, C.c_uint64)
_server_stats = _sig("acopf_server_get_stats", C.c_int32, _vp, C.POINTER(ServerStats))
_server_set_option = _sig("acopf_server_set_option", C.c_int32, _vp, C.c_int32, C.c_int64)
SERVE_OPT_INFLIGHT = 1
SERVE_OPT_TICK_WORK = 2

_pipeline_create = _sig("acopf_pipeline_create", C.c_int32, _vp, C.c_int32, C.POINTER(_vp))
_pipeline_destroy = _sig("acopf_pipeline_destroy", C.c_int32, _vp)
_pipeline_submit = _sig("acopf_pipeline_submit", C.c_int32, _vp, _vp, _vp, C.c_double, _vp, _vp,
                        C.c_double, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp)
_pipeline_wait = _sig("acopf_pipeline_wait", C.c_int32, _vp)

ITERATE_FIELDS = ("x", "s", "xl", "xu", "sl", "su", "zl_x", "zu_x", "zl_s", "zu_s", "p_x", "p_s",
                  "p_y", "p_zl_x", "p_zu_x", "p_zl_s", "p_zu_s")


class Iterate(C.Structure):
    """An interior iterate and its Newton right-hand sides (device addresses)."""
    _fields_ = [(k, _vp) for k in ITERATE_FIELDS]


_condense = _sig("acopf_condense", C.c_int32, _vp, C.POINTER(Iterate), _vp, C.c_double,
                 C.c_double, _vp, _vp, _vp, _vp, _vp)
_recover_step = _sig("acopf_recover_step", C.c_int32, _vp, C.POINTER(Iterate), _vp, C.c_double,
                     C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp)

_kkt_residual = _sig("acopf_kkt_residual", C.c_int32, _vp, C.POINTER(Iterate), _vp, _vp, _vp,
                     _vp, C.c_double, _vp, _vp)
RESIDUAL_FIELDS = ("residual", "dual_inf", "primal_inf", "compl_inf", "y_l1", "z_l1", "n_z",
                   "s_d", "s_c")

_chol_create = _sig("acopf_chol_create", C.c_int32, _vp, C.POINTER(_vp))
_chol_destroy = _sig("acopf_chol_destroy", C.c_int32, _vp)
_chol_factor = _sig("acopf_chol_factor", C.c_int32, _vp, _vp, C.c_double, C.POINTER(C.c_int32),
                    _vp)
_chol_solve = _sig("acopf_chol_solve", C.c_int32, _vp, _vp, _vp, _vp)


class CholStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_full", C.c_int64), ("nnz_factor", C.c_int64),
                ("max_col", C.c_int64), ("factor_flops", C.c_double),
                ("n_supernodes", C.c_int64), ("n_levels", C.c_int64), ("storage", C.c_int64),
                ("update_storage", C.c_int64), ("factor_tasks", C.c_int64),
                ("factor_launches", C.c_int64), ("solve_launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_chol_info = _sig("acopf_chol_info", C.c_int32, _vp, C.POINTER(CholStats), C.POINTER(C.c_int64))
_chol_analyze = _sig("acopf_chol_analyze", C.c_int32, _vp, C.POINTER(CholStats), _vp)
_chol_permutation = _sig("acopf_chol_permutation", C.c_int32, _vp, _vp)
_chol_set_trace = _sig("acopf_chol_set_trace", C.c_int32, _vp, C.c_int32)
_chol_get_trace = _sig("acopf_chol_get_trace", C.c_int32, _vp, C.c_int32, _vp, C.c_int64,
                       C.POINTER(C.c_int64))

class IpmOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("mu_init", C.c_double)]


class IpmResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("factorizations", C.c_int32),
                ("trial_points", C.c_int32), ("objective", C.c_double), ("residual", C.c_double),
                ("mu", C.c_double), ("seconds", C.c_double), ("setup_seconds", C.c_double)]


IPM_CONVERGED, IPM_MAX_ITER, IPM_LINE_SEARCH_FAILED, IPM_INERTIA_FAILED = 0, 1, 2, 3
IPM_INFEASIBLE = 4
IPM_HISTORY_FIELDS = ("f", "residual", "mu", "theta", "alpha", "alpha_z", "delta_w")
_ipm_solve_chol = _sig("acopf_ipm_solve_chol", C.c_int32, _vp, _vp, C.POINTER(IpmOptions), _vp,
                       _vp, C.POINTER(IpmResult), _vp)
_ipm_solve = _sig("acopf_ipm_solve", C.c_int32, _vp, C.POINTER(IpmOptions), _vp, _vp,
                  C.POINTER(IpmResult), _vp)

# Exported symbols the header declares (checked by the CPU tests).
EXPORTED = [
    "acopf_status_string", "acopf_last_error", "acopf_model_create", "acopf_model_destroy",
    "acopf_model_dims", "acopf_model_counts", "acopf_bounds", "acopf_jac_structure",
    "acopf_hess_structure", "acopf_kkt_structure", "acopf_eval_obj", "acopf_eval_grad",
    "acopf_eval_cons", "acopf_eval_jac_coo", "acopf_eval_hess_coo",
    "acopf_assemble_condensed_kkt_csr", "acopf_eval_assemble", "acopf_eval_assemble_host",
    "acopf_launches_per_call", "acopf_measure_fp64_gflops", "acopf_measure_fp64_rates",
    "acopf_profile_begin",
    "acopf_profile_end", "acopf_model_set_option", "acopf_objective_noalloc",
    "acopf_batch_create", "acopf_batch_destroy", "acopf_batch_set_io",
    "acopf_batch_eval_assemble", "acopf_batch_set_schedule", "acopf_batch_autotune",
    "acopf_batch_info", "acopf_server_create", "acopf_server_destroy", "acopf_server_submit",
    "acopf_server_poll", "acopf_server_wait", "acopf_server_request_times",
    "acopf_server_release", "acopf_server_get_stats", "acopf_server_set_option",
    "acopf_pipeline_create", "acopf_pipeline_destroy", "acopf_pipeline_submit",
    "acopf_pipeline_wait", "acopf_condense", "acopf_recover_step", "acopf_kkt_residual",
    "acopf_chol_create", "acopf_chol_destroy", "acopf_chol_factor", "acopf_chol_solve",
    "acopf_chol_info", "acopf_chol_permutation", "acopf_chol_analyze", "acopf_ipm_solve",
    "acopf_ipm_solve_chol",
    "acopf_chol_set_trace", "acopf_chol_get_trace",
]


class AcopfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _last_error().decode(errors="replace")
        super().__init__(f"{where}: {status_string(status)}: {msg}")


def status_string(status: int) -> str:
    return _status_string(status).decode()


def last_error() -> str:
    return _last_error().decode(errors="replace")


def _check(status: int, where: str) -> None:
    if status != OK:
        raise AcopfError(status, where)


def _ptr(a) -> int | None:
    """Device address of a tensor (or an int address, or None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"expected a tensor or a device address, got {type(a)!r}")


def _hptr(a: np.ndarray | None):
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host array must be C-contiguous")
    return a.ctypes.data


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream or None
        except Exception:  # no torch / no CUDA: legacy default stream
            return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


class Model:
    """An ACOPF model (owner of an ``acopf_model*``)."""

    def __init__(self, handle: int, keepalive):
        self._h = C.c_void_p(handle)
        self._keep = keepalive
        n, m, nj, nh, nk, db = (C.c_int64() for _ in range(6))
        _check(_model_dims(self._h, C.byref(n), C.byref(m), C.byref(nj), C.byref(nh),
                           C.byref(nk), C.byref(db)), "acopf_model_dims")
        self.n, self.m = n.value, m.value
        self.nnz_jac, self.nnz_hess, self.nnz_kkt = nj.value, nh.value, nk.value
        nb, nl, ng, nr = (C.c_int32() for _ in range(4))
        _check(_model_counts(self._h, C.byref(nb), C.byref(nl), C.byref(ng), C.byref(nr)),
               "acopf_model_counts")
        self.n_bus, self.n_branch, self.n_gen, self.n_ref = nb.value, nl.value, ng.value, nr.value

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    @property
    def device_bytes(self) -> int:
        db = C.c_int64()
        _check(_model_dims(self._h, None, None, None, None, None, C.byref(db)), "acopf_model_dims")
        return db.value

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _model_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- host queries --------------------------------------------------------
    def bounds(self):
        xl, xu = np.empty(self.n), np.empty(self.n)
        gl, gu = np.empty(self.m), np.empty(self.m)
        _check(_bounds(self._h, _hptr(xl), _hptr(xu), _hptr(gl), _hptr(gu)), "acopf_bounds")
        return xl, xu, gl, gu

    def jac_structure(self):
        r, c = np.empty(self.nnz_jac, np.int32), np.empty(self.nnz_jac, np.int32)
        _check(_jac_structure(self._h, _hptr(r), _hptr(c)), "acopf_jac_structure")
        return r, c

    def hess_structure(self):
        r, c = np.empty(self.nnz_hess, np.int32), np.empty(self.nnz_hess, np.int32)
        _check(_hess_structure(self._h, _hptr(r), _hptr(c)), "acopf_hess_structure")
        return r, c

    def kkt_structure(self):
        rp, ci = np.empty(self.n + 1, np.int32), np.empty(self.nnz_kkt, np.int32)
        _check(_kkt_structure(self._h, _hptr(rp), _hptr(ci)), "acopf_kkt_structure")
        return rp, ci


def _as(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def model_create(grid, device: int = 0) -> Model:
    """acopf_model_create from a grid object exposing the bus, branch and
    generator arrays (see ``synth.Grid``); device = -1 builds a host-only
    model (structure queries only)."""
    keep = {}

    def f64(name):
        keep[name] = _as(getattr(grid, name), np.float64)
        return keep[name].ctypes.data_as(_f64p)

    def i32(name):
        keep[name] = _as(getattr(grid, name), np.int32)
        return keep[name].ctypes.data_as(_i32p)

    nb, nl, ng = len(grid.Pd), len(grid.f), len(grid.gen_bus)
    buses = Buses(nb, i32("bus_type"), f64("Pd"), f64("Qd"), f64("Gs"), f64("Bs"), f64("Vmin"),
                  f64("Vmax"))
    branches = Branches(nl, i32("f"), i32("t"), f64("r"), f64("x"), f64("b"), f64("tap"),
                        f64("shift"), f64("rate_a"), f64("angmin"), f64("angmax"))
    gens = Gens(ng, i32("gen_bus"), f64("Pmin"), f64("Pmax"), f64("Qmin"), f64("Qmax"),
                f64("c2"), f64("c1"), f64("c0"))
    h = C.c_void_p()
    _check(_model_create(C.byref(buses), C.byref(branches), C.byref(gens), int(device),
                         C.byref(h)), "acopf_model_create")
    return Model(h.value, None)


def eval_obj(model: Model, x, f_dev, stream=None) -> None:
    _check(_eval_obj(model.handle, _ptr(x), _ptr(f_dev), _stream(stream)), "acopf_eval_obj")


def eval_grad(model: Model, x, grad, stream=None) -> None:
    _check(_eval_grad(model.handle, _ptr(x), _ptr(grad), _stream(stream)), "acopf_eval_grad")


def eval_cons(model: Model, x, cons, stream=None) -> None:
    _check(_eval_cons(model.handle, _ptr(x), _ptr(cons), _stream(stream)), "acopf_eval_cons")


def eval_jac_coo(model: Model, x, jvals, stream=None) -> None:
    _check(_eval_jac_coo(model.handle, _ptr(x), _ptr(jvals), _stream(stream)),
           "acopf_eval_jac_coo")


def eval_hess_coo(model: Model, x, y, obj_weight: float, hvals, stream=None) -> None:
    _check(_eval_hess_coo(model.handle, _ptr(x), _ptr(y), float(obj_weight), _ptr(hvals),
                          _stream(stream)), "acopf_eval_hess_coo")


def assemble_condensed_kkt_csr(model: Model, hvals, jvals, sigma_x, sigma_s, delta_w: float,
                               delta_c: float, kvals, stream=None) -> None:
    _check(_assemble(model.handle, _ptr(hvals), _ptr(jvals), _ptr(sigma_x), _ptr(sigma_s),
                     float(delta_w), float(delta_c), _ptr(kvals), _stream(stream)),
           "acopf_assemble_condensed_kkt_csr")


def eval_assemble(model: Model, x, y, obj_weight: float, sigma_x, sigma_s, delta_w: float,
                  delta_c: float, f_dev, grad, cons, jvals, hvals, kvals, stream=None) -> None:
    _check(_eval_assemble(model.handle, _ptr(x), _ptr(y), float(obj_weight), _ptr(sigma_x),
                          _ptr(sigma_s), float(delta_w), float(delta_c), _ptr(f_dev), _ptr(grad),
                          _ptr(cons), _ptr(jvals), _ptr(hvals), _ptr(kvals), _stream(stream)),
           "acopf_eval_assemble")


def eval_assemble_host(model: Model, x, y, obj_weight: float, sigma_x, sigma_s, delta_w: float,
                       delta_c: float, f, grad, cons, jvals, hvals, kvals, stream=None) -> None:
    """Host-buffer variant: numpy arrays (or pinned torch CPU tensors) in and out."""
    def hp(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return _hptr(a)
    _check(_eval_assemble_host(model.handle, hp(x), hp(y), float(obj_weight), hp(sigma_x),
                               hp(sigma_s), float(delta_w), float(delta_c), hp(f), hp(grad),
                               hp(cons), hp(jvals), hp(hvals), hp(kvals), _stream(stream)),
           "acopf_eval_assemble_host")


def launches_per_call(kind: int) -> int:
    return int(_launches_per_call(int(kind)))


def measure_fp64_gflops(device: int = 0) -> float:
    v = C.c_double()
    _check(_measure_fp64(int(device), C.byref(v)), "acopf_measure_fp64_gflops")
    return v.value


def measure_fp64_rates(device: int = 0):
    """(fma, add, mul) lane operations per second, in G/s."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(_measure_fp64_rates(device, C.byref(a), C.byref(b), C.byref(c)),
           "acopf_measure_fp64_rates")
    return a.value, b.value, c.value


def profile_begin(model: Model, capacity: int) -> None:
    _check(_profile_begin(model.handle, int(capacity)), "acopf_profile_begin")


def profile_end(model: Model):
    """Returns (calls, phase1_ms, phase2_ms, total_ms) summed over profiled calls."""
    n = C.c_int32()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(_profile_end(model.handle, C.byref(n), C.byref(a), C.byref(b), C.byref(c)),
           "acopf_profile_end")
    return n.value, a.value, b.value, c.value


def model_set_option(model: Model, option: int, value: int) -> None:
    _check(_model_set_option(model.handle, int(option), int(value)), "acopf_model_set_option")


def objective_noalloc(n_gen: int, pg, c2, c1, c0, f_dev, stream=None) -> None:
    """acopf_objective_noalloc: sum c2 pg^2 + c1 pg + c0 over n_gen device
    doubles, for callers that may not allocate (static scratch, no model)."""
    _check(_objective_noalloc(int(n_gen), _ptr(pg), _ptr(c2), _ptr(c1), _ptr(c0), _ptr(f_dev),
                              _stream(stream)), "acopf_objective_noalloc")


class Batch:
    """A batch of instances (owner of an ``acopf_batch*``); the models must
    outlive it."""

    def __init__(self, models):
        self.models = list(models)
        arr = (_vp * len(self.models))(*[m.handle.value for m in self.models])
        h = _vp()
        _check(_batch_create(arr, len(self.models), C.byref(h)), "acopf_batch_create")
        self._h = h
        self._io = None

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_create(models) -> Batch:
    return Batch(models)


def batch_set_io(batch: Batch, ios, stream=None) -> None:
    """ios: one dict per instance with keys x, y, sigma_x, sigma_s, obj_weight,
    delta_w, delta_c, f, grad, cons, jvals, hvals, kvals and optionally Pd, Qd
    (tensors or device addresses)."""
    arr = (BatchIO * len(ios))()
    for k, d in enumerate(ios):
        r = arr[k]
        for name in ("x", "y", "sigma_x", "sigma_s", "f", "grad", "cons", "jvals", "hvals",
                     "kvals", "Pd", "Qd"):
            setattr(r, name, _ptr(d.get(name)))
        r.obj_weight = float(d.get("obj_weight", 1.0))
        r.delta_w = float(d.get("delta_w", 0.0))
        r.delta_c = float(d.get("delta_c", 0.0))
    _check(_batch_set_io(batch.handle, arr, len(ios), _stream(stream)), "acopf_batch_set_io")
    batch._io = ios  # keep the tensors alive with the batch


def batch_eval_assemble(batch: Batch, stream=None) -> None:
    _check(_batch_eval_assemble(batch.handle, _stream(stream)), "acopf_batch_eval_assemble")


def batch_set_schedule(batch: Batch, schedule: int) -> None:
    _check(_batch_set_schedule(batch.handle, schedule), "acopf_batch_set_schedule")


def batch_autotune(batch: Batch, reps: int = 10, stream=None):
    """Returns (best schedule, {schedule: ms per evaluation})."""
    best = C.c_int32()
    times = (C.c_float * BATCH_SCHEDULES)()
    _check(_batch_autotune(batch.handle, _stream(stream), reps, C.byref(best), times),
           "acopf_batch_autotune")
    return best.value, {k: times[k] for k in range(BATCH_SCHEDULES) if times[k] >= 0}


def batch_info(batch: Batch):
    """Returns (schedule, phase-1 items, phase-2 items, device bytes)."""
    s, a, b, d = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(_batch_info(batch.handle, C.byref(s), C.byref(a), C.byref(b), C.byref(d)),
           "acopf_batch_info")
    return s.value, a.value, b.value, d.value


class Server:
    """A request server (owner of an ``acopf_server*``)."""

    def __init__(self, device: int, budget_bytes: int, mode: int = SERVE_CONTINUOUS,
                 max_active: int = 256):
        h = _vp()
        _check(_server_create(device, int(budget_bytes), mode, max_active, C.byref(h)),
               "acopf_server_create")
        self._h = h
        self._keep = {}  # ticket -> host arrays the server reads or writes

    def submit(self, model: Model, n_calls: int, x, y, sigma_x, sigma_s, *, obj_weight=1.0,
               delta_w=0.0, delta_c=0.0, Pd=None, Qd=None, f_calls=None, grad=None, cons=None,
               jvals=None, hvals=None, kvals=None) -> int:
        """Queues a request.  x, y, sigma_x, sigma_s: host arrays of n_points
        point sets (shape (n_points, n) or (n,)); outputs are host arrays the
        server fills (page-locked memory keeps the copies asynchronous).
        Returns the ticket."""
        arrays = dict(x=x, y=y, sigma_x=sigma_x, sigma_s=sigma_s, Pd=Pd, Qd=Qd, f_calls=f_calls,
                      grad=grad, cons=cons, jvals=jvals, hvals=hvals, kvals=kvals)
        for k, a in arrays.items():
            if a is not None and (not isinstance(a, np.ndarray) or a.dtype != np.float64):
                raise TypeError(f"{k} must be a float64 numpy array")
        n_points = 1 if x.ndim == 1 else x.shape[0]
        if x.size != n_points * model.n or sigma_x.size != n_points * model.n:
            raise ValueError("x / sigma_x must hold n_points * n values")
        if y.size != n_points * model.m or sigma_s.size != n_points * model.m:
            raise ValueError("y / sigma_s must hold n_points * m values")
        sizes = dict(f_calls=n_calls, grad=model.n, cons=model.m, jvals=model.nnz_jac,
                     hvals=model.nnz_hess, kvals=model.nnz_kkt, Pd=model.n_bus, Qd=model.n_bus)
        for k, n in sizes.items():
            if arrays[k] is not None and arrays[k].size != n:
                raise ValueError(f"{k} must hold {n} values")
        r = Request()
        r.model = model.handle.value
        r.n_calls, r.n_points = n_calls, n_points
        for k, a in arrays.items():
            setattr(r, k, _hptr(a))
        r.obj_weight, r.delta_w, r.delta_c = float(obj_weight), float(delta_w), float(delta_c)
        t = C.c_uint64()
        _check(_server_submit(self._h, C.byref(r), C.byref(t)), "acopf_server_submit")
        self._keep[t.value] = (model, arrays)
        return t.value

    def poll(self, ticket: int):
        """Returns (done, status)."""
        d, st = C.c_int32(), C.c_int32()
        _check(_server_poll(self._h, ticket, C.byref(d), C.byref(st)), "acopf_server_poll")
        return bool(d.value), st.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        """Waits for a ticket; returns its status (raises on timeout)."""
        st = C.c_int32()
        _check(_server_wait(self._h, ticket, float(timeout_s), C.byref(st)), "acopf_server_wait")
        return st.value

    def times(self, ticket: int):
        """(admitted, done) in seconds after submission."""
        a, d = C.c_double(), C.c_double()
        _check(_server_times(self._h, ticket, C.byref(a), C.byref(d)),
               "acopf_server_request_times")
        return a.value, d.value

    def release(self, ticket: int) -> None:
        _check(_server_release(self._h, ticket), "acopf_server_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        s = ServerStats()
        _check(_server_stats(self._h, C.byref(s)), "acopf_server_get_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def set_option(self, option: int, value: int) -> None:
        _check(_server_set_option(self._h, option, value), "acopf_server_set_option")

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _server_destroy(self._h)
        self._h = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def server_create(device: int, budget_bytes: int, mode: int = SERVE_CONTINUOUS,
                  max_active: int = 256) -> Server:
    return Server(device, budget_bytes, mode, max_active)


class Pipeline:
    """Pipelined host-buffer evaluation of one model (owner of an
    ``acopf_pipeline*``)."""

    def __init__(self, model: Model, depth: int = 2):
        h = _vp()
        _check(_pipeline_create(model.handle, depth, C.byref(h)), "acopf_pipeline_create")
        self._h = h
        self.model = model
        self._keep = []

    def submit(self, x, y, obj_weight: float, sigma_x, sigma_s, delta_w: float, delta_c: float,
               f, grad, cons, jvals, hvals, kvals) -> None:
        """Queues one call; host numpy arrays (kept alive until wait())."""
        arrs = (x, y, sigma_x, sigma_s, f, grad, cons, jvals, hvals, kvals)
        for a in arrs:
            if not isinstance(a, np.ndarray) or a.dtype != np.float64:
                raise TypeError("pipeline buffers must be float64 numpy arrays")
        _check(_pipeline_submit(self._h, _hptr(x), _hptr(y), float(obj_weight), _hptr(sigma_x),
                                _hptr(sigma_s), float(delta_w), float(delta_c), _hptr(f),
                                _hptr(grad), _hptr(cons), _hptr(jvals), _hptr(hvals),
                                _hptr(kvals)), "acopf_pipeline_submit")
        self._keep.append(arrs)

    def wait(self) -> None:
        _check(_pipeline_wait(self._h), "acopf_pipeline_wait")
        self._keep.clear()

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _pipeline_destroy(self._h)
        self._h = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pipeline_create(model: Model, depth: int = 2) -> Pipeline:
    return Pipeline(model, depth)


def _iterate(it) -> Iterate:
    """it: mapping (or object) with the ITERATE_FIELDS as tensors / addresses."""
    get = it.get if isinstance(it, dict) else (lambda k: getattr(it, k))
    r = Iterate()
    for k in ITERATE_FIELDS:
        setattr(r, k, _ptr(get(k)))
    return r


def condense(model: Model, it, jvals, delta_w: float, delta_c: float, sigma_x, sigma_s, q_s,
             rhs, stream=None) -> None:
    r = _iterate(it)
    _check(_condense(model.handle, C.byref(r), _ptr(jvals), float(delta_w), float(delta_c),
                     _ptr(sigma_x), _ptr(sigma_s), _ptr(q_s), _ptr(rhs), _stream(stream)),
           "acopf_condense")


def recover_step(model: Model, it, jvals, delta_w: float, delta_c: float, sigma_s, q_s, dx, ds,
                 dy, dzl_x, dzu_x, dzl_s, dzu_s, stream=None) -> None:
    r = _iterate(it)
    _check(_recover_step(model.handle, C.byref(r), _ptr(jvals), float(delta_w), float(delta_c),
                         _ptr(sigma_s), _ptr(q_s), _ptr(dx), _ptr(ds), _ptr(dy), _ptr(dzl_x),
                         _ptr(dzu_x), _ptr(dzl_s), _ptr(dzu_s), _stream(stream)),
           "acopf_recover_step")


def kkt_residual(model: Model, it, y, grad, cons, jvals, mu: float, out, stream=None) -> None:
    """out: device array of 9 doubles (see RESIDUAL_FIELDS)."""
    r = _iterate(it)
    _check(_kkt_residual(model.handle, C.byref(r), _ptr(y), _ptr(grad), _ptr(cons), _ptr(jvals),
                         float(mu), _ptr(out), _stream(stream)), "acopf_kkt_residual")


class Chol:
    """Sparse Cholesky factorization of a model's M_cond (owner of an
    ``acopf_chol*``)."""

    def __init__(self, model: Model):
        h = _vp()
        _check(_chol_create(model.handle, C.byref(h)), "acopf_chol_create")
        self._h = h
        self.model = model

    def factor(self, kvals, pivot_tol: float = 0.0, stream=None) -> int:
        """Factorizes M_cond from its lower-CSR values (device); returns -1
        when every pivot passes (positive definite), else the first failing
        pivot's position in the factorization order."""
        pos = C.c_int32(0)
        _check(_chol_factor(self._h, _ptr(kvals), float(pivot_tol), C.byref(pos),
                            _stream(stream)), "acopf_chol_factor")
        return pos.value

    def solve(self, b, x, stream=None) -> None:
        _check(_chol_solve(self._h, _ptr(b), _ptr(x), _stream(stream)), "acopf_chol_solve")

    def info(self) -> dict:
        """The symbolic counts (CholStats fields) and device_bytes (all
        device memory of the object)."""
        st, nbytes = CholStats(), C.c_int64(0)
        _check(_chol_info(self._h, C.byref(st), C.byref(nbytes)), "acopf_chol_info")
        return {**st.as_dict(), "device_bytes": nbytes.value}

    def set_trace(self, enable: bool) -> None:
        """Turns the per-task trace of later factorizations and solves on/off."""
        _check(_chol_set_trace(self._h, 1 if enable else 0), "acopf_chol_set_trace")

    def trace(self, which: int = 0) -> np.ndarray:
        """The last run's trace of graph `which` (0 factorization block tasks;
        solve block tasks 1 forward, 2 backward; solve warp tasks 3 forward,
        4 backward; 5 factorization warp tasks):
        one row per task, (kind word, argument, taken ns, ready ns, finished
        ns, SM)."""
        n = C.c_int64(0)
        _check(_chol_get_trace(self._h, int(which), None, 0, C.byref(n)), "acopf_chol_get_trace")
        out = np.zeros((n.value, 6), dtype=np.int64)
        _check(_chol_get_trace(self._h, int(which), out.ctypes.data, n.value, C.byref(n)),
               "acopf_chol_get_trace")
        return out

    def permutation(self) -> np.ndarray:
        """The fill-reducing order (row i of P M_cond P' is row perm[i])."""
        p = np.empty(self.model.n, dtype=np.int32)
        _check(_chol_permutation(self._h, p.ctypes.data), "acopf_chol_permutation")
        return p

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _chol_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def chol_create(model: Model) -> Chol:
    return Chol(model)


def chol_analyze(model: Model, with_perm: bool = False):
    """Symbolic counts of a factorization of the model's M_cond (a dict);
    with_perm: also the order (dict, perm)."""
    st = CholStats()
    perm = np.empty(model.n, dtype=np.int32) if with_perm else None
    _check(_chol_analyze(model.handle, C.byref(st), None if perm is None else perm.ctypes.data),
           "acopf_chol_analyze")
    return (st.as_dict(), perm) if with_perm else st.as_dict()


def ipm_solve(model: Model, tol: float = 1e-4, max_iter: int = 200, mu_init: float = 0.1,
              stream=None, chol: "Chol | None" = None):
    """Algorithm 1 on the model (acopf_ipm_solve; with ``chol``, a Cholesky
    object of this model the caller keeps, acopf_ipm_solve_chol).  Returns
    (result dict, final x, history array of shape (max_iter + 1, 7))."""
    opts = IpmOptions(float(tol), int(max_iter), float(mu_init))
    res = IpmResult()
    x = np.empty(model.n, dtype=np.float64)
    hist = np.empty((int(max_iter) + 1, len(IPM_HISTORY_FIELDS)), dtype=np.float64)
    if chol is None:
        _check(_ipm_solve(model.handle, C.byref(opts), x.ctypes.data, hist.ctypes.data,
                          C.byref(res), _stream(stream)), "acopf_ipm_solve")
    else:
        _check(_ipm_solve_chol(model.handle, chol._h, C.byref(opts), x.ctypes.data,
                               hist.ctypes.data, C.byref(res), _stream(stream)),
               "acopf_ipm_solve_chol")
    return {k: getattr(res, k) for k, _ in res._fields_}, x, hist
