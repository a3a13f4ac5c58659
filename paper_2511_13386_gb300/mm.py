"""Python binding of the libmm C ABI (include/mm.h).

Argument marshalling only: every array is passed as a raw pointer (a torch
tensor's data_ptr(), on the GPU or in host memory, or a numpy array's
buffer) together with the current CUDA stream.  All computation happens in
libmm.so; if the library cannot be loaded this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

MM_OK, MM_ERR_INVALID, MM_ERR_OOM, MM_ERR_CUDA, MM_ERR_TIMEOUT, MM_ERR_UNSTABLE, \
    MM_ERR_BUSY, MM_ERR_NOT_READY, MM_ERR_UNKNOWN_TICKET = range(9)
MM_FP64, MM_FP32G = 0, 1
STATUS_NAMES = ["MM_OK", "MM_ERR_INVALID", "MM_ERR_OOM", "MM_ERR_CUDA", "MM_ERR_TIMEOUT",
                "MM_ERR_UNSTABLE", "MM_ERR_BUSY", "MM_ERR_NOT_READY", "MM_ERR_UNKNOWN_TICKET"]

EXPORTED = ["mm_params_default", "mm_create", "mm_destroy", "mm_query", "mm_fine_propagate",
            "mm_fine_propagate_noalloc", "mm_autotune", "mm_set_chunk_entry", "mm_coarse", "mm_lift", "parareal_run", "mm_coarse_guess",
            "mm_parareal_correct", "mm_batch_footprint",
            "mm_batch_create", "mm_batch_add", "mm_batch_step", "mm_batch_query", "mm_batch_take",
            "mm_batch_bytes", "mm_batch_counters", "mm_batch_destroy", "parareal_run_many", "mm_server_create", "serve_submit",
            "serve_poll", "mm_server_destroy", "mm_probe_fp32", "mm_last_error"]


class MMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


class mm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nv", ctypes.c_int32), ("x_len", ctypes.c_double),
                ("v_max", ctypes.c_double), ("eps", ctypes.c_double), ("rho_bar", ctypes.c_double),
                ("adapt", ctypes.c_int32), ("thr_g", ctypes.c_double), ("thr_R", ctypes.c_double),
                ("r_scale", ctypes.c_int32), ("flux_rule", ctypes.c_int32), ("dt", ctypes.c_double),
                ("cfl_theta", ctypes.c_double), ("coarse_kind", ctypes.c_int32),
                ("coarse_steps", ctypes.c_int32), ("lift_order", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("fine_kernel", ctypes.c_int32),
                ("fine_vpt", ctypes.c_int32)]


class mm_alloc(ctypes.Structure):
    _fields_ = [("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("user", ctypes.c_void_p)]


class mm_info(ctypes.Structure):
    _fields_ = [("dt_limit", ctypes.c_double), ("dt", ctypes.c_double), ("n_steps", ctypes.c_int64),
                ("m2", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("state_bytes", ctypes.c_size_t), ("vpt", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("fine_kernel", ctypes.c_int32), ("cluster", ctypes.c_int32)]


class mm_fine_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("kinetic_updates", ctypes.c_int64),
                ("full_updates", ctypes.c_int64), ("device_status", ctypes.c_int32),
                ("elapsed_ms", ctypes.c_double), ("launches", ctypes.c_int32)]


class mm_tune_result(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("fine_kernel", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("vpt", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("cand_kernel", ctypes.c_int32 * 16),
                ("cand_cluster", ctypes.c_int32 * 16), ("cand_vpt", ctypes.c_int32 * 16),
                ("cand_ms", ctypes.c_double * 16), ("res_entry_steps", ctypes.c_double)]


MM_PARAREAL_RHO_LIFT, MM_PARAREAL_FULL_STATE = 0, 1


class mm_parareal_cfg(ctypes.Structure):
    _fields_ = [("t_end", ctypes.c_double), ("n_slices", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("mode", ctypes.c_int32)]


class mm_parareal_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("err", ctypes.c_double * 64),
                ("mass_drift", ctypes.c_double), ("fine_steps", ctypes.c_int64),
                ("kinetic_updates", ctypes.c_int64), ("elapsed_ms", ctypes.c_double),
                ("fine_ms", ctypes.c_double), ("fine_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32)]


class mm_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32)]


class mm_request(ctypes.Structure):
    _fields_ = [("params", mm_params), ("cfg", mm_parareal_cfg), ("rho0", ctypes.c_void_p),
                ("g0", ctypes.c_void_p)]


class mm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("rho_T", ctypes.c_void_p), ("iterations", ctypes.c_int32),
                ("latency_ns", ctypes.c_int64), ("kinetic_updates", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmm.so (building it first when missing and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libmm is not built ({_build.LIB}); call build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        V, P = ctypes.c_void_p, ctypes.POINTER
        sig = {
            "mm_params_default": (None, [P(mm_params)]),
            "mm_create": (ctypes.c_int, [P(mm_params), P(mm_alloc), P(V)]),
            "mm_destroy": (None, [V]),
            "mm_query": (ctypes.c_int, [V, ctypes.c_double, P(mm_info)]),
            "mm_fine_propagate": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_double, V, V, V, V, V,
                                                 P(mm_fine_stats), V]),
            "mm_fine_propagate_noalloc": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_double, V, V, V,
                                                         V, V, P(mm_fine_stats), V]),
            "mm_autotune": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_int32, V, V, V, V, P(mm_tune_result), V]),
            "mm_set_chunk_entry": (ctypes.c_int, [V, ctypes.c_double]),
            "mm_coarse": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_double, V, V, V]),
            "mm_lift": (ctypes.c_int, [V, ctypes.c_int32, V, V, V]),
            "parareal_run": (ctypes.c_int, [V, P(mm_parareal_cfg), V, V, V, P(mm_parareal_stats), V]),
            "mm_coarse_guess": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_double, V, V, V]),
            "mm_parareal_correct": (ctypes.c_int, [V, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, V, V, V,
                                                   V, V]),
            "mm_server_create": (ctypes.c_int, [P(mm_server_cfg), P(mm_alloc), P(V)]),
            "serve_submit": (ctypes.c_int, [V, P(mm_request), P(ctypes.c_uint64)]),
            "serve_poll": (ctypes.c_int, [V, ctypes.c_uint64, P(mm_result), ctypes.c_int32]),
            "mm_server_destroy": (ctypes.c_int, [V]),
            "mm_last_error": (ctypes.c_char_p, []),
            "mm_probe_fp32": (ctypes.c_int, [P(ctypes.c_double), V]),
            "mm_batch_footprint": (ctypes.c_size_t, [P(mm_params), P(mm_parareal_cfg)]),
            "mm_batch_create": (ctypes.c_int, [P(mm_alloc), P(V)]),
            "mm_batch_add": (ctypes.c_int, [V, P(mm_params), P(mm_parareal_cfg), V, V, P(ctypes.c_uint64)]),
            "mm_batch_step": (ctypes.c_int, [V, P(ctypes.c_int32), V]),
            "mm_batch_query": (ctypes.c_int, [V, ctypes.c_uint64, P(ctypes.c_int32)]),
            "mm_batch_take": (ctypes.c_int, [V, ctypes.c_uint64, V, P(mm_parareal_stats)]),
            "mm_batch_bytes": (ctypes.c_size_t, [V]),
            "mm_batch_counters": (ctypes.c_int, [V, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_double)]),
            "mm_batch_destroy": (None, [V]),
            "parareal_run_many": (ctypes.c_int, [ctypes.c_int32, P(mm_params), P(mm_parareal_cfg), P(V), P(V),
                                                 P(V), P(mm_parareal_stats), V]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def mm_probe_fp32(stream=None) -> float:
    """Measured FP32 FMA rate of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().mm_probe_fp32(ctypes.byref(t), _stream(stream)))
    return t.value


def mm_last_error() -> str:
    return load().mm_last_error().decode()


def _check(st: int):
    if st != MM_OK:
        raise MMError(st, mm_last_error())


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous(), "arrays must be contiguous"
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def mm_params_default(**overrides) -> mm_params:
    p = mm_params()
    load().mm_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


# ------------------------------------------------------------ allocators --

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator:
    """Device-memory callbacks handed to the library (the mm_alloc of
    include/mm.h).  alloc(nbytes, stream) returns a device address (0 to
    refuse, which the library reports as MM_ERR_OOM); free(ptr, stream)
    releases one.  The library may call them from its own threads (the
    server's schedulers); exceptions are turned into a refusal.  The object
    must outlive every context, batch or server created with it."""

    def __init__(self, alloc, free):
        self._alloc, self._free = alloc, free

        def a(n, stream, user):
            try:
                return int(self._alloc(int(n), stream or 0) or 0)
            except Exception:
                return 0

        def f(ptr, stream, user):
            try:
                if ptr:
                    self._free(int(ptr), stream or 0)
            except Exception:
                pass
        self._cb_a, self._cb_f = _ALLOC_FN(a), _FREE_FN(f)
        self.struct = mm_alloc(ctypes.cast(self._cb_a, ctypes.c_void_p),
                               ctypes.cast(self._cb_f, ctypes.c_void_p), None)


_torch_alloc = None


def torch_allocator():
    """The torch caching allocator as the library's device memory: workspace
    and batch arrays come out of (and go back to) torch's pool, on the
    stream the library passes."""
    global _torch_alloc
    if _torch_alloc is None:
        import torch

        def alloc(n, stream):
            return torch.cuda.caching_allocator_alloc(n, device=torch.cuda.current_device(), stream=stream)

        def free(ptr, stream):
            torch.cuda.caching_allocator_delete(ptr)
        _torch_alloc = Allocator(alloc, free)
    return _torch_alloc


def _default_alloc():
    try:
        import torch
        if torch.cuda.is_available():
            return torch_allocator()
    except Exception:
        pass
    return None


def _alloc_arg(alloc):
    """alloc: "torch" (torch's caching allocator, the default when CUDA is
    available), None (the library's own stream-ordered cudaMallocAsync) or
    an Allocator."""
    if isinstance(alloc, str):
        if alloc != "torch":
            raise ValueError(f"unknown allocator {alloc!r}")
        alloc = _default_alloc()
    return (ctypes.byref(alloc.struct) if alloc is not None else None), alloc


class Ctx:
    """Owning handle of an mm_ctx."""

    def __init__(self, handle, params: mm_params):
        self.handle = handle
        self.params = params

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().mm_destroy(self.handle)
            self.handle = None


def mm_create(params: mm_params, alloc="torch") -> Ctx:
    h = ctypes.c_void_p()
    ref, keep = _alloc_arg(alloc)
    _check(load().mm_create(ctypes.byref(params), ref, ctypes.byref(h)))
    c = Ctx(h, params)
    c.alloc = keep
    return c


def mm_destroy(ctx: Ctx):
    ctx.close()


def mm_query(ctx: Ctx, t_span: float) -> dict:
    info = mm_info()
    _check(load().mm_query(ctx.handle, t_span, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in mm_info._fields_}


def mm_set_chunk_entry(ctx: Ctx, entry_steps: float):
    _check(load().mm_set_chunk_entry(ctx.handle, float(entry_steps)))


def mm_fine_propagate(ctx: Ctx, batch: int, t_span: float, rho_in, g_in, rho_out, g_out,
                      mask_out=None, stats: bool = False, stream=None):
    st = mm_fine_stats() if stats else None
    _check(load().mm_fine_propagate(ctx.handle, batch, t_span, _ptr(rho_in), _ptr(g_in),
                                    _ptr(rho_out), _ptr(g_out), _ptr(mask_out),
                                    ctypes.byref(st) if st is not None else None,
                                    _stream(stream)))
    return {f: getattr(st, f) for f, _ in mm_fine_stats._fields_} if st is not None else None


def mm_fine_propagate_noalloc(ctx: Ctx, batch: int, t_span: float, rho_in, g_in, rho_out, g_out,
                              mask_out=None, stats: bool = False, stream=None):
    """F with the library's fixed device scratch instead of allocated
    workspace (device arrays only; see include/mm.h)."""
    st = mm_fine_stats() if stats else None
    _check(load().mm_fine_propagate_noalloc(ctx.handle, batch, t_span, _ptr(rho_in), _ptr(g_in),
                                            _ptr(rho_out), _ptr(g_out), _ptr(mask_out),
                                            ctypes.byref(st) if st is not None else None,
                                            _stream(stream)))
    return {f: getattr(st, f) for f, _ in mm_fine_stats._fields_} if st is not None else None


NOALLOC_SCRATCH_BYTES = 64 << 20


def mm_autotune(ctx: Ctx, batch: int, steps: int, rho_in, g_in, rho_out, g_out, stream=None) -> dict:
    """Pick F's fastest launch shape for this context by timing every
    candidate on the given batch (outputs are scratch); batch == 0 restores
    the default.  Returns the choice and the candidates' times."""
    r = mm_tune_result()
    _check(load().mm_autotune(ctx.handle, batch, steps, _ptr(rho_in), _ptr(g_in), _ptr(rho_out),
                              _ptr(g_out), ctypes.byref(r), _stream(stream)))
    n = min(r.n_candidates, 16)
    return {"n_candidates": r.n_candidates, "fine_kernel": r.fine_kernel, "cluster": r.cluster,
            "vpt": r.vpt, "lanes": r.lanes, "best_ms": r.best_ms, "res_entry_steps": r.res_entry_steps,
            "candidates": [{"fine_kernel": r.cand_kernel[q], "cluster": r.cand_cluster[q],
                            "vpt": r.cand_vpt[q], "ms": r.cand_ms[q]} for q in range(n)]}


def mm_coarse(ctx: Ctx, batch: int, t_span: float, rho_in, rho_out, stream=None):
    _check(load().mm_coarse(ctx.handle, batch, t_span, _ptr(rho_in), _ptr(rho_out), _stream(stream)))


def mm_lift(ctx: Ctx, batch: int, rho, g_out, stream=None):
    _check(load().mm_lift(ctx.handle, batch, _ptr(rho), _ptr(g_out), _stream(stream)))


def parareal_run(ctx: Ctx, t_end: float, n_slices: int, max_iter: int, tol: float, rho0, g0,
                 rho_slices_out, stream=None, mode: int = MM_PARAREAL_RHO_LIFT) -> dict:
    cfg = mm_parareal_cfg(t_end, n_slices, max_iter, tol, mode)
    st = mm_parareal_stats()
    _check(load().parareal_run(ctx.handle, ctypes.byref(cfg), _ptr(rho0), _ptr(g0),
                               _ptr(rho_slices_out), ctypes.byref(st), _stream(stream)))
    it = st.iterations
    return {"iterations": it, "err": [st.err[k] for k in range(min(it, 64))],
            "mass_drift": st.mass_drift, "fine_steps": st.fine_steps,
            "kinetic_updates": st.kinetic_updates, "elapsed_ms": st.elapsed_ms,
            "fine_ms": st.fine_ms, "fine_launches": st.fine_launches,
            "kernel_launches": st.kernel_launches}


def mm_coarse_guess(ctx: Ctx, n_slices: int, t_span: float, rho_slices, g_prev, stream=None):
    _check(load().mm_coarse_guess(ctx.handle, n_slices, t_span, _ptr(rho_slices), _ptr(g_prev),
                                  _stream(stream)))


def mm_parareal_correct(ctx: Ctx, n_slices: int, k: int, t_span: float, rho_slices, f_rho, g_prev, err,
                        stream=None):
    _check(load().mm_parareal_correct(ctx.handle, n_slices, k, t_span, _ptr(rho_slices), _ptr(f_rho),
                                      _ptr(g_prev), _ptr(err), _stream(stream)))


def _stats_dict(st: "mm_parareal_stats") -> dict:
    it = st.iterations
    return {"iterations": it, "err": [st.err[k] for k in range(min(it, 64))],
            "mass_drift": st.mass_drift, "fine_steps": st.fine_steps,
            "kinetic_updates": st.kinetic_updates, "elapsed_ms": st.elapsed_ms,
            "fine_ms": st.fine_ms, "fine_launches": st.fine_launches,
            "kernel_launches": st.kernel_launches}


class Batch:
    """Owning handle of an mm_batch (many parareal solves advanced together)."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            load().mm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def mm_batch_footprint(params: mm_params, t_end: float, n_slices: int, max_iter: int, tol: float) -> int:
    cfg = mm_parareal_cfg(t_end, n_slices, max_iter, tol)
    return load().mm_batch_footprint(ctypes.byref(params), ctypes.byref(cfg))


def mm_batch_create(alloc="torch") -> Batch:
    h = ctypes.c_void_p()
    ref, keep = _alloc_arg(alloc)
    _check(load().mm_batch_create(ref, ctypes.byref(h)))
    b = Batch(h)
    b.alloc = keep
    return b


def mm_batch_add(batch: Batch, params: mm_params, t_end: float, n_slices: int, max_iter: int, tol: float,
                 rho0, g0, mode: int = MM_PARAREAL_RHO_LIFT) -> int:
    cfg = mm_parareal_cfg(t_end, n_slices, max_iter, tol, mode)
    i = ctypes.c_uint64()
    _check(load().mm_batch_add(batch.handle, ctypes.byref(params), ctypes.byref(cfg), _ptr(rho0), _ptr(g0),
                               ctypes.byref(i)))
    return i.value


def mm_batch_step(batch: Batch, stream=None) -> int:
    a = ctypes.c_int32()
    _check(load().mm_batch_step(batch.handle, ctypes.byref(a), _stream(stream)))
    return a.value


def mm_batch_query(batch: Batch, solve_id: int) -> bool:
    d = ctypes.c_int32()
    _check(load().mm_batch_query(batch.handle, solve_id, ctypes.byref(d)))
    return bool(d.value)


def mm_batch_take(batch: Batch, solve_id: int, rho_slices_out) -> dict:
    st = mm_parareal_stats()
    _check(load().mm_batch_take(batch.handle, solve_id, _ptr(rho_slices_out), ctypes.byref(st)))
    return _stats_dict(st)


def mm_batch_bytes(batch: Batch) -> int:
    return load().mm_batch_bytes(batch.handle)


def mm_batch_counters(batch: Batch) -> dict:
    k, n, t = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
    _check(load().mm_batch_counters(batch.handle, ctypes.byref(k), ctypes.byref(n), ctypes.byref(t)))
    return {"kinetic_updates": k.value, "fine_launches": n.value, "fine_ms": t.value}


def mm_batch_destroy(batch: Batch):
    batch.close()


def parareal_run_many(params: list, cfgs: list, rho0: list, g0: list, outs: list, stream=None) -> list:
    """cfgs: (t_end, n_slices, max_iter, tol) tuples; arrays host or device."""
    n = len(params)
    P = (mm_params * n)(*params)
    C = (mm_parareal_cfg * n)(*[mm_parareal_cfg(*c) for c in cfgs])
    V = ctypes.c_void_p
    R = (V * n)(*[_ptr(a) for a in rho0])
    G = (V * n)(*[_ptr(a) for a in g0])
    O = (V * n)(*[_ptr(a) for a in outs])
    S = (mm_parareal_stats * n)()
    _check(load().parareal_run_many(n, P, C, R, G, O, S, _stream(stream)))
    return [_stats_dict(S[q]) for q in range(n)]


class Server:
    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            load().mm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def mm_server_create(hbm_budget_bytes: int, max_slots: int, wait_limit_ms: int = 60000,
                     alloc="torch") -> Server:
    cfg = mm_server_cfg(hbm_budget_bytes, max_slots, wait_limit_ms)
    h = ctypes.c_void_p()
    ref, keep = _alloc_arg(alloc)
    _check(load().mm_server_create(ctypes.byref(cfg), ref, ctypes.byref(h)))
    srv = Server(h)
    srv.alloc = keep
    return srv


def serve_submit(server: Server, params: mm_params, t_end: float, n_slices: int, max_iter: int,
                 tol: float, rho0: np.ndarray, g0: np.ndarray) -> int:
    req = mm_request(params, mm_parareal_cfg(t_end, n_slices, max_iter, tol), _ptr(rho0), _ptr(g0))
    t = ctypes.c_uint64()
    _check(load().serve_submit(server.handle, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def serve_poll(server: Server, ticket: int, nx: int, timeout_ms: int = 0):
    """Returns None when not ready, else a dict with the result."""
    out = np.empty(nx)
    res = mm_result(0, out.ctypes.data, 0, 0, 0)
    st = load().serve_poll(server.handle, ticket, ctypes.byref(res), timeout_ms)
    if st == MM_ERR_NOT_READY:
        return None
    _check(st)
    return {"status": res.status, "rho_T": out, "iterations": res.iterations,
            "latency_ns": res.latency_ns, "kinetic_updates": res.kinetic_updates}


def mm_server_destroy(server: Server):
    server.close()


def nan() -> float:
    return math.nan
