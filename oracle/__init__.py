"""Oracle for the space-time hybrid parareal method (Laidin, arXiv 2511.13386).

TEST INFRASTRUCTURE ONLY.  A plain, sequential FP64 C implementation of the
fine hybrid propagator S^HMM (Sec. 2.3), the limit scheme S^0, the lifting of
Def. 1 and Algorithm 1, used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA path; the two
only meet through the seeded input generators.

Parity unpinned (no printed value or closed form fixes it): the discrete
time derivative of E inside R.  Which scaling of the remainder criterion the
paper means (literal |R| or eps^2 |R|) is a reading; both switches are pinned
(exact-rational brute force and the threshold-crossing test), as is the
cell-based density update of eq. S^HMM (brute force and its mass defect).
Lifting orders above one are pinned to their continuous limit and to the
scheme's relaxed perturbation, not to a printed value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction, so that
    results are the same on x86-64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    fresh = os.path.exists(_LIB) and all(
        os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in (_SRC, _HDR))
    if force or not fresh:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("x_len", ctypes.c_double), ("v_max", ctypes.c_double),
                ("eps", ctypes.c_double), ("rho_bar", ctypes.c_double),
                ("adapt", ctypes.c_int32), ("thr_g", ctypes.c_double),
                ("thr_R", ctypes.c_double), ("r_scale", ctypes.c_int32),
                ("flux_rule", ctypes.c_int32)]


class _FineStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("kinetic_updates", ctypes.c_int64)]


class _PararealCfg(ctypes.Structure):
    _fields_ = [("t_end", ctypes.c_double), ("n_slices", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double),
                ("coarse_kind", ctypes.c_int32), ("coarse_steps", ctypes.c_int32),
                ("dt_fine", ctypes.c_double), ("lift_order", ctypes.c_int32),
                ("mode", ctypes.c_int32)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            sig = {
                "orc_velocity_grid": (ctypes.c_double, [P, _D, _D, _D]),
                "orc_fd_coefficients": (None, [ctypes.c_int, _D]),
                "orc_fd_derivative": (None, [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _D]),
                "orc_poisson": (None, [P, _D, _D]),
                "orc_flux_J": (None, [P, _D, _D, _D]),
                "orc_gnorm": (None, [P, _D, _D]),
                "orc_remainder": (None, [P, _D, _D, _D]),
                "orc_initial_status": (None, [P, _D, _D, _U8]),
                "orc_update_status": (None, [P, _D, _D, _U8]),
                "orc_dt_limit": (ctypes.c_double, [P, ctypes.c_double]),
                "orc_fine_step": (ctypes.c_int64, [P, ctypes.c_double, _D, _D, _U8]),
                "orc_fine": (None, [P, ctypes.c_int64, ctypes.c_double, _D, _D, _U8,
                                    ctypes.POINTER(_FineStats)]),
                "orc_limit_step": (None, [P, ctypes.c_double, _D]),
                "orc_limit_step_implicit": (None, [P, ctypes.c_double, _D]),
                "orc_coarse": (None, [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]),
                "orc_lift": (None, [P, _D, _D]),
                "orc_lift_order": (None, [P, ctypes.c_int, _D, _D]),
                "orc_parareal": (ctypes.c_int, [P, ctypes.POINTER(_PararealCfg), _D, _D, _D, _D]),
                "orc_sequential": (None, [P, ctypes.POINTER(_PararealCfg), _D, _D, _D]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


@dataclass
class Params:
    """Problem parameters; field names follow the paper's notation."""
    nx: int
    nv: int
    eps: float
    v_max: float = 8.0
    x_len: float = 1.0
    rho_bar: float = 1.0
    adapt: bool = False
    thr_g: float = 1e-3
    thr_R: float = 1e-2
    r_scale: int = 0
    flux_rule: int = 0

    def _c(self) -> _Params:
        return _Params(self.nx, self.nv, self.x_len, self.v_max, self.eps,
                       self.rho_bar, int(self.adapt), self.thr_g, self.thr_R,
                       int(self.r_scale), int(self.flux_rule))


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def velocity_grid(p: Params):
    """(v, w, M, m2) of the velocity discretisation."""
    lib = _load()
    v, w, M = (np.empty(p.nv) for _ in range(3))
    m2 = lib.orc_velocity_grid(ctypes.byref(p._c()), _dptr(v), _dptr(w), _dptr(M))
    return v, w, M, m2


def fd_coefficients(d: int) -> np.ndarray:
    c = np.empty(7)
    _load().orc_fd_coefficients(d, _dptr(c))
    return c


def fd_derivative(f, dx: float, d: int) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    _load().orc_fd_derivative(f.size, dx, d, _dptr(f), _dptr(out))
    return out


def poisson(p: Params, rho) -> np.ndarray:
    rho = _f64(rho)
    E = np.empty(p.nx)
    _load().orc_poisson(ctypes.byref(p._c()), _dptr(rho), _dptr(E))
    return E


def flux_J(p: Params, rho, E) -> np.ndarray:
    rho, E = _f64(rho), _f64(E)
    J = np.empty(p.nx)
    _load().orc_flux_J(ctypes.byref(p._c()), _dptr(rho), _dptr(E), _dptr(J))
    return J


def gnorm(p: Params, g) -> np.ndarray:
    g = _f64(g)
    N = np.empty(p.nx)
    _load().orc_gnorm(ctypes.byref(p._c()), _dptr(g), _dptr(N))
    return N


def remainder(p: Params, rho, E) -> np.ndarray:
    rho, E = _f64(rho), _f64(E)
    R = np.empty(p.nx)
    _load().orc_remainder(ctypes.byref(p._c()), _dptr(rho), _dptr(E), _dptr(R))
    return R


def initial_status(p: Params, rho, g) -> np.ndarray:
    rho, g = _f64(rho), _f64(g)
    m = np.empty(p.nx, dtype=np.uint8)
    _load().orc_initial_status(ctypes.byref(p._c()), _dptr(rho), _dptr(g),
                               m.ctypes.data_as(_U8))
    return m


def update_status(p: Params, rho, g, mask) -> np.ndarray:
    rho, g = _f64(rho), _f64(g)
    m = np.ascontiguousarray(np.array(mask, dtype=np.uint8))
    _load().orc_update_status(ctypes.byref(p._c()), _dptr(rho), _dptr(g),
                              m.ctypes.data_as(_U8))
    return m


def dt_limit(p: Params, theta: float = 0.9) -> float:
    return _load().orc_dt_limit(ctypes.byref(p._c()), theta)


def fine_step(p: Params, dt: float, rho, g, mask):
    """One S^HMM step; returns (rho, g, mask, kinetic interfaces)."""
    rho, g = _f64(rho).copy(), _f64(g).copy()
    m = np.ascontiguousarray(np.array(mask, dtype=np.uint8))
    n = _load().orc_fine_step(ctypes.byref(p._c()), dt, _dptr(rho), _dptr(g),
                              m.ctypes.data_as(_U8))
    return rho, g, m, n


def fine(p: Params, n_steps: int, dt: float, rho, g):
    """F: n_steps steps of S^HMM; returns (rho, g, final mask, stats dict)."""
    rho, g = _f64(rho).copy(), _f64(g).copy()
    m = np.empty(p.nx, dtype=np.uint8)
    st = _FineStats()
    _load().orc_fine(ctypes.byref(p._c()), int(n_steps), dt, _dptr(rho), _dptr(g),
                     m.ctypes.data_as(_U8), ctypes.byref(st))
    return rho, g, m, {"steps": st.steps, "kinetic_updates": st.kinetic_updates}


def limit_step(p: Params, dt: float, rho) -> np.ndarray:
    rho = _f64(rho).copy()
    _load().orc_limit_step(ctypes.byref(p._c()), dt, _dptr(rho))
    return rho


def limit_step_implicit(p: Params, dt: float, rho) -> np.ndarray:
    rho = _f64(rho).copy()
    _load().orc_limit_step_implicit(ctypes.byref(p._c()), dt, _dptr(rho))
    return rho


def coarse(p: Params, t_span: float, rho, kind: int = 0, n_sub: int = 1) -> np.ndarray:
    rho = _f64(rho).copy()
    _load().orc_coarse(ctypes.byref(p._c()), kind, n_sub, t_span, _dptr(rho))
    return rho


def lift(p: Params, rho, order: int = 1) -> np.ndarray:
    """Lifting of order `order` (Def. 1); order 1 is the first-order term
    alone, orders 2 and 3 add the Chapman-Enskog terms h2, h3."""
    rho = _f64(rho)
    g = np.empty((p.nx, p.nv))
    if order <= 1:
        _load().orc_lift(ctypes.byref(p._c()), _dptr(rho), _dptr(g))
    else:
        _load().orc_lift_order(ctypes.byref(p._c()), int(order), _dptr(rho), _dptr(g))
    return g


def _cfg(t_end, n_slices, max_iter, tol, coarse_kind, coarse_steps, dt_fine, lift_order=1, mode=0):
    return _PararealCfg(t_end, n_slices, max_iter, tol, coarse_kind, coarse_steps, dt_fine, lift_order, mode)


def parareal(p: Params, rho0, g0, t_end: float, n_slices: int, max_iter: int,
             tol: float = 0.0, coarse_kind: int = 0, coarse_steps: int = 1,
             dt_fine: float | None = None, lift_order: int = 1, mode: int = 0):
    """Algorithm 1; returns (rho_slices [(N+1), nx], errors, iterations).
    mode 0: density only with relifting; mode 1: full state (rho, g)."""
    rho0, g0 = _f64(rho0), _f64(g0)
    if dt_fine is None:
        dt_fine = dt_limit(p)
    out = np.empty((n_slices + 1, p.nx))
    err = np.zeros(max(max_iter, 1))
    c = _cfg(t_end, n_slices, max_iter, tol, coarse_kind, coarse_steps, dt_fine, lift_order, mode)
    it = _load().orc_parareal(ctypes.byref(p._c()), ctypes.byref(c), _dptr(rho0),
                              _dptr(g0), _dptr(out), _dptr(err))
    return out, err[:it], it


def sequential(p: Params, rho0, g0, t_end: float, n_slices: int,
               dt_fine: float | None = None, lift_order: int = 1, mode: int = 0) -> np.ndarray:
    """Sequential fine reference with relifting at every slice boundary
    (mode 0), or the plain F carried through the slices (mode 1)."""
    rho0, g0 = _f64(rho0), _f64(g0)
    if dt_fine is None:
        dt_fine = dt_limit(p)
    out = np.empty((n_slices + 1, p.nx))
    c = _cfg(t_end, n_slices, 0, 0.0, 0, 1, dt_fine, lift_order, mode)
    _load().orc_sequential(ctypes.byref(p._c()), ctypes.byref(c), _dptr(rho0),
                           _dptr(g0), _dptr(out))
    return out
