"""Python entry to Oracle A (direct Volterra march, `volterra.c`).

TEST INFRASTRUCTURE ONLY — see the package docstring.  The C file is compiled with
gcc on first use (or by `build()`), into `oracle/_build/`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_volterra.so")
_SO_CS = os.path.join(_HERE, "_build", "liboracle_volterra_cs.so")
_lib = None
_lib_cs = None


def _compile(so: str, defines: list[str], force: bool) -> None:
    src = os.path.join(_HERE, "volterra.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(so), exist_ok=True)
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", *defines,
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, so)


def build(force: bool = False) -> str:
    """Compile the real build and the complex-step build of `volterra.c`."""
    _compile(_SO, [], force)
    _compile(_SO_CS, ["-DORACLE_COMPLEX_STEP"], force)
    return _SO


def _bind(f):
    d = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_long, d, d, ctypes.c_int, ctypes.c_double, ctypes.c_long,
                  ctypes.c_int, ctypes.c_int, d, d, d, d, ctypes.c_long, d, ctypes.c_int,
                  d, d, d, d]
    f.restype = ctypes.c_int


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _bind(_lib.oracle_volterra_march)
    return _lib


def _load_cs():
    global _lib_cs
    if _lib_cs is None:
        build()
        _lib_cs = ctypes.CDLL(_SO_CS)
        _bind(_lib_cs.oracle_volterra_march_cs)
    return _lib_cs


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def march(x, beta, periodic: bool, dt: float, Nt: int, p: int, amp=(), center=(), width=(),
          g=None, xr=()):
    """Direct march.  Returns (sigma[(Nt+1), M], u[(Nt+1), R]); row n is time t_n = n dt.

    g: optional (Nt+1, M) forcing samples g_j(t_n) replacing the incident-wave forcing.
    """
    return _run(_load().oracle_volterra_march, np.float64, x, beta, periodic, dt, Nt, p, amp,
                center, width, g, xr)


def march_complex_step(x, beta, periodic: bool, dt: float, Nt: int, p: int, amp=(), center=(),
                       width=(), g=None, xr=()):
    """The same march with complex stiffnesses (the complex-step build): returns complex sigma
    and u.  With beta + i h e_j, Im(output) / h is d(output)/d beta_j up to O(h^2)."""
    return _run(_load_cs().oracle_volterra_march_cs, np.complex128, x, beta, periodic, dt, Nt, p,
                amp, center, width, g, xr)


def _run(f, vtype, x, beta, periodic, dt, Nt, p, amp, center, width, g, xr):
    x = np.ascontiguousarray(x, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=vtype)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    center = np.ascontiguousarray(center, dtype=np.float64)
    width = np.ascontiguousarray(width, dtype=np.float64)
    xr = np.ascontiguousarray(xr, dtype=np.float64).reshape(-1)
    M, R = x.shape[0], xr.shape[0]
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert g.shape == (Nt + 1, M)
    ng = p // 2 + 2
    gx, gw = np.polynomial.legendre.leggauss(ng)
    sigma = np.zeros((Nt + 1, M), dtype=vtype)
    u = np.zeros((Nt + 1, max(R, 1)), dtype=vtype)
    rc = f(M, _ptr(x), _ptr(beta), int(periodic), float(dt), int(Nt), int(p), int(amp.shape[0]),
           _ptr(amp), _ptr(center), _ptr(width), _ptr(g), R, _ptr(xr) if R else _ptr(np.zeros(1)),
           ng, _ptr(gx), _ptr(gw), _ptr(sigma), _ptr(u))
    if rc != 0:
        raise RuntimeError(f"the direct march failed with status {rc}")
    return sigma, u[:, :R]


def march_workload(w, Nt=None, dt=None, p=None):
    """Oracle A on a `workloads.Workload` (optionally with another Nt, dt or p)."""
    return march(w.x, w.beta, w.bc == 0, dt if dt is not None else w.dt,
                 Nt if Nt is not None else w.Nt, p if p is not None else w.p,
                 w.amp, w.center, w.width, None, w.xr)
