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
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "volterra.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        f = _lib.oracle_volterra_march
        d = ctypes.POINTER(ctypes.c_double)
        f.argtypes = [ctypes.c_long, d, d, ctypes.c_int, ctypes.c_double, ctypes.c_long,
                      ctypes.c_int, ctypes.c_int, d, d, d, d, ctypes.c_long, d, ctypes.c_int,
                      d, d, d, d]
        f.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def march(x, beta, periodic: bool, dt: float, Nt: int, p: int, amp=(), center=(), width=(),
          g=None, xr=()):
    """Direct march.  Returns (sigma[(Nt+1), M], u[(Nt+1), R]); row n is time t_n = n dt.

    g: optional (Nt+1, M) forcing samples g_j(t_n) replacing the incident-wave forcing.
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
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
    sigma = np.zeros((Nt + 1, M))
    u = np.zeros((Nt + 1, max(R, 1)))
    rc = lib.oracle_volterra_march(M, _ptr(x), _ptr(beta), int(periodic), float(dt), int(Nt),
                                   int(p), int(amp.shape[0]), _ptr(amp), _ptr(center), _ptr(width),
                                   _ptr(g), R, _ptr(xr) if R else _ptr(np.zeros(1)), ng, _ptr(gx),
                                   _ptr(gw), _ptr(sigma), _ptr(u))
    if rc != 0:
        raise RuntimeError(f"oracle_volterra_march failed with status {rc}")
    return sigma, u[:, :R]


def march_workload(w, Nt=None, dt=None, p=None):
    """Oracle A on a `workloads.Workload` (optionally with another Nt, dt or p)."""
    return march(w.x, w.beta, w.bc == 0, dt if dt is not None else w.dt,
                 Nt if Nt is not None else w.Nt, p if p is not None else w.p,
                 w.amp, w.center, w.width, None, w.xr)
