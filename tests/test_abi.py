"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/wave1d.h
declares.  No GPU work is done here (argument checks return before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2507_07823_gb300 import build, wave1d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return wave1d.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "wave1d.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(wave1d_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(wave1d.EXPORTED)


def test_defaults_and_strerror(lib):
    o = wave1d.wave1d_opts_default()
    assert o.p == 8 and o.gamma == 0.5 and o.Ng == 32 and o.W == 0
    for st in (0, -1, -2, -3, -4, -6, -7, -9):
        assert isinstance(wave1d.wave1d_strerror(st), str)


def test_argument_validation_without_gpu(lib):
    x = np.array([0.1, 0.2])
    b = np.array([1.0, 2.0])
    assert wave1d.wave1d_plan(x, b, 0, 0, 0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EINVAL
    assert wave1d.wave1d_plan(x, b, 2, 7, 0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EINVAL
    assert wave1d.wave1d_plan(x, b, 2, 0, -0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EINVAL
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.01, 10, 0.5)[0] == wave1d.WAVE1D_EINVAL
    o = wave1d.wave1d_opts_default()
    o.p = 7
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.01, 10, 1e-10, o)[0] == wave1d.WAVE1D_EINVAL
    # window wider than pi (Sec. 3 assumes delta < pi)
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.2, 10, 1e-10)[0] == wave1d.WAVE1D_EDOMAIN
    # free-space spring outside Omega (Sec. 4.4)
    assert wave1d.wave1d_plan(np.array([3.1, 0.0]), b, 2, 1, 0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EDOMAIN
    bad = np.array([np.nan, 0.0])
    assert wave1d.wave1d_plan(bad, b, 2, 0, 0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EINVAL
    assert wave1d.wave1d_plan(x, np.array([1.0, -1.0]), 2, 0, 0.01, 10, 1e-10)[0] == wave1d.WAVE1D_EINVAL
    o = wave1d.wave1d_opts_default()
    assert o.precision == 0                                    # FP64 by default
    o.precision = 2
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.01, 10, 1e-10, o)[0] == wave1d.WAVE1D_EINVAL
    o.precision, o.nufft_w = 1, 9                              # mixed runs the width-7 kernel only
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.01, 10, 1e-10, o)[0] == wave1d.WAVE1D_EINVAL
    o = wave1d.wave1d_opts_default()
    assert o.local_weights == 0                                # stored weights by default
    o.local_weights = 2
    assert wave1d.wave1d_plan(x, b, 2, 0, 0.01, 10, 1e-10, o)[0] == wave1d.WAVE1D_EINVAL
    assert wave1d.wave1d_destroy(None) == 0


def test_nufft_argument_validation_without_gpu(lib):
    """wave1d_nufft_plan / wave1d_nufft_plan_many reject bad arguments before any CUDA call."""
    L = lib
    x = np.array([0.1, 0.2, 0.3])
    h = ctypes.c_void_p()
    xp = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def plan(M, K, tol, prec):
        return L.wave1d_nufft_plan(xp, M, K, tol, prec, None, ctypes.byref(h))

    assert plan(0, 10, 1e-10, 0) == wave1d.WAVE1D_EINVAL                 # no points
    assert plan(3, 0, 1e-10, 0) == wave1d.WAVE1D_EINVAL                  # no modes
    assert plan(3, 10, 0.5, 0) == wave1d.WAVE1D_EINVAL                   # tolerance out of (0, 0.1)
    assert plan(3, 10, 1e-10, 2) == wave1d.WAVE1D_EINVAL                 # unknown precision
    assert plan(3, 10, 1e-8, 1) == wave1d.WAVE1D_EINVAL                  # mixed precision below 1e-6
    assert L.wave1d_nufft_plan(None, 3, 10, 1e-10, 0, None, ctypes.byref(h)) == wave1d.WAVE1D_EINVAL

    def many(offsets, n):
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        return L.wave1d_nufft_plan_many(xp, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n, 10, 1e-10, 0,
                                        None, ctypes.byref(h))

    assert many([1, 3], 1) == wave1d.WAVE1D_EINVAL                       # offsets[0] != 0
    assert many([0, 2, 2, 3], 3) == wave1d.WAVE1D_EINVAL                 # an empty instance
    assert many([0, 3], 0) == wave1d.WAVE1D_EINVAL                       # no instances
    assert isinstance(L.wave1d_nufft_strerror(), bytes)
    assert L.wave1d_nufft_destroy(None) == 0
    assert L.wave1d_nufft_autotune(None, None, None, 3, None, None) == wave1d.WAVE1D_EINVAL


def test_adjoint_argument_validation_without_gpu(lib):
    """wave1d_adjoint refuses a missing plan before touching any device memory."""
    L = wave1d.lib()
    assert L.wave1d_adjoint(None, 1, None, None, None, None, None) == wave1d.WAVE1D_EINVAL


def test_batch_argument_validation_without_gpu(lib):
    """wave1d_batch_plan refuses bad instance layouts before touching the GPU."""
    L = wave1d.lib()
    I64 = ctypes.POINTER(ctypes.c_int64)
    x = np.array([0.1, 0.5, -0.3])
    b = np.array([1.0, 2.0, 3.0])
    pulse = np.array([[1.0, -2.0, 0.1], [1.0, -2.0, 0.1]])

    def plan(offsets, n, pl=pulse, opts=None):
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        h = ctypes.c_void_p()
        return L.wave1d_batch_plan(n, off.ctypes.data_as(I64), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   np.ascontiguousarray(pl).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   None, None, 0.01, 10, 1e-10, ctypes.byref(opts) if opts else None,
                                   ctypes.byref(h))
    assert plan([0, 3], 0) == wave1d.WAVE1D_EINVAL                       # no instances
    assert plan([1, 3], 1) == wave1d.WAVE1D_EINVAL                       # offsets[0] != 0
    assert plan([0, 0, 3], 2) == wave1d.WAVE1D_EINVAL                    # an instance without springs
    assert plan([0, 1, 3], 2, pl=np.array([[1.0, -2.0, 0.1], [1.0, -2.0, 0.0]])) == wave1d.WAVE1D_EINVAL
    o = wave1d.wave1d_opts_default()
    o.precision = 1                                                     # the batched march is FP64
    assert plan([0, 1, 3], 2, opts=o) == wave1d.WAVE1D_EINVAL
    o = wave1d.wave1d_opts_default()
    o.local_weights = 3                                                 # forms 0, 1 or 2 only
    assert plan([0, 1, 3], 2, opts=o) == wave1d.WAVE1D_EINVAL
    forms = (ctypes.c_int * 2)()
    assert L.wave1d_batch_forms(None, forms) == wave1d.WAVE1D_EINVAL
    assert L.wave1d_batch_destroy(None) == 0
    assert isinstance(L.wave1d_batch_strerror(), bytes)


def test_budget_and_block_limits_without_gpu(lib):
    """Host-side fault injection: a local-weight budget too small for the layout gives
    WAVE1D_ENOMEM, and a block of springs closer than dt larger than opts.max_block gives
    WAVE1D_EUNSUPPORTED, both before any device work."""
    x = np.array([-0.5, 0.1, 0.103, 0.106, 0.6])          # three springs within dt = 0.01 of each other
    b = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    o = wave1d.wave1d_opts_default()
    o.max_local_bytes = 1024
    st, _ = wave1d.wave1d_plan(x, b, 5, 0, 0.01, 10, 1e-10, o)
    assert st == wave1d.WAVE1D_ENOMEM
    assert "budget" in wave1d.wave1d_strerror(st)
    o = wave1d.wave1d_opts_default()
    o.max_block = 2
    st, _ = wave1d.wave1d_plan(x, b, 5, 0, 0.01, 10, 1e-10, o)
    assert st == wave1d.WAVE1D_EUNSUPPORTED
    assert "max_block" in wave1d.wave1d_strerror(st)
