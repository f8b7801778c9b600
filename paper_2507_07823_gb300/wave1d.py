"""ctypes binding of the wave1d C-ABI (include/wave1d.h).  Argument marshalling only.

Every function below has the name and argument order of the C entry point.  Arrays are
numpy float64 arrays (host) or torch tensors (device, via `data_ptr()`); the CUDA library
does all the work.  There is no CPU fallback: `lib()` raises if the library is missing.
`Plan` is a small convenience wrapper used by the tests and the benchmark.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwave1d.so")

WAVE1D_PERIODIC = 0
WAVE1D_FREE = 1

WAVE1D_OK = 0
WAVE1D_EINVAL = -1
WAVE1D_EDOMAIN = -2
WAVE1D_ENOMEM = -3
WAVE1D_ECUDA = -4
WAVE1D_ENOTCONV = -5
WAVE1D_ENONFINITE = -6
WAVE1D_EDONE = -7
WAVE1D_EUNSUPPORTED = -9
WAVE1D_ETIMEOUT = -10

WAVE1D_ARR_ALPHA = 0
WAVE1D_ARR_ALPHA_P = 1
WAVE1D_ARR_S_LAST = 2
WAVE1D_ARR_UH = 3
WAVE1D_ARR_LOCAL = 4
WAVE1D_ARR_SIGMA_RING = 5
WAVE1D_ARR_PERM = 6

EXPORTED = ["wave1d_opts_default", "wave1d_plan", "wave1d_set_incident_gaussians",
            "wave1d_set_receivers", "wave1d_step", "wave1d_solve", "wave1d_read_receivers",
            "wave1d_get_sigma", "wave1d_sync", "wave1d_get_info", "wave1d_inspect",
            "wave1d_destroy", "wave1d_strerror", "wave1d_profile", "wave1d_profile_read",
            "wave1d_nufft1_noalloc", "wave1d_state_size", "wave1d_state_save", "wave1d_state_load",
            "wave1d_nufft_plan", "wave1d_nufft_plan_many", "wave1d_nufft_info", "wave1d_nufft_perm",
            "wave1d_nufft_spread",
            "wave1d_nufft_interp", "wave1d_nufft_type1", "wave1d_nufft_type2", "wave1d_nufft_destroy",
            "wave1d_nufft_strerror", "wave1d_adjoint", "wave1d_checkpoint_size", "wave1d_solve_checkpointed",
            "wave1d_adjoint_checkpointed", "wave1d_batch_plan", "wave1d_batch_solve",
            "wave1d_batch_destroy", "wave1d_batch_strerror", "wave1d_batch_step_kernel", "wave1d_batch_forms",
            "wave1d_nufft_autotune"]

WAVE1D_NSTAGE = 9
STAGES = ["local", "spread", "fft_fwd", "modes", "rbc", "fft_inv", "interp", "solve", "receivers"]


class wave1d_opts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("gamma", ctypes.c_double), ("W", ctypes.c_int),
                ("NL", ctypes.c_int), ("Ng", ctypes.c_int), ("nufft_w", ctypes.c_int),
                ("rbc_period", ctypes.c_int), ("max_block", ctypes.c_int),
                ("max_local_bytes", ctypes.c_int64), ("step_kernel", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("precision", ctypes.c_int), ("local_weights", ctypes.c_int),
                ("spin_limit", ctypes.c_int), ("hold_unit", ctypes.c_int)]


class wave1d_info(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("R", ctypes.c_int64), ("Nt", ctypes.c_int64),
                ("n", ctypes.c_int64),
                ("K", ctypes.c_int), ("NF", ctypes.c_int), ("W", ctypes.c_int),
                ("m_max", ctypes.c_int), ("p", ctypes.c_int), ("NL", ctypes.c_int),
                ("Ng", ctypes.c_int), ("nufft_w", ctypes.c_int), ("nf", ctypes.c_int),
                ("rbc_period", ctypes.c_int),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double), ("b", ctypes.c_double),
                ("delta", ctypes.c_double),
                ("local_pairs", ctypes.c_int64), ("local_weights", ctypes.c_int64),
                ("nearby_pairs", ctypes.c_int64), ("blocks", ctypes.c_int64),
                ("max_block", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("local_bytes", ctypes.c_int64), ("local_terms", ctypes.c_int64),
                ("solve_sweeps", ctypes.c_int64)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib(path: str = LIB_PATH):
    """Load the CUDA library (built by `paper_2507_07823_gb300.build.build()`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"wave1d CUDA library not built: {path} (run __graft_entry__.build())")
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.wave1d_opts_default.argtypes = [ctypes.POINTER(wave1d_opts)]
        L.wave1d_plan.argtypes = [_D, _D, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int64, ctypes.c_double, ctypes.POINTER(wave1d_opts),
                                  ctypes.POINTER(P)]
        L.wave1d_set_incident_gaussians.argtypes = [P, ctypes.c_int, _D, _D, _D]
        L.wave1d_set_receivers.argtypes = [P, _D, ctypes.c_int64]
        L.wave1d_step.argtypes = [P, _D, ctypes.c_int]
        L.wave1d_solve.argtypes = [P, ctypes.c_int64, _D, _D, ctypes.c_int]
        L.wave1d_read_receivers.argtypes = [P, _D, ctypes.c_int]
        L.wave1d_get_sigma.argtypes = [P, _D, ctypes.c_int]
        L.wave1d_sync.argtypes = [P]
        L.wave1d_get_info.argtypes = [P, ctypes.POINTER(wave1d_info)]
        L.wave1d_inspect.argtypes = [P, ctypes.c_int, _D, ctypes.c_int64]
        L.wave1d_destroy.argtypes = [P]
        L.wave1d_profile.argtypes = [P, ctypes.c_int]
        L.wave1d_profile_read.argtypes = [P, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        L.wave1d_nufft1_noalloc.argtypes = [_D, _D, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                            _D, ctypes.c_void_p]
        L.wave1d_state_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.wave1d_state_save.argtypes = [P, ctypes.c_void_p, ctypes.c_size_t]
        L.wave1d_state_load.argtypes = [P, ctypes.c_void_p, ctypes.c_size_t]
        L.wave1d_nufft_plan.argtypes = [_D, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.POINTER(P)]
        L.wave1d_nufft_plan_many.argtypes = [_D, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int, P, ctypes.POINTER(P)]
        L.wave1d_nufft_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.wave1d_nufft_perm.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        for nm in ("wave1d_nufft_spread", "wave1d_nufft_interp", "wave1d_nufft_type1", "wave1d_nufft_type2"):
            getattr(L, nm).argtypes = [P, _D, _D]
        L.wave1d_nufft_destroy.argtypes = [P]
        L.wave1d_nufft_autotune.argtypes = [P, _D, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int)]
        L.wave1d_adjoint.argtypes = [P, ctypes.c_int64, _D, _D, _D, _D, _D]
        L.wave1d_checkpoint_size.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
        L.wave1d_solve_checkpointed.argtypes = [P, ctypes.c_int64, ctypes.c_int64, _D, ctypes.c_int, P,
                                                ctypes.c_size_t]
        L.wave1d_adjoint_checkpointed.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_size_t, _D, _D, _D]
        _I64 = ctypes.POINTER(ctypes.c_int64)
        L.wave1d_batch_plan.argtypes = [ctypes.c_int, _I64, _D, _D, _D, _I64, _D, ctypes.c_double, ctypes.c_int64,
                                        ctypes.c_double, ctypes.POINTER(wave1d_opts), ctypes.POINTER(ctypes.c_void_p)]
        L.wave1d_batch_solve.argtypes = [P, ctypes.c_int64, _D, _D, ctypes.c_int]
        L.wave1d_batch_destroy.argtypes = [P]
        L.wave1d_batch_step_kernel.argtypes = [P]
        L.wave1d_batch_forms.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        L.wave1d_batch_strerror.argtypes = []
        L.wave1d_batch_strerror.restype = ctypes.c_char_p
        L.wave1d_nufft_strerror.argtypes = []
        L.wave1d_nufft_strerror.restype = ctypes.c_char_p
        L.wave1d_strerror.argtypes = [ctypes.c_int]
        L.wave1d_strerror.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("wave1d_strerror", "wave1d_nufft_strerror", "wave1d_batch_strerror"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class Wave1DError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().wave1d_strerror(status).decode()
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(status, where):
    if status != WAVE1D_OK:
        raise Wave1DError(status, where)


def _hptr(a):
    return a.ctypes.data_as(_D)


def _dptr(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), _D)


# --- the C entry points, same names -------------------------------------------------------
def wave1d_opts_default():
    o = wave1d_opts()
    _check(lib().wave1d_opts_default(ctypes.byref(o)), "wave1d_opts_default")
    return o


def wave1d_plan(x, beta, M, bc, dt, Nt, tol, opts=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib().wave1d_plan(_hptr(x), _hptr(beta), int(M), int(bc), float(dt), int(Nt), float(tol),
                           ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return st, h


def wave1d_set_incident_gaussians(plan, n, amp, center, width):
    a, c, w = (np.ascontiguousarray(v, dtype=np.float64) for v in (amp, center, width))
    return lib().wave1d_set_incident_gaussians(plan, int(n), _hptr(a), _hptr(c), _hptr(w))


def wave1d_set_receivers(plan, xr, R):
    xr = np.ascontiguousarray(xr, dtype=np.float64)
    return lib().wave1d_set_receivers(plan, _hptr(xr) if R else None, int(R))


def wave1d_step(plan, g_next=None, g_on_device=0):
    if g_next is None:
        return lib().wave1d_step(plan, None, 0)
    ptr = _dptr(g_next) if g_on_device else _hptr(g_next)
    return lib().wave1d_step(plan, ptr, int(g_on_device))


def wave1d_solve(plan, nsteps, u_rec, sigma, out_on_device):
    f = _dptr if out_on_device else _hptr
    return lib().wave1d_solve(plan, int(nsteps), f(u_rec) if u_rec is not None else None,
                              f(sigma) if sigma is not None else None, int(out_on_device))


def wave1d_adjoint(plan, nsteps, sigma, g, ubar, grad_beta, grad_g):
    """sigma, g (nsteps x M), ubar (nsteps x R), grad_beta (M), grad_g (nsteps x M): device tensors;
    g, ubar (when R = 0), grad_beta and grad_g may be None."""
    def opt(t):
        return _dptr(t) if t is not None else None
    return lib().wave1d_adjoint(plan, int(nsteps), _dptr(sigma), opt(g), opt(ubar), opt(grad_beta), opt(grad_g))


def wave1d_checkpoint_size(plan, nsteps, interval):
    b = ctypes.c_size_t()
    _check(lib().wave1d_checkpoint_size(plan, int(nsteps), int(interval), ctypes.byref(b)), "wave1d_checkpoint_size")
    return b.value


def wave1d_solve_checkpointed(plan, nsteps, interval, u_rec, ckpt):
    """u_rec: device tensor (nsteps x R) or None; ckpt: device tensor of wave1d_checkpoint_size bytes."""
    return lib().wave1d_solve_checkpointed(plan, int(nsteps), int(interval),
                                           _dptr(u_rec) if u_rec is not None else None, 1,
                                           ctypes.c_void_p(ckpt.data_ptr()), ckpt.numel() * ckpt.element_size())


def wave1d_adjoint_checkpointed(plan, nsteps, interval, ckpt, ubar, grad_beta, grad_g):
    def opt(t):
        return _dptr(t) if t is not None else None
    return lib().wave1d_adjoint_checkpointed(plan, int(nsteps), int(interval), ctypes.c_void_p(ckpt.data_ptr()),
                                             ckpt.numel() * ckpt.element_size(), opt(ubar), opt(grad_beta),
                                             opt(grad_g))


class Nufft:
    """Standalone type-1 / type-2 NUFFT plan (device arrays are torch CUDA tensors of float64;
    point arrays in the plan's point order, see `perm`).  `x` is one point set, or a list of
    point sets (the batched form: grids, S and alpha are then instance-major)."""

    def __init__(self, x, K, tol, precision=0, stream=None):
        h = ctypes.c_void_p()
        st_ptr = ctypes.c_void_p(stream) if stream is not None else None
        if isinstance(x, (list, tuple)):
            sets = [np.ascontiguousarray(v, dtype=np.float64).ravel() for v in x]
            offsets = np.zeros(len(sets) + 1, dtype=np.int64)
            offsets[1:] = np.cumsum([v.size for v in sets])
            xa = np.ascontiguousarray(np.concatenate(sets))
            st = lib().wave1d_nufft_plan_many(_hptr(xa), offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              len(sets), int(K), float(tol), int(precision), st_ptr,
                                              ctypes.byref(h))
            name, self.B, self.offsets = "wave1d_nufft_plan_many", len(sets), offsets
        else:
            xa = np.ascontiguousarray(x, dtype=np.float64)
            st = lib().wave1d_nufft_plan(_hptr(xa), xa.shape[0], int(K), float(tol), int(precision), st_ptr,
                                         ctypes.byref(h))
            name, self.B, self.offsets = "wave1d_nufft_plan", 1, np.array([0, xa.shape[0]], dtype=np.int64)
        if st != WAVE1D_OK:
            raise Wave1DError(st, name + ": " + lib().wave1d_nufft_strerror().decode())
        self.h, self.M, self.K = h, xa.shape[0], int(K)
        nf, w, deg, err = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().wave1d_nufft_info(h, ctypes.byref(nf), ctypes.byref(w), ctypes.byref(deg),
                                       ctypes.byref(err)), "wave1d_nufft_info")
        self.nf, self.w, self.degree, self.kernel_err = nf.value, w.value, deg.value, err.value
        perm = np.zeros(self.M, dtype=np.int64)
        _check(lib().wave1d_nufft_perm(h, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "wave1d_nufft_perm")
        self.perm = perm

    def _call(self, name, a, b):
        st = getattr(lib(), name)(self.h, _dptr(a), _dptr(b))
        if st != WAVE1D_OK:
            raise Wave1DError(st, name + ": " + lib().wave1d_nufft_strerror().decode())

    def spread(self, c, grid):
        self._call("wave1d_nufft_spread", c, grid)

    def interp(self, grid, u):
        self._call("wave1d_nufft_interp", grid, u)

    def type1(self, c, S):
        self._call("wave1d_nufft_type1", c, S)

    def type2(self, alpha, u):
        self._call("wave1d_nufft_type2", alpha, u)

    def autotune(self, c, grid, reps=5):
        """Time the spreading's candidate work splits on c (device, point order) and keep the
        fastest; returns its (cells, points) caps.  grid (device) is overwritten."""
        cells, points = ctypes.c_int(), ctypes.c_int()
        st = lib().wave1d_nufft_autotune(self.h, _dptr(c), _dptr(grid), int(reps), ctypes.byref(cells),
                                         ctypes.byref(points))
        if st != WAVE1D_OK:
            raise Wave1DError(st, "wave1d_nufft_autotune: " + lib().wave1d_nufft_strerror().decode())
        return cells.value, points.value

    def close(self):
        if self.h:
            lib().wave1d_nufft_destroy(self.h)
            self.h = None


def wave1d_state_size(plan):
    n = ctypes.c_size_t(0)
    _check(lib().wave1d_state_size(plan, ctypes.byref(n)), "wave1d_state_size")
    return n.value


def wave1d_state_save(plan, buf):
    """buf: a contiguous numpy uint8 array of at least wave1d_state_size(plan) bytes."""
    return lib().wave1d_state_save(plan, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes)


def wave1d_state_load(plan, buf):
    return lib().wave1d_state_load(plan, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes)


def wave1d_read_receivers(plan, u, on_device):
    return lib().wave1d_read_receivers(plan, _dptr(u) if on_device else _hptr(u), int(on_device))


def wave1d_get_sigma(plan, out, on_device):
    return lib().wave1d_get_sigma(plan, _dptr(out) if on_device else _hptr(out), int(on_device))


def wave1d_sync(plan):
    return lib().wave1d_sync(plan)


def wave1d_get_info(plan):
    info = wave1d_info()
    _check(lib().wave1d_get_info(plan, ctypes.byref(info)), "wave1d_get_info")
    return info


def wave1d_inspect(plan, array, host_out):
    return lib().wave1d_inspect(plan, int(array), _hptr(host_out), int(host_out.size))


def wave1d_destroy(plan):
    return lib().wave1d_destroy(plan)


def wave1d_profile(plan, enable):
    return lib().wave1d_profile(plan, int(enable))


def wave1d_profile_read(plan):
    ms = np.zeros(WAVE1D_NSTAGE)
    steps = ctypes.c_int64()
    _check(lib().wave1d_profile_read(plan, _hptr(ms), WAVE1D_NSTAGE, ctypes.byref(steps)),
           "wave1d_profile_read")
    return ms, steps.value


def wave1d_nufft1_noalloc(x, c, M, K, tol, S, stream=None):
    """x, c, S: device tensors (float64); S holds 2 (K+1) values."""
    return lib().wave1d_nufft1_noalloc(_dptr(x), _dptr(c), int(M), int(K), float(tol), _dptr(S),
                                       ctypes.c_void_p(stream) if stream else None)


def wave1d_strerror(status):
    return lib().wave1d_strerror(int(status)).decode()


# --- convenience wrapper ------------------------------------------------------------------
class Plan:
    """One wave1d plan built from a `workloads.Workload` (or explicit arrays)."""

    def __init__(self, x, beta, bc, dt, Nt, tol, amp=(), center=(), width=(), xr=(), stream=None,
                 **opt):
        o = wave1d_opts_default()
        for k, v in opt.items():
            setattr(o, k, v)
        if stream is not None:
            o.stream = ctypes.c_void_p(stream)
        x = np.ascontiguousarray(x, dtype=np.float64)
        st, h = wave1d_plan(x, beta, x.shape[0], bc, dt, Nt, tol, o)
        _check(st, "wave1d_plan")
        self.h = h
        self.M = x.shape[0]
        if len(amp):
            _check(wave1d_set_incident_gaussians(h, len(amp), amp, center, width), "set_incident")
        xr = np.ascontiguousarray(xr, dtype=np.float64).reshape(-1)
        self.R = xr.shape[0]
        if self.R:
            _check(wave1d_set_receivers(h, xr, self.R), "set_receivers")
        self.info = wave1d_get_info(h)

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.x, w.beta, w.bc, w.dt, w.Nt, w.tol, w.amp, w.center, w.width, w.xr,
                   p=w.p, **kw)

    def solve(self, nsteps, with_sigma=True):
        u = np.zeros((nsteps, max(self.R, 1)))
        s = np.zeros((nsteps, self.M)) if with_sigma else None
        _check(wave1d_solve(self.h, nsteps, u if self.R else None, s, 0), "wave1d_solve")
        return (s, u[:, :self.R])

    def solve_device(self, nsteps):
        """The march with device outputs: (sigma, u) torch CUDA tensors, rows s = step s + 1."""
        import torch
        s = torch.empty((nsteps, self.M), dtype=torch.float64, device="cuda")
        u = torch.empty((nsteps, max(self.R, 1)), dtype=torch.float64, device="cuda")
        _check(wave1d_solve(self.h, nsteps, u if self.R else None, s, 1), "wave1d_solve")
        return s, u[:, :self.R]

    def adjoint(self, sigma, ubar, g=None, forcing_gradient=False):
        """dL/dbeta (torch CUDA tensor, caller order) from the march's densities sigma (nsteps x M)
        and the receiver adjoints ubar = dL/du (nsteps x R), both torch CUDA tensors.  g: the
        forcing vectors of a march driven by `step(g)` (nsteps x M), None for the incident wave.
        With forcing_gradient=True, returns (dL/dbeta, dL/dg) with dL/dg of shape nsteps x M."""
        import torch
        n = sigma.shape[0]
        gb = torch.empty(self.M, dtype=torch.float64, device=sigma.device)
        gg = torch.empty((n, self.M), dtype=torch.float64, device=sigma.device) if forcing_gradient else None
        ub = ubar.contiguous() if self.R else None
        gin = g.contiguous() if g is not None else None
        _check(wave1d_adjoint(self.h, n, sigma.contiguous(), gin, ub, gb, gg), "wave1d_adjoint")
        return (gb, gg) if forcing_gradient else gb

    def solve_checkpointed(self, nsteps, interval):
        """The march from step 0 keeping its state every `interval` steps: (u, ckpt), u the
        receiver fields (nsteps x R torch CUDA tensor), ckpt the checkpoints (a uint8 CUDA tensor)."""
        import torch
        ckpt = torch.empty(wave1d_checkpoint_size(self.h, nsteps, interval), dtype=torch.uint8, device="cuda")
        u = torch.empty((nsteps, max(self.R, 1)), dtype=torch.float64, device="cuda")
        _check(wave1d_solve_checkpointed(self.h, nsteps, interval, u if self.R else None, ckpt),
               "wave1d_solve_checkpointed")
        return u[:, :self.R], ckpt

    def adjoint_checkpointed(self, ckpt, nsteps, interval, ubar, forcing_gradient=False):
        """dL/dbeta (and dL/dg with forcing_gradient=True) from the checkpoints of
        solve_checkpointed(nsteps, interval) and ubar = dL/du (nsteps x R torch CUDA tensor)."""
        import torch
        gb = torch.empty(self.M, dtype=torch.float64, device="cuda")
        gg = torch.empty((nsteps, self.M), dtype=torch.float64, device="cuda") if forcing_gradient else None
        ub = ubar.contiguous() if self.R else None
        _check(wave1d_adjoint_checkpointed(self.h, nsteps, interval, ckpt, ub, gb, gg), "wave1d_adjoint_checkpointed")
        return (gb, gg) if forcing_gradient else gb

    def step(self, g=None):
        _check(wave1d_step(self.h, g, 0), "wave1d_step")

    def sigma(self):
        out = np.zeros(self.M)
        _check(wave1d_get_sigma(self.h, out, 0), "wave1d_get_sigma")
        return out

    def receivers(self):
        out = np.zeros(max(self.R, 1))
        _check(wave1d_read_receivers(self.h, out, 0), "wave1d_read_receivers")
        return out[:self.R]

    def inspect(self, array):
        inf = wave1d_get_info(self.h)
        sizes = {WAVE1D_ARR_ALPHA: 2 * (inf.K + 1), WAVE1D_ARR_ALPHA_P: 2 * (inf.K + 1),
                 WAVE1D_ARR_S_LAST: 2 * (inf.K + 1), WAVE1D_ARR_UH: self.M,
                 WAVE1D_ARR_LOCAL: self.M, WAVE1D_ARR_SIGMA_RING: (inf.m_max + 1) * self.M,
                 WAVE1D_ARR_PERM: self.M}
        out = np.zeros(sizes[array])
        _check(wave1d_inspect(self.h, array, out), "wave1d_inspect")
        if array in (WAVE1D_ARR_ALPHA, WAVE1D_ARR_ALPHA_P, WAVE1D_ARR_S_LAST):
            return out[0::2] + 1j * out[1::2]
        if array == WAVE1D_ARR_SIGMA_RING:
            return out.reshape(inf.m_max + 1, self.M)
        return out

    def close(self):
        if self.h:
            wave1d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def receiver_fields(beta, w, nsteps):
    """The receiver fields u (nsteps x R, torch CUDA float64) of an nsteps march of workload `w`
    with stiffnesses `beta` (torch CUDA float64 tensor), differentiable in beta: the backward pass
    is the library's reverse-time march (wave1d_adjoint).  Each call builds and frees a plan."""
    import torch

    class _ReceiverFields(torch.autograd.Function):
        @staticmethod
        def forward(ctx, b):
            plan = Plan(w.x, b.detach().cpu().numpy(), w.bc, w.dt, max(w.Nt, nsteps), w.tol, w.amp,
                        w.center, w.width, w.xr, p=w.p)
            sigma, u = plan.solve_device(nsteps)
            ctx.plan = plan
            ctx.save_for_backward(sigma)
            return u

        @staticmethod
        def backward(ctx, gu):
            (sigma,) = ctx.saved_tensors
            try:
                return ctx.plan.adjoint(sigma, gu)
            finally:
                ctx.plan.close()

    return _ReceiverFields.apply(beta)


class Batch:
    """Batched march of independent periodic instances (`wave1d_batch_plan`): `instances` is a list
    of `workloads.Workload` sharing dt, tol and p (one incident Gaussian each, at least one
    receiver each or none at all).  `solve(n)` returns (sigma, u): n x (all springs) and
    n x (all receivers), instance-major in each workload's own order; `offsets` / `r_offsets`
    split them."""

    def __init__(self, instances, Nt=None, **opt):
        w0 = instances[0]
        o = wave1d_opts_default()
        o.p = w0.p
        for k, v in opt.items():
            setattr(o, k, v)
        x = np.ascontiguousarray(np.concatenate([w.x for w in instances]), dtype=np.float64)
        beta = np.ascontiguousarray(np.concatenate([w.beta for w in instances]), dtype=np.float64)
        self.offsets = np.zeros(len(instances) + 1, dtype=np.int64)
        self.offsets[1:] = np.cumsum([w.x.size for w in instances])
        self.r_offsets = np.zeros(len(instances) + 1, dtype=np.int64)
        self.r_offsets[1:] = np.cumsum([len(w.xr) for w in instances])
        pulse = np.ascontiguousarray([[w.amp[0], w.center[0], w.width[0]] for w in instances], dtype=np.float64)
        xr = np.ascontiguousarray(np.concatenate([np.asarray(w.xr, dtype=np.float64) for w in instances]))
        has_r = self.r_offsets[-1] > 0
        I64 = ctypes.POINTER(ctypes.c_int64)
        h = ctypes.c_void_p()
        st = lib().wave1d_batch_plan(len(instances), self.offsets.ctypes.data_as(I64), _hptr(x), _hptr(beta),
                                     _hptr(pulse), self.r_offsets.ctypes.data_as(I64) if has_r else None,
                                     _hptr(xr) if has_r else None, float(w0.dt), int(Nt or w0.Nt), float(w0.tol),
                                     ctypes.byref(o), ctypes.byref(h))
        if st != WAVE1D_OK:
            raise Wave1DError(st, "wave1d_batch_plan: " + lib().wave1d_batch_strerror().decode())
        self.h, self.M, self.R = h, int(self.offsets[-1]), int(self.r_offsets[-1])

    @property
    def one_launch(self):
        """True if the joined instances' steps run as one persistent launch."""
        return lib().wave1d_batch_step_kernel(self.h) == 1

    @property
    def forms(self):
        """Per instance: 0 in the joined tables (stored weights), 1 marched as its own plan without
        pair lists (`local_weights` = 1, or 2 with the choice made per instance)."""
        f = np.zeros(len(self.offsets) - 1, dtype=np.int32)
        st = lib().wave1d_batch_forms(self.h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if st != WAVE1D_OK:
            raise Wave1DError(st, "wave1d_batch_forms: " + lib().wave1d_batch_strerror().decode())
        return f

    def solve(self, nsteps, with_sigma=True):
        u = np.zeros((nsteps, max(self.R, 1)))
        s = np.zeros((nsteps, self.M)) if with_sigma else None
        st = lib().wave1d_batch_solve(self.h, int(nsteps), _hptr(u) if self.R else None,
                                      _hptr(s) if s is not None else None, 0)
        if st != WAVE1D_OK:
            raise Wave1DError(st, "wave1d_batch_solve: " + lib().wave1d_batch_strerror().decode())
        return s, u[:, :self.R]

    def close(self):
        if self.h:
            lib().wave1d_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
