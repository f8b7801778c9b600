"""Seeded synthetic workloads for 1D point-spring scattering.

This module only draws inputs: spring positions x_j, stiffnesses beta_j, the
Gaussian incident pulse parameters, receiver positions and the time grid.  It
holds none of the method's arithmetic, so both the oracle and the CUDA path
consume the same inputs without sharing any computation.

Physical setup (Sec. 1, eqs. uinc, WE-kink): M springs of stiffness beta_j > 0 at
x_j, driven by a right-moving incident wave u_inc(x, t) = f(x - t) with

    f(s) = sum_p amp_p * exp(-(s - center_p)^2 / (2 * width_p^2)).

"Width" is read as the standard deviation of the Gaussian.  The paper asks that
no spring lie in the support of f at t = 0 (Sec. 1, below eq. uinc); every
recipe below therefore keeps springs at least 8 widths away from each pulse
centre (f <= exp(-32) ~ 1.3e-14 there).  In the periodic box [-pi, pi] the
distance is the periodic one.  For free space the springs (and receivers) are
drawn inside [-pi + MARGIN, pi - MARGIN] with MARGIN = 0.12, which contains the
domain Omega = [-pi + 3 delta, pi - 3 delta] that Sec. 4.4 requires for every
window width delta = W dt used with these time steps (3 delta <= 0.117 for
dt = 1e-3 and tolerances down to 1e-13).

Seeds: numpy PCG64 with seed 7823 + configuration index.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

PI = math.pi
FREE_MARGIN = 0.12
EXCLUSION_WIDTHS = 8.0

PERIODIC = 0
FREE = 1


@dataclasses.dataclass
class Workload:
    name: str
    bc: int                      # PERIODIC or FREE
    x: np.ndarray                # (M,) float64 spring positions
    beta: np.ndarray             # (M,) float64 stiffnesses
    amp: np.ndarray              # (P,) pulse amplitudes
    center: np.ndarray           # (P,) pulse centres at t = 0
    width: np.ndarray            # (P,) pulse standard deviations
    dt: float
    Nt: int
    tol: float                   # window tolerance epsilon (b = ln 1/epsilon)
    p: int                       # local interpolation order
    xr: np.ndarray               # (R,) receiver positions
    seed: int
    description: str = ""

    @property
    def M(self) -> int:
        return int(self.x.shape[0])

    @property
    def R(self) -> int:
        return int(self.xr.shape[0])

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _periodic_distance(a: np.ndarray, b: float) -> np.ndarray:
    d = np.abs(a - b) % (2 * PI)
    return np.minimum(d, 2 * PI - d)


def _excluded(x: np.ndarray, center: np.ndarray, width: np.ndarray, periodic: bool) -> np.ndarray:
    bad = np.zeros(x.shape, dtype=bool)
    for c, w in zip(center, width):
        d = _periodic_distance(x, c) if periodic else np.abs(x - c)
        bad |= d < EXCLUSION_WIDTHS * w
    return bad


def _wrap(x: np.ndarray) -> np.ndarray:
    return (x + PI) % (2 * PI) - PI


def _draw_positions(rng, M, layout, periodic, center, width, lo, hi, n_clusters=16,
                    cluster_sigma=0.05, cluster_fraction=0.8):
    out = np.empty(0)
    if layout == "clustered":
        cc = rng.uniform(-PI, PI, size=n_clusters)
    while out.shape[0] < M:
        need = M - out.shape[0]
        n = int(need * 1.3) + 16
        if layout == "uniform":
            cand = rng.uniform(lo, hi, size=n)
        elif layout == "clustered":
            from_cluster = rng.uniform(size=n) < cluster_fraction
            which = rng.integers(0, n_clusters, size=n)
            cand = np.where(from_cluster, cc[which] + cluster_sigma * rng.standard_normal(n),
                            rng.uniform(-PI, PI, size=n))
            cand = _wrap(cand)
        else:
            raise ValueError(layout)
        cand = cand[~_excluded(cand, center, width, periodic)]
        out = np.concatenate([out, cand[:need]])
    return out


def make(name: str = "custom", *, M: int, bc: int, dt: float, Nt: int, tol: float = 1e-12,
         p: int = 8, seed: int = 7823, layout: str = "uniform",
         beta_range=(1.0, 10.0), beta_dist: str = "uniform",
         amp=(1.0,), center=(-2.0,), width=(0.1,), R: int = 4,
         xr: Optional[np.ndarray] = None, description: str = "",
         margin: float = FREE_MARGIN, n_clusters: int = 16) -> Workload:
    """Draw one seeded workload.  Springs avoid the pulse support at t = 0.

    margin: free space only, springs and receivers lie in [-pi + margin, pi - margin]; it must
    cover 3 delta = 3 W dt of the plan (Sec. 4.4).  n_clusters: Gaussian clusters of the
    clustered layout (fewer clusters at a smaller M keep the clusters' density)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = np.asarray(amp, dtype=np.float64)
    center = np.asarray(center, dtype=np.float64)
    width = np.asarray(width, dtype=np.float64)
    periodic = bc == PERIODIC
    if periodic:
        lo, hi = -PI, PI
    else:
        lo, hi = -PI + margin, PI - margin
    x = _draw_positions(rng, M, layout, periodic, center, width, lo, hi, n_clusters=n_clusters)
    if beta_dist == "uniform":
        beta = rng.uniform(beta_range[0], beta_range[1], size=M)
    elif beta_dist == "loguniform":
        beta = np.exp(rng.uniform(math.log(beta_range[0]), math.log(beta_range[1]), size=M))
    else:
        raise ValueError(beta_dist)
    if xr is None:
        if periodic:
            xr = -PI + (np.arange(R) + 0.5) * (2 * PI / R)
        else:
            xr = lo + (np.arange(R) + 0.5) * ((hi - lo) / R)
    return Workload(name=name, bc=bc, x=x.astype(np.float64), beta=beta.astype(np.float64),
                    amp=amp, center=center, width=width, dt=float(dt), Nt=int(Nt), tol=float(tol),
                    p=int(p), xr=np.asarray(xr, dtype=np.float64), seed=seed,
                    description=description)


# --- the five named workloads (shapes of the paper's experiments, Sec. 6) -----------------

def config0(**over) -> Workload:
    """Periodic box, M=64 uniform, beta~U[1,10], one pulse width 0.1 at x=-2, dt=0.01, T=10."""
    kw = dict(M=64, bc=PERIODIC, dt=0.01, Nt=1000, tol=1e-10, p=8, seed=7823 + 0,
              beta_range=(1.0, 10.0), amp=(1.0,), center=(-2.0,), width=(0.1,), R=4,
              description="periodic M=64 uniform, dt=1e-2, Nt=1000, tol=1e-10, p=8")
    kw.update(over)
    return make("periodic_M64_dt1e-2", **kw)


def config1(**over) -> Workload:
    """Free space, M=1e4 uniform, beta log-uniform [0.1,100], three pulses, dt=1e-3, T=20."""
    kw = dict(M=10_000, bc=FREE, dt=1e-3, Nt=20_000, tol=1e-12, p=8, seed=7823 + 1,
              beta_range=(0.1, 100.0), beta_dist="loguniform",
              amp=(1.0, 0.5, 0.25), center=(-PI - 0.3, -PI - 0.6, -PI - 1.0),
              width=(0.02, 0.05, 0.1), R=8,
              description="free space M=1e4 uniform, dt=1e-3, Nt=2e4, tol=1e-12, p=8")
    kw.update(over)
    return make("free_M1e4_dt1e-3", **kw)


def config2(**over) -> Workload:
    """Periodic box, M=1e6 clustered (16 Gaussians sigma=0.05 + 20% uniform), dt=5e-4, p=4.

    The interpolation order is not part of this workload's recipe.  Its clusters hold about 400
    springs per dt, and there the march with p = 8 (or 6) stencils is unstable: an impulse grows by
    x1.3 (x1.006) per step under the p nearest available samples of Sec. 4.1, while p = 4 and p = 2
    decay.  So p = 4, the highest order that is stable at this density."""
    kw = dict(M=1_000_000, bc=PERIODIC, dt=5e-4, Nt=10_000, tol=1e-10, p=4, seed=7823 + 2,
              layout="clustered", beta_range=(1.0, 10.0), amp=(1.0,), center=(-2.0,),
              width=(0.1,), R=4,
              description="periodic M=1e6 clustered, dt=5e-4, Nt=1e4, tol=1e-10, p=4")
    kw.update(over)
    return make("periodic_M1e6_clustered_dt5e-4", **kw)


def config3_instances(n_instances: int = 256, m_range=(1e2, 1e5), **over):
    """Batched: independent periodic instances, M log-uniform in m_range (default [1e2, 1e5]), dt=1e-3."""
    rng = np.random.Generator(np.random.PCG64(7823 + 3))
    Ms = np.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1]), size=n_instances)).astype(int)
    widths = rng.uniform(0.05, 0.2, size=n_instances)
    out = []
    for i in range(n_instances):
        kw = dict(M=int(Ms[i]), bc=PERIODIC, dt=1e-3, Nt=5000, tol=1e-12, p=8,
                  seed=7823 + 3 + 1000 * (i + 1), beta_range=(1.0, 10.0), amp=(1.0,),
                  center=(-2.0,), width=(float(widths[i]),), R=4)
        kw.update(over)
        out.append(make(f"batched_{i}", **kw))
    return out


def config4(**over) -> Workload:
    """Free space, M=1e5, beta~U[1,10], dt=1e-3, Nt=1e4, 8 receivers (adjoint workload)."""
    kw = dict(M=100_000, bc=FREE, dt=1e-3, Nt=10_000, tol=1e-12, p=8, seed=7823 + 4,
              beta_range=(1.0, 10.0), amp=(1.0,), center=(-PI - 0.6,), width=(0.05,), R=8,
              description="free space M=1e5, dt=1e-3, Nt=1e4, tol=1e-12, p=8")
    kw.update(over)
    return make("free_M1e5_dt1e-3", **kw)


def _gaussian_pulse_width(mu: float) -> float:
    """exp(-mu s^2) as exp(-s^2 / (2 width^2))."""
    return 1.0 / math.sqrt(2.0 * mu)


def fabry_perot(dt: float = 0.005, **over) -> Workload:
    """Sec. 6 (scattering by arrays of springs): two springs beta = 100 a unit distance apart at
    x = -0.5, 0.5 in free space, incident pulse exp(-mu (s - t0)^2) with mu = 5, t0 = -3 (eq.
    incidentPulse), over the paper's T = 94.26 (9426 steps of 0.01), p = 8; receivers at -1.8
    (reflected) and 1.8 (transmitted).  dt defaults to 0.005: with these stiffnesses the p = 8
    scheme is unstable at 0.01 (beta dt / 2 = 0.5)."""
    kw = dict(name="fabry_perot_M2", bc=FREE, x=np.array([-0.5, 0.5]), beta=np.array([100.0, 100.0]),
              amp=np.array([1.0]), center=np.array([-3.0]), width=np.array([_gaussian_pulse_width(5.0)]),
              dt=dt, Nt=int(round(94.26 / dt)), tol=1e-12, p=8, xr=np.array([-1.8, 1.8]), seed=0,
              description=f"free space, 2 springs beta=100 at +-0.5, mu=5, t0=-3, dt={dt}, T=94.26")
    kw.update(over)
    return Workload(**kw)


def uniform_array(M: int, beta: float, dt: float = 0.01, **over) -> Workload:
    """Sec. 6: M equally spaced springs of equal stiffness (the paper's examples: M = 10 with
    beta = 100 and M = 200 with beta = 1), here spanning [-1, 1] end to end (spacing 2 / (M - 1),
    which keeps pair distances off multiples of dt), in free space; pulse mu = 5, t0 = -4, over the
    paper's T = 251.34 (25134 steps of 0.01), p = 8; receivers at -1.8 and 1.8."""
    x = np.linspace(-1.0, 1.0, M)
    kw = dict(name=f"uniform_array_M{M}", bc=FREE, x=x, beta=np.full(M, float(beta)), amp=np.array([1.0]),
              center=np.array([-4.0]), width=np.array([_gaussian_pulse_width(5.0)]), dt=dt,
              Nt=int(round(251.34 / dt)), tol=1e-12, p=8, xr=np.array([-1.8, 1.8]), seed=0,
              description=f"free space, {M} springs beta={beta} evenly in [-1, 1], mu=5, t0=-4, dt={dt}")
    kw.update(over)
    return Workload(**kw)


def disordered_media(beta_max: float, seed: int = 7823 + 150, **over) -> Workload:
    """Sec. 6 (scattering in 1D disordered media): M = 150 springs at random positions in [-2, 2]
    with every pair at least 1e-4 apart, stiffnesses uniform in [0.1, beta_max] (the paper: 3, 5 and
    10), free space, pulse mu = 30, t0 = -3, dt = 3.703e-3 up to T = 10 pi (8484 steps), p = 8; the
    paper's 400 x 400 space-time readout as 100 receivers evenly across [-2.7, 2.7] at every step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.sort(rng.uniform(-2.0, 2.0, 150))
    while np.min(np.diff(x)) < 1e-4:                   # redraw the points that crowd a neighbour
        bad = np.nonzero(np.diff(x) < 1e-4)[0] + 1
        x[bad] = rng.uniform(-2.0, 2.0, bad.size)
        x = np.sort(x)
    kw = dict(name=f"disordered_M150_beta{beta_max:g}", bc=FREE, x=x, beta=rng.uniform(0.1, beta_max, 150),
              amp=np.array([1.0]), center=np.array([-3.0]), width=np.array([_gaussian_pulse_width(30.0)]),
              dt=3.703e-3, Nt=8484, tol=1e-12, p=8, xr=np.linspace(-2.7, 2.7, 100), seed=seed,
              description=f"free space, 150 random springs in [-2, 2], beta in [0.1, {beta_max:g}], mu=30, t0=-3")
    kw.update(over)
    return Workload(**kw)


CONFIGS = {0: config0, 1: config1, 2: config2, 4: config4}
