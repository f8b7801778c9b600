"""The bodies of the GPU reverse-time march (csrc/adjoint.cuh) checked without a GPU: a host
harness runs them, one element at a time in the kernels' launch order, over the tables the plan
builder makes (local-sum items of springs and receivers, m = 0 receiver terms, block inverses,
FIR and rotation tables, projection tables), with exact Fourier sums in place of the library's
NUFFT plan, and its dL/dbeta must equal the adjoint oracle's (oracle/adjoint.py), which is
pinned by finite differences and by the complex-step derivative of the direct march."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import adjoint, wfp
from paper_2507_07823_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2507_07823_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")


@pytest.fixture(scope="module")
def harness():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    build_dir = os.path.join(HERE, "native", "_build")         # git-ignored, inside the repository
    os.makedirs(build_dir, exist_ok=True)
    out = os.path.join(build_dir, "adjoint_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "adjoint_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _run(harness, w, sigma, ubar, g=None):
    """dL/dbeta (and dL/dg, Nt x M, when the march is driven by forcing vectors g) from the
    harness; sigma, ubar and g hold rows 1 .. Nt."""
    text = f"{w.M} {len(w.xr)} {w.bc} {w.dt!r} {w.tol!r} {w.p} {w.Nt} {int(g is not None)}\n"
    arrays = (w.x, w.beta, w.xr, sigma.ravel(), ubar.ravel()) + ((g.ravel(),) if g is not None else ())
    for arr in arrays:
        text += " ".join(repr(float(v)) for v in arr) + "\n"
    r = subprocess.run([harness], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    out = np.array([float(v) for v in r.stdout.split()[1:]])
    if g is None:
        return out
    return out[:w.M], out[w.M:].reshape(w.Nt, w.M)


def _layout(bc, seed, M, p, dt, Nt, block):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(-0.8, 0.8, M))
    for i in range(1, block):                       # a block of `block` springs closer than dt
        x[2 + i] = x[2] + 0.4 * dt * i
    x = np.sort(x)
    beta = rng.uniform(1.0, 6.0, M)
    xr = np.array([-0.95, 0.1, x[M // 2], 0.95])    # one receiver on a spring (m = 0 terms)
    return W.Workload(name="adjoint", bc=bc, x=x, beta=beta, amp=np.array([1.0]), center=np.array([-1.6]),
                      width=np.array([0.12]), dt=dt, Nt=Nt, tol=1e-10, p=p, xr=xr, seed=seed)


@pytest.mark.parametrize("bc,p,block", [(W.PERIODIC, 6, 2), (W.FREE, 6, 2), (W.PERIODIC, 8, 3),
                                        (W.FREE, 4, 4)])
def test_adjoint_bodies_match_the_oracle_gradient(harness, bc, p, block):
    w = _layout(bc, seed=11 + p + block, M=10, p=p, dt=0.02, Nt=400, block=block)
    sigma, u = wfp.from_workload(w).run(w.Nt)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])
    ubar = u[1:] - d[1:]
    o = wfp.from_workload(w)
    if bc == W.FREE:
        assert w.Nt >= 2 * o.P.rbc_period                 # several projections inside the march
    _, g_oracle = adjoint.misfit_and_gradient(o, w.Nt, d)
    g = _run(harness, w, sigma[1:], ubar)
    assert np.max(np.abs(g - g_oracle)) <= 1e-12 * np.max(np.abs(g_oracle)), (g, g_oracle)


PI = np.pi
EDGE_LAYOUTS = {
    # a pair closer than dt across the periodic seam, a receiver on the seam
    "seam_pair": (W.PERIODIC, [-PI + 0.003, -0.5, 0.1, 0.4, 1.0, PI - 0.004], 6, [PI - 0.001, 0.2, -PI + 0.01], 300),
    # springs at one position (distance 0 between distinct springs), a receiver on them
    "duplicates": (W.FREE, [-0.5, -0.2, -0.2, -0.19, 0.3, 0.7], 6, [-0.2, 0.5], 300),
    # a chain of six springs 0.9 dt apart: one block of six
    "chain": (W.FREE, list(-0.3 + 0.018 * np.arange(6)) + [0.5, 0.9], 8, [-0.95, 0.1, 0.95], 300),
    # springs dt apart: pair distances on the near / far switch within rounding
    "spacing_dt": (W.FREE, list(-0.4 + 0.02 * np.arange(8)), 4, [-0.95, 0.1, 0.95], 300),
    # thirty springs filling the periodic box
    "periodic_dense": (W.PERIODIC, list(np.sort(np.random.default_rng(4).uniform(-PI, PI, 30))), 8,
                       [-0.95, 0.1, 0.95], 200),
}


@pytest.mark.parametrize("name", sorted(EDGE_LAYOUTS))
def test_adjoint_bodies_on_edge_layouts(harness, name):
    """The same comparison on layouts whose tables have edge cases: implicit blocks across the
    periodic seam, coincident springs, a long chain, distances on the near / far switch."""
    bc, x, p, xr, Nt = EDGE_LAYOUTS[name]
    x = np.array(x, dtype=np.float64)
    beta = np.random.default_rng(1).uniform(1.0, 6.0, x.size)
    w = W.Workload(name=name, bc=bc, x=x, beta=beta, amp=np.array([1.0]), center=np.array([-1.6]),
                   width=np.array([0.12]), dt=0.02, Nt=Nt, tol=1e-10, p=p, xr=np.array(xr, dtype=np.float64),
                   seed=1)
    sigma, u = wfp.from_workload(w).run(w.Nt)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])
    _, g_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d)
    g = _run(harness, w, sigma[1:], u[1:] - d[1:])
    assert np.max(np.abs(g - g_oracle)) <= 1e-12 * np.max(np.abs(g_oracle)), (g, g_oracle)


@pytest.mark.parametrize("bc", [W.PERIODIC, W.FREE])
def test_adjoint_bodies_with_forcing_vectors(harness, bc):
    """A march driven by forcing vectors g (not scaled by beta): dL/dbeta with the term
    (sigma_j + g_j) / beta_j and dL/dg = -rhsbar against the adjoint oracle."""
    w = _layout(bc, seed=21, M=10, p=6, dt=0.02, Nt=300, block=2)
    rng = np.random.default_rng(5)
    g = 0.2 * rng.standard_normal((w.Nt + 1, w.M))
    sigma, u = wfp.from_workload(w).run(w.Nt, g)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])
    _, gb_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d, g=g)
    gg_oracle = adjoint.forcing_gradient(wfp.from_workload(w), w.Nt, d, g)
    gb, gg = _run(harness, w, sigma[1:], u[1:] - d[1:], g[1:])
    assert np.max(np.abs(gb - gb_oracle)) <= 1e-12 * np.max(np.abs(gb_oracle)), (gb, gb_oracle)
    assert np.max(np.abs(gg - gg_oracle[1:])) <= 1e-12 * np.max(np.abs(gg_oracle[1:]))
