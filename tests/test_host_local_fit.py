"""Piecewise-polynomial local weights (csrc/local_fit.h, for weights computed from pair distances)
against the plan's own stored-weight rule on the host: the breakpoints are those of the Gauss-Legendre
nodes crossing multiples of dt (and d = dt), and the per-interval Chebyshev series of degree 7
reproduce Q_m(d) within 1e-12 of max |Q| (degree 3 within 1e-5), the same figures the oracle's
weights give (tests/test_oracle_local_weight_fits.py)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2507_07823_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")


@pytest.fixture(scope="module")
def checker():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    build_dir = os.path.join(HERE, "native", "_build")         # git-ignored, inside the repository
    os.makedirs(build_dir, exist_ok=True)
    out = os.path.join(build_dir, "local_fit_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "local_fit_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("dt,tol,deg,bar", [(1e-3, 1e-12, 7, 1e-12), (0.01, 1e-12, 7, 1e-12), (1e-3, 1e-12, 3, 1e-5),
                                            (5e-4, 1e-6, 5, 1e-7)])
def test_piecewise_fit_reproduces_the_plan_rule(checker, dt, tol, deg, bar):
    r = subprocess.run([checker], input=f"{dt!r} {tol!r} 8 {deg} 400\n", capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
    _, n, size, err = r.stdout.split()
    assert float(err) < bar, r.stdout
    if tol == 1e-12:
        # about N_L W / 2 intervals (W = N_L = 36): the oracle's breakpoints give 636, the builder
        # merges the few closer than 1e-15 delta
        assert 600 <= int(n) <= 640, r.stdout


@pytest.fixture(scope="module")
def rows_checker():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    build_dir = os.path.join(HERE, "native", "_build")
    os.makedirs(build_dir, exist_ok=True)
    out = os.path.join(build_dir, "local_fit_rows_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "local_fit_rows_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("bc,dt,layout", [(1, 1e-3, "uniform"), (0, 1e-3, "cluster"), (0, 0.01, "seam")])
def test_local_sums_from_pair_distances_match_stored_weights(rows_checker, bc, dt, layout):
    """Every spring row's local sum (m >= 1) with weights evaluated per pair (bisection into the
    breakpoints, the interval's non-zero m range, Clenshaw) at distances recomputed from the
    positions, against the plan's stored FP64 weights: within 1e-12 of the largest row sum."""
    import numpy as np
    rng = np.random.default_rng(9)
    if layout == "uniform":
        x = np.sort(rng.uniform(-2.5, 2.5, 2000))
    elif layout == "cluster":
        x = np.sort(np.concatenate([0.4 + 0.01 * rng.standard_normal(600), rng.uniform(-np.pi, np.pi, 400)]))
    else:                                           # pairs across the periodic seam
        x = np.sort(np.concatenate([np.pi - 0.05 * rng.random(40), -np.pi + 0.05 * rng.random(40), rng.uniform(-3, 3, 200)]))
    text = f"{x.size} {dt!r} 1e-12 {bc} 7\n" + " ".join(repr(float(v)) for v in x) + "\n"
    r = subprocess.run([rows_checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
    _, err, pairs = r.stdout.split()
    assert float(err) < 1e-12 and int(pairs) > x.size, r.stdout


@pytest.fixture(scope="module")
def fly_checker():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    build_dir = os.path.join(HERE, "native", "_build")
    os.makedirs(build_dir, exist_ok=True)
    out = os.path.join(build_dir, "fly_items_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "fly_items_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("bc,dt", [(1, 1e-3), (0, 0.01)])
def test_computed_weight_items_match_stored_rows(fly_checker, bc, dt):
    """The traversal of the local sum with weights computed per pair (the step's items, their real
    source counts, distances from the positions, m >= 1), for spring rows and receiver rows, against
    the stored FP64 weights: within 1e-12 of the largest row sum."""
    import numpy as np
    rng = np.random.default_rng(13)
    lim = 2.5 if bc == 1 else np.pi
    x = np.sort(np.concatenate([rng.uniform(-lim, lim, 700), 0.2 + 0.003 * rng.standard_normal(100)]))
    xr = np.array([-1.0, 0.2, float(x[10]), 1.7])                # one receiver on a spring
    text = f"{x.size} {xr.size} {dt!r} 1e-12 {bc}\n" + " ".join(repr(float(v)) for v in x) + "\n" + \
        " ".join(repr(float(v)) for v in xr) + "\n"
    r = subprocess.run([fly_checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
    assert float(r.stdout.split()[1]) < 1e-12, r.stdout
