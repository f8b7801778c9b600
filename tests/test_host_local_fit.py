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
