"""The mixed-precision time step runs the standalone FP32 NUFFT kernels (tol 1e-6, width 7) on the
plan's springs and hands their grid to the plan's own FFT, mode update and deconvolution.  That is
exact only if a plan built with NUFFT width 7 and the standalone plan share fine grid, FFT split,
kernel shape, spreading weights and deconvolution factors; checked here bit for bit on the host,
periodic and free space, for several time steps (hence fine grids)."""
import os
import shutil
import subprocess

import numpy as np
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
    out = os.path.join(build_dir, "mixed_grid_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "mixed_grid_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.mark.parametrize("bc,dt,tol", [(0, 0.01, 1e-10), (1, 0.005, 1e-12), (0, 1e-3, 1e-12), (1, 0.02, 1e-8)])
def test_width7_plan_and_mixed_nufft_share_grid_kernel_and_deconvolution(checker, bc, dt, tol):
    rng = np.random.default_rng(11)
    x = np.sort(rng.uniform(-1.0, 1.0, 50))
    beta = rng.uniform(1.0, 10.0, x.size)
    text = f"{x.size} {dt!r} {tol!r} {bc} 8\n" + " ".join(repr(float(v)) for v in x) + "\n" + \
        " ".join(repr(float(v)) for v in beta) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
    assert int(r.stdout.split()[2]) == 7
