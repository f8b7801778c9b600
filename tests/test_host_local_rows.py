"""Host logic of the local sum (Sec. 4.1) without a GPU: the m-ordered rows and the 32-source work
items the step kernel reads must reproduce the plain weight table row by row, for the springs
(m >= 1) and for the receivers (m >= 0) (to the FP32-pair
rounding of the stored weights, about 2^-48 of the sum of the terms' magnitudes).  Layouts: random
springs, springs spaced exactly dt apart (pair distances on dt and on delta within rounding, where
a source with no weights once broke the rows), a dense cluster, and a periodic box."""
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
    out = os.path.join(build_dir, "host_rows_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "host_rows_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _worst(checker, x, beta, dt, tol, bc, xr):
    text = f"{len(x)} {dt!r} {tol!r} {bc} {len(xr)}\n" + " ".join(repr(float(v)) for v in x) + "\n" + \
        " ".join(repr(float(v)) for v in beta) + "\n" + " ".join(repr(float(v)) for v in xr) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True, check=True)
    return float(r.stdout.split()[0])


@pytest.mark.parametrize("layout", ["random", "spacing_dt", "cluster", "periodic"])
def test_rows_and_items_reproduce_the_weight_table(checker, layout):
    rng = np.random.default_rng(3)
    dt, tol, bc = 0.01, 1e-12, 1
    if layout == "random":
        x = np.sort(rng.uniform(-1.5, 1.5, 400))
    elif layout == "spacing_dt":
        x = -1.0 + (np.arange(200) + 0.5) * (2.0 / 200)
    elif layout == "cluster":
        x = np.sort(np.concatenate([0.3 + 0.02 * rng.standard_normal(300), rng.uniform(-1.5, 1.5, 100)]))
    else:
        x, bc = np.sort(rng.uniform(-np.pi, np.pi, 300)), 0
    beta = rng.uniform(1.0, 10.0, x.size)
    # receivers: among the springs, one exactly on a spring, one a spacing away
    xr = np.array([-1.2, float(x[5]), float(x[5]) + 0.01, 0.0, 1.3])
    assert _worst(checker, x, beta, dt, tol, bc, xr) < 1e-13
