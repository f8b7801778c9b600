"""Host logic of the implicit solve (eq. linearSystem) without a GPU: the packed solve groups and
the tasks of large blocks, decoded as the step kernel decodes them, solve every spring exactly
once with row i of its block's inverse.  Layouts with blocks of 1 .. 33 members (packing edge
cases around 32 lanes), of 200 (32-row tasks, staged right-hand sides) and of 300 members (the
single-task path above 256)."""
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
    out = os.path.join(build_dir, "solve_tables_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "solve_tables_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _chains(sizes, dt, lo=-1.9):
    """Blocks of the given sizes: springs 0.4 dt apart inside a block, blocks 3 dt apart."""
    xs, x = [], lo
    for s in sizes:
        xs.extend(x + 0.4 * dt * np.arange(s))
        x = xs[-1] + 3.0 * dt
    return np.array(xs)


@pytest.mark.parametrize("sizes", [[1, 2, 31, 1, 32, 33, 5, 16, 17, 1, 30, 3, 29],
                                   [200, 3, 1], [300, 2], [33, 64, 65, 2]])
def test_solve_tasks_cover_every_spring_with_its_block_row(checker, sizes):
    dt = 0.01
    x = _chains(sizes, dt)
    assert x[-1] < 1.9
    beta = np.random.default_rng(len(sizes)).uniform(1.0, 10.0, x.size)
    text = f"{x.size} {dt!r}\n" + " ".join(repr(float(v)) for v in x) + "\n" + " ".join(repr(float(v)) for v in beta) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
    _, err, largest = r.stdout.split()
    assert float(err) < 1e-12 and int(largest) == max(sizes)
