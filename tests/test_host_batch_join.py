"""Joined tables of a batched plan (csrc/batch_host.cpp) checked on the CPU against the instances'
own tables: local sums of springs and receivers, the receivers' m = 0 terms and the block solves bit
for bit, every spring solved once by the packed groups with its own item range, and the permutation.
Instances of uneven sizes (1 spring to a few hundred, dense clusters with implicit blocks, the
periodic seam), some without receivers."""
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
    out = os.path.join(build_dir, "batch_join_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "batch_join_check.cpp"), os.path.join(CSRC, "plan_host.cpp"),
           os.path.join(CSRC, "batch_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def test_joined_tables_reproduce_every_instance(checker):
    rng = np.random.default_rng(17)
    dt, tol, p = 0.01, 1e-10, 8
    inst = []
    for M in (1, 7, 40, 300, 2, 120):
        x = rng.uniform(-np.pi, np.pi, M)
        if M >= 40:
            x[:5] = 0.3 + 0.004 * np.arange(5)                 # a block of five springs
            x[5] = np.pi - 0.002                               # and a pair across the seam
            x[6] = -np.pi + 0.003
        beta = rng.uniform(1.0, 10.0, M)
        R = 0 if M in (2, 120) else 3
        xr = rng.uniform(-np.pi, np.pi, R)
        inst.append((x, beta, xr))
    text = f"{len(inst)} {dt!r} {tol!r} {p}\n"
    for x, beta, xr in inst:
        text += f"{x.size} {xr.size}\n"
        for arr in (x, beta, xr):
            text += " ".join(repr(float(v)) for v in arr) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    _, M, R, items = r.stdout.split()
    assert int(M) == sum(x.size for x, _, _ in inst) and int(R) == 12 and int(items) > 0
