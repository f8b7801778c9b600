"""The two sizes that choose an instance's form in a batched plan with local_weights = 2
(csrc/batch_host.cpp, instance_shape): the largest block of springs closer than dt (the connected
components of eq. linearSystem's nearby graph) and the ordered pairs closer than delta (the local
sum's, Sec. 4.1), both in the periodic box.  Checked against brute force over every pair: a union-find
over the pairs closer than dt, and a count of the pairs closer than delta, on layouts with the
periodic seam inside a block, coincident springs, one spring, one block of everything, and
positions given outside [-pi, pi)."""
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
    out = os.path.join(build_dir, "instance_shape_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "instance_shape_check.cpp"), os.path.join(CSRC, "plan_host.cpp"),
           os.path.join(CSRC, "batch_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _shape(checker, x, dt, delta):
    text = f"{len(x)} {dt!r} {delta!r}\n" + "\n".join(repr(float(v)) for v in x) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True, check=True)
    a, b = r.stdout.split()
    return int(a), int(b)


def _brute(x, dt, delta):
    x = np.asarray(x, dtype=np.float64)
    M = len(x)
    d = np.abs(x[:, None] - x[None, :])
    d = np.minimum(np.mod(d, 2 * np.pi), 2 * np.pi - np.mod(d, 2 * np.pi))
    off = ~np.eye(M, dtype=bool)
    pairs = int(np.sum((d < delta) & off))
    parent = list(range(M))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for i, j in zip(*np.nonzero((d < dt) & off)):
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[ri] = rj
    roots = [find(i) for i in range(M)]
    return int(np.max(np.bincount(roots))), pairs


def _layouts():
    rng = np.random.default_rng(5)
    yield "uniform", rng.uniform(-np.pi, np.pi, 400), 0.01, 0.1
    # a dense cluster across the seam, plus sparse springs
    seam = np.concatenate([np.pi - rng.uniform(0, 0.05, 40), -np.pi + rng.uniform(0, 0.05, 40),
                           rng.uniform(-2.5, 2.5, 30)])
    yield "seam", seam, 0.004, 0.2
    coinc = np.repeat(rng.uniform(-3, 3, 50), 3)
    yield "coincident", coinc, 1e-6, 0.05
    yield "one", np.array([0.3]), 0.01, 0.1
    yield "everything", np.linspace(-np.pi, np.pi, 300, endpoint=False), 0.05, 0.3
    yield "outside the box", rng.uniform(-3 * np.pi, 3 * np.pi, 200), 0.02, 0.15


@pytest.mark.parametrize("case", list(_layouts()), ids=lambda c: c[0])
def test_instance_shape_matches_brute_force(checker, case):
    _, x, dt, delta = case
    # positions on a grid of 2^-20: no pair distance lands within rounding of dt or delta
    x = np.round(np.asarray(x) * 2.0**20) / 2.0**20
    dt, delta = dt + 2.0**-22, delta + 2.0**-22
    assert _shape(checker, x, dt, delta) == _brute(x, dt, delta)
