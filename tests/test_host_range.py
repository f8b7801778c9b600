"""Local sums of plans without pair lists (opts.local_weights = 1), on the host.

The harness tests/native/range_check.cpp compiles the plan builder (csrc/plan_host.cpp) and the
pair arithmetic of csrc/range.cuh with -ffp-contract=off and runs the k_rs_local kernel's traversal
(chunks of 32 sources, interval windows walked once per source, chunks with few pairs per e-vector
folding one per pair, blocks spanning more than two window widths walking each target's own
sources; the interval walk, the e-vectors, the compensated accumulator) on the CPU:

* the distance polynomials of the range tables reproduce the plan's own weight rule Q_m(d)
  (Sec. 4.1: N_L-point Gauss-Legendre over [d, delta] of (1 - phi) times the p-point interpolant)
  within 1e-14 of max |Q| as FP64 Chebyshev series and within 2e-12 as the float-pair monomials the
  device evaluates;
* the local sums of every spring equal those of the stored FP64 weights of an ordinary plan: within
  2e-12 of the largest row sum where rows hold thousands of pairs, 4e-11 where they hold a few (the
  single-float rounding of each source's curvature terms, which averages out over many sources);
* the reverse march's transposed sums per m (its own traversal, moments flushed per interval)
  equal the stored weights' within 1e-9.
"""
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
    out = os.path.join(build_dir, "range_check")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "range_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _run(exe, text):
    r = subprocess.run([exe], input=text, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    return r.stdout.split()[1:]


@pytest.mark.parametrize("dt,tol", [(5e-4, 1e-10), (1e-3, 1e-12), (0.01, 1e-12)])
def test_distance_polynomials_reproduce_the_rule(checker, dt, tol):
    nint, e64, e32 = _run(checker, f"fit 1 {dt!r} {tol!r} 0\n0.0\n")
    assert float(e64) < 1e-14 and float(e32) < 2e-12, (nint, e64, e32)
    # about N_L W / 2 breakpoints of the rule, plus the cuts of intervals wider than 0.15 dt
    assert 400 <= int(nint) <= 800


def _layout(name, rng):
    if name == "uniform":
        return 1, 1e-3, 1e-12, np.sort(rng.uniform(-2.5, 2.5, 2000))
    if name == "cluster":
        return 0, 1e-3, 1e-12, np.sort(np.concatenate([0.4 + 0.01 * rng.standard_normal(600),
                                                       rng.uniform(-np.pi, np.pi, 400)]))
    if name == "seam":          # pairs across the periodic seam, a block spanning the whole box
        return 0, 0.01, 1e-12, np.sort(np.concatenate([np.pi - 0.05 * rng.random(40),
                                                       -np.pi + 0.05 * rng.random(40), rng.uniform(-3, 3, 200)]))
    if name == "coincident":    # equal positions and pairs exactly dt apart
        base = np.sort(rng.uniform(-1.0, 1.0, 300))
        return 1, 1e-3, 1e-12, np.sort(np.concatenate([base, base[:50], base[50:80] + 1e-3]))
    if name == "single":
        return 1, 1e-3, 1e-12, np.array([0.0])
    if name == "grouped":       # groups of 100 springs dt / 12 apart, 1.5 dt between groups: chunks
        dt = 0.01               # whose interval ranges take many e-vector windows
        period = 100 * dt / 12 + 1.5 * dt
        return 1, dt, 1e-12, np.sort(np.concatenate([-1.0 + k * period + np.arange(100) * dt / 12
                                                     + rng.uniform(0, dt / 60, 100) for k in range(20)]))
    if name == "sparse":        # blocks of 256 springs spanning several window widths
        return 0, 1e-3, 1e-12, np.sort(rng.uniform(-np.pi, np.pi, 3000))
    raise ValueError(name)


@pytest.mark.parametrize("name,bar", [("uniform", 4e-11), ("cluster", 4e-12), ("seam", 4e-11),
                                      ("coincident", 4e-11), ("single", 4e-11), ("grouped", 1e-11),
                                      ("sparse", 4e-11)])
def test_range_sums_match_stored_weights(checker, name, bar):
    bc, dt, tol, x = _layout(name, np.random.default_rng(9))
    text = f"sum {x.size} {dt!r} {tol!r} {bc}\n" + " ".join(repr(float(v)) for v in x) + "\n"
    err, pairs = _run(checker, text)
    assert float(err) < bar and int(pairs) >= x.size, (err, pairs)


@pytest.mark.parametrize("name", ["uniform", "cluster", "seam", "coincident", "single", "grouped", "sparse"])
def test_transposed_range_sums_match_stored_weights(checker, name):
    """The reverse march's transposed local sums out_j[m] = sum_e Q_m(d_je) cbar_e (m >= 1) through
    the k_rs_local_T kernel's traversal (each output walking the forward block's window, the
    moments of its current interval flushed per m when the interval changes) against the stored
    FP64 weights: within 1e-9 of the largest sum (the curvature moments are single floats, about
    3e-10 here; a dropped or doubled pair would show at 1e-3)."""
    bc, dt, tol, x = _layout(name, np.random.default_rng(9))
    text = f"tsum {x.size} {dt!r} {tol!r} {bc}\n" + " ".join(repr(float(v)) for v in x) + "\n"
    err, pairs = _run(checker, text)
    assert float(err) < 1e-9 and int(pairs) >= 1, (err, pairs)


def test_range_sums_at_clustered_million_spring_density(checker):
    """The clustered layout of the million-spring workload (16 Gaussian clusters of width 0.05 and
    20 % uniform springs, dt = 5e-4, tol = 1e-10) thinned to 4000 springs."""
    from paper_2507_07823_gb300 import workloads as W
    w = W.config2(M=4000, width=(0.005,))
    x = np.sort(w.x)
    text = f"sum {x.size} {w.dt!r} {w.tol!r} 0\n" + " ".join(repr(float(v)) for v in x) + "\n"
    err, pairs = _run(checker, text)
    assert float(err) < 4e-11, (err, pairs)
