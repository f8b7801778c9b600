"""Host logic of the NUFFT spreading ranges (nufft_ranges, no GPU): for clustered, uniform,
sparse, one-giant-cell and seam-straddling point sets, single and batched, with several kernel
widths and caps, the ranges tile every instance's grid once, each run stages exactly its cell's
points (the halo wrapping round the periodic box), empty ranges have no point in reach, and
spreading through the ranges equals direct spreading."""
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
    out = os.path.join(build_dir, "nufft_ranges_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "nufft_ranges_check.cpp"), os.path.join(CSRC, "plan_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _cells(rng, kind, m, nf):
    if kind == "uniform":
        c = rng.integers(0, nf, m)
    elif kind == "cluster":
        c = (nf // 3 + np.round(3 * rng.standard_normal(m))).astype(int) % nf
    elif kind == "sparse":
        c = rng.choice(np.arange(0, nf, max(1, nf // 7)), m)
    elif kind == "giant":
        c = np.full(m, int(rng.integers(0, nf)))
    else:                                               # points on both sides of the seam
        c = np.concatenate([rng.integers(0, 2, m // 2), rng.integers(nf - 2, nf, m - m // 2)])
    return np.sort(c)


@pytest.mark.parametrize("kinds", [("uniform",), ("cluster",), ("sparse",), ("giant",), ("seam",),
                                   ("cluster", "seam", "sparse", "giant", "uniform")])
# the plans' caps, the autotuner's smaller candidates (mixed: 60 / 120 cells x 512 / 1024 points;
# FP64: 32 / 64 x 1024 / 2048) and a tiny set
@pytest.mark.parametrize("w,caps", [(7, (240, 2048, 8192)), (11, (128, 4096, 8192)), (4, (16, 64, 32)),
                                    (7, (60, 512, 8192)), (7, (120, 1024, 8192)), (13, (32, 1024, 8192)),
                                    (13, (64, 2048, 8192))])
def test_ranges_tile_the_grids_and_reproduce_direct_spreading(checker, kinds, w, caps):
    rng = np.random.default_rng(hash((kinds, w)) % 2**32)
    for nf in (64, 1024):
        sizes = [int(rng.integers(1, 5000)) for _ in kinds]
        cells = [_cells(rng, k, m, nf) for k, m in zip(kinds, sizes)]
        offsets = np.concatenate([[0], np.cumsum(sizes)])
        max_cells, max_points, empty = caps
        text = f"{len(kinds)} {nf} {w} {max_cells} {max_points} {empty} 256\n" + \
            " ".join(str(int(v)) for v in offsets) + "\n" + " ".join(str(int(v)) for v in np.concatenate(cells)) + "\n"
        r = subprocess.run([checker], input=text, capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
        assert float(r.stdout.split()[1]) < 1e-12
