"""The split of a batched plan's instances by form (csrc/batch_host.cpp, batch_instances), on the
host: with local_weights = 2 an instance goes without pair lists when its largest block of springs
closer than dt passes opts.max_block, when more than 2^19 ordered pairs of its springs lie closer
than delta, or when its stored weights (8 bytes each) would pass what is left of opts.max_local_bytes
after the joined instances before it (their work items' bytes); local_weights = 0 joins every
instance and 1 none.  Expected forms come from a brute-force pair count and union-find in numpy and
from the budget rule applied in instance order to each instance's own weight sizes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from test_host_instance_shape import _brute

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2507_07823_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")
DT, TOL = 0.01, 1e-10          # W = 30, delta = 0.3


@pytest.fixture(scope="module")
def checker():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    build_dir = os.path.join(HERE, "native", "_build")         # git-ignored, inside the repository
    os.makedirs(build_dir, exist_ok=True)
    out = os.path.join(build_dir, "batch_forms_check")
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-o", out,
           os.path.join(HERE, "native", "batch_forms_check.cpp"), os.path.join(CSRC, "plan_host.cpp"),
           os.path.join(CSRC, "batch_host.cpp"), "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _instances():
    rng = np.random.default_rng(23)
    xs = [rng.uniform(-np.pi, np.pi, M) for M in (60, 250, 40, 120)]
    xs.insert(2, rng.uniform(-np.pi, np.pi, 2600))                       # more than 2^19 pairs
    xs.insert(4, np.sort(np.concatenate([0.5 + 0.002 * np.arange(90),   # one block of 90 springs
                                          rng.uniform(-3.0, -1.0, 30)])))
    xs.append(rng.uniform(-np.pi, np.pi, 1500))                          # below 2^19 pairs
    return xs


def _run(checker, xs, lw, max_block, max_bytes):
    text = f"{len(xs)} {DT!r} {TOL!r} {lw} {max_block} {max_bytes}\n"
    text += "\n".join(f"{len(x)} " + " ".join(repr(float(v)) for v in x) for x in xs) + "\n"
    r = subprocess.run([checker], input=text, capture_output=True, text=True, check=True)
    lines = r.stdout.split("\n")
    if lines[0].startswith("error"):
        return None, lines[0]
    forms = [int(v) for v in lines[0].split()[1:]]
    joined = {int(a): (int(b), int(c)) for _, a, b, c in (ln.split() for ln in lines[1:] if ln.startswith("joined"))}
    return forms, joined


def _shape_forms(xs, max_block):
    delta = 30 * DT
    return [int(b > max_block or p > 2**19) for b, p in (_brute(x, DT, delta) for x in xs)]


def test_local_weights_0_and_1_take_every_instance_one_way(checker):
    xs = _instances()
    forms, joined = _run(checker, xs, 0, 4096, 1 << 34)
    assert forms == [0] * len(xs) and sorted(joined) == list(range(len(xs)))
    forms, joined = _run(checker, xs, 1, 4096, 1 << 34)
    assert forms == [1] * len(xs) and joined == {}


@pytest.mark.parametrize("max_block", [64, 4096])
def test_shape_rule(checker, max_block):
    xs = _instances()
    want = _shape_forms(xs, max_block)
    assert sum(want) >= 1 and want[2] == 1
    forms, joined = _run(checker, xs, 2, max_block, 1 << 34)
    assert forms == want
    assert sorted(joined) == [b for b, f in enumerate(want) if f == 0]


def test_budget_rule_in_instance_order(checker):
    xs = _instances()
    shape = _shape_forms(xs, 4096)
    _, sizes = _run(checker, xs, 0, 4096, 1 << 34)          # each instance's own weight sizes
    budget = sizes[1][1] + sizes[0][1] + sizes[3][0] // 2   # the first two fit, the fourth does not
    want, used = [], 0
    for b in range(len(xs)):
        if shape[b]:
            want.append(1)
        elif sizes[b][0] > budget - used:
            want.append(1)
        else:
            want.append(0)
            used += sizes[b][1]
    assert 0 < sum(want) - sum(shape) < len(xs) - sum(shape)
    forms, _ = _run(checker, xs, 2, 4096, budget)
    assert forms == want
    # with local_weights = 0 the same budget is an error naming the instance
    forms, msg = _run(checker, xs, 0, 4096, budget)
    assert forms is None and "instance" in msg and "budget" in msg
