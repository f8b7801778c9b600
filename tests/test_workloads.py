"""The seeded workloads keep the paper's hypotheses (Sec. 1: no spring in supp f at t = 0;
Sec. 4.4: free-space springs inside Omega)."""
import math

import numpy as np

from paper_2507_07823_gb300 import workloads as W


def _pdist(a, b):
    d = np.abs(a - b) % (2 * math.pi)
    return np.minimum(d, 2 * math.pi - d)


def test_config_shapes_and_seeds():
    w0 = W.config0()
    assert w0.M == 64 and w0.Nt == 1000 and w0.bc == W.PERIODIC and w0.R == 4
    assert np.array_equal(w0.x, W.config0().x)                 # seeded, reproducible
    assert np.all((w0.beta >= 1) & (w0.beta <= 10))
    w1 = W.config1(M=2000)
    assert w1.bc == W.FREE and w1.Nt == 20000 and w1.R == 8
    assert np.all((w1.beta >= 0.1) & (w1.beta <= 100))


def test_springs_avoid_pulse_support():
    for w in (W.config0(), W.config1(M=3000), W.config2(M=20000)):
        for c, wd in zip(w.center, w.width):
            d = _pdist(w.x, c) if w.bc == W.PERIODIC else np.abs(w.x - c)
            assert np.min(d) >= 8 * wd


def test_free_space_springs_inside_omega():
    w = W.config1(M=5000)
    # Omega = [-pi + 3 delta, pi - 3 delta] with delta = W dt <= 0.039 for eps >= 1e-13, dt = 1e-3
    assert np.max(np.abs(w.x)) <= math.pi - W.FREE_MARGIN
    assert np.max(np.abs(w.xr)) <= math.pi - W.FREE_MARGIN


def test_clustered_layout_is_clustered():
    w = W.config2(M=50000)
    hist, _ = np.histogram(w.x, bins=256, range=(-math.pi, math.pi))
    assert hist.max() > 20 * np.percentile(hist, 10)
