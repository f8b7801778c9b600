"""The local weights Q_m(d) (Sec. 4.1, the N_L-point Gauss-Legendre rule over [d, delta]) as
functions of the distance d: smooth between breakpoints, which are the distances where a
quadrature node d + (delta - d)(g_i + 1)/2 crosses a multiple of dt, plus d = dt, where the
near/far rule switches.  So per-interval polynomials can stand for the stored weights when those do
not fit the device (weights computed from a pair's distance).  Pinned here on the oracle's own
Q_m: degree-7 Chebyshev fits on every interval reproduce it within 1e-12 of max |Q|, and degree 3
within 1e-5."""
import numpy as np
import pytest

from oracle import wfp


def _breakpoints(P):
    g, _ = np.polynomial.legendre.leggauss(P.NL)
    c = (g + 1) / 2
    bps = [0.0, P.dt, P.delta]
    for ci in c:
        for k in range(P.W + 2):
            d = (k * P.dt - P.delta * ci) / (1 - ci)
            if 0 < d < P.delta:
                bps.append(d)
    return np.unique(np.array(bps))


@pytest.mark.parametrize("dt,deg,bar", [(1e-3, 7, 1e-12), (0.01, 7, 1e-12), (1e-3, 3, 1e-5)])
def test_local_weights_are_piecewise_smooth_between_breakpoints(dt, deg, bar):
    P = wfp.params(dt, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    bps = _breakpoints(P)
    assert len(bps) - 1 < P.NL * (P.W + 2)                        # about N_L W / 2 intervals
    scale = np.max(np.abs(wfp.local_weights(np.linspace(0.0, 0.999 * P.delta, 400), P, win)))
    z = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    zt = np.linspace(-0.97, 0.97, 5)
    worst = 0.0
    for a, b in zip(bps[:-1], bps[1:]):
        if b - a < 1e-15:
            continue
        coef = np.polynomial.chebyshev.chebfit(z, wfp.local_weights(a + (b - a) * (z + 1) / 2, P, win), deg)
        fit = np.polynomial.chebyshev.chebval(zt, coef).T
        exact = wfp.local_weights(a + (b - a) * (zt + 1) / 2, P, win)
        worst = max(worst, float(np.max(np.abs(fit - exact))) / scale)
    assert worst < bar, worst


def test_fits_across_breakpoints_can_fail():
    """The breakpoints are real, though not all of them matter: one polynomial over two neighbouring
    intervals holds across some breakpoints (to rounding) and misses by orders of magnitude more than
    the per-interval fits across others."""
    P = wfp.params(1e-3, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    bps = _breakpoints(P)
    scale = np.max(np.abs(wfp.local_weights(np.linspace(0.0, 0.999 * P.delta, 400), P, win)))
    z = np.cos(np.pi * (np.arange(8) + 0.5) / 8)
    zt = np.linspace(-0.97, 0.97, 41)
    errs = []
    for i in range(1, len(bps) - 1, 20):
        a, b = bps[i - 1], bps[i + 1]
        coef = np.polynomial.chebyshev.chebfit(z, wfp.local_weights(a + (b - a) * (z + 1) / 2, P, win), 7)
        fit = np.polynomial.chebyshev.chebval(zt, coef).T
        errs.append(float(np.max(np.abs(fit - wfp.local_weights(a + (b - a) * (zt + 1) / 2, P, win)))) / scale)
    assert max(errs) > 1e-8 and min(errs) < 1e-12, (min(errs), max(errs))
