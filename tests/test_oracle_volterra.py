"""Pins for Oracle A (direct Volterra march) against what the paper and mathematics fix."""
import math

import numpy as np
import pytest

import closed_forms as cf
from oracle import volterra


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_single_spring_closed_form_converges(p):
    """eq. IEfree with M = 1 has the erf closed form; the march converges at order >= p."""
    beta, x1, x0, w = 6.0, 0.3, -1.2, 0.1
    sig_ex, u_ex = cf.single_spring_free(beta, x1, 1.0, x0, w)
    errs = []
    for dt in (0.01, 0.005):
        Nt = int(round(5.0 / dt))
        s, u = volterra.march([x1], [beta], False, dt, Nt, p, [1.0], [x0], [w], None, [1.0, -0.5])
        t = np.arange(Nt + 1) * dt
        errs.append(_rel(s[:, 0], sig_ex(t)))
        # the field at receivers on both sides of the spring, eq. singleLayerSol
        eu = max(_rel(u[:, 0], u_ex(1.0, t)), _rel(u[:, 1], u_ex(-0.5, t)))
        assert eu < 50 * errs[-1] + 1e-12
    order = math.log2(errs[0] / errs[1])
    assert order > p - 0.3, (errs, order)
    if p == 8:
        assert errs[1] < 5e-12


def test_reflection_transmission_energy():
    """|R|^2 + |T|^2 = 1 for the time-harmonic spring (from eqs. WE-kink)."""
    for beta in (0.1, 1.0, 10.0, 100.0):
        for om in (0.3, 1.0, 7.0):
            R, T = cf.reflection_transmission(beta, om)
            assert abs(abs(R) ** 2 + abs(T) ** 2 - 1.0) < 1e-14
            assert abs(1 + R - T) < 1e-14       # continuity at the spring


def test_single_spring_spectrum_matches_reflection_coefficient():
    """The scattered field's spectrum upstream equals R(omega) times the incident spectrum."""
    beta, x1, x0, w = 4.0, 0.0, -1.0, 0.15
    dt, Nt = 0.005, 2400
    xr = -0.5
    s, u = volterra.march([x1], [beta], False, dt, Nt, 8, [1.0], [x0], [w], None, [xr])
    t = np.arange(Nt + 1) * dt
    # reflected wave at xr travels left: u(xr, t) = R * f(2 x1 - xr - t) in the frequency domain
    inc = np.exp(-0.5 * ((2 * x1 - xr - t - x0) / w) ** 2)
    om = np.array([1.0, 3.0, 6.0])
    U = np.array([np.sum(u[:, 0] * np.exp(1j * o * t)) * dt for o in om])
    F = np.array([np.sum(inc * np.exp(1j * o * t)) * dt for o in om])
    R, _ = cf.reflection_transmission(beta, om)
    assert np.max(np.abs(U / F - R)) < 1e-8


def test_zero_stiffness_is_inert():
    """beta = 0 gives g = 0 and sigma = 0, u = 0 exactly; an inert spring changes nothing."""
    x = np.array([-0.7, 0.1, 0.1003, 1.2])
    beta = np.array([3.0, 0.0, 5.0, 2.0])
    s0, u0 = volterra.march(x, np.zeros(4), True, 0.01, 200, 8, [1.0], [-2.0], [0.1], None, [0.0])
    assert np.all(s0 == 0.0) and np.all(u0 == 0.0)
    s1, u1 = volterra.march(x, beta, True, 0.01, 300, 8, [1.0], [-2.0], [0.1], None, [0.5, 2.0])
    keep = beta != 0
    s2, u2 = volterra.march(x[keep], beta[keep], True, 0.01, 300, 8, [1.0], [-2.0], [0.1], None,
                            [0.5, 2.0])
    assert np.all(s1[:, ~keep] == 0.0)
    assert _rel(s1[:, keep], s2) < 1e-13
    assert _rel(u1, u2) < 1e-13


@pytest.mark.parametrize("p", [1, 2])
def test_one_spring_difference_equations(p):
    """Sec. 5.1 difference equations for M = 1, to rounding."""
    beta, dt, Nt = 7.0, 0.02, 400
    x1, x0, w = 0.2, -1.0, 0.12
    t = np.arange(Nt + 1) * dt
    g = beta * np.exp(-0.5 * ((x1 - t - x0) / w) ** 2)
    g[0] = 0.0
    s, _ = volterra.march([x1], [beta], False, dt, Nt, p, [1.0], [x0], [w], None, [])
    ref = cf.recursion_M1(beta, dt, g, p)
    assert _rel(s[:, 0], ref) < 1e-12


@pytest.mark.parametrize("p,L", [(1, 0.013), (1, 0.137), (2, 0.0061), (2, 0.0537), (2, 0.21)])
def test_two_spring_discrete_equations(p, L):
    """eqs. dvie2 (p=1), dvie3 (p=2, L<dt) and dvie4 (p=2, L>dt), to rounding."""
    beta, dt, Nt = 5.0, 0.01, 300
    x = np.array([0.0, L])
    x0, w = -1.0, 0.1
    t = np.arange(Nt + 1) * dt
    g = beta * np.exp(-0.5 * ((x[:, None] - t[None, :] - x0) / w) ** 2)
    g[:, 0] = 0.0
    s, _ = volterra.march(x, [beta, beta], False, dt, Nt, p, [1.0], [x0], [w], None, [])
    r1, r2 = cf.recursion_M2(beta, dt, L, g[0], g[1], p)
    assert _rel(s[:, 0], r1) < 1e-11
    assert _rel(s[:, 1], r2) < 1e-11


def test_two_spring_stability_bound():
    """Theorem stability1: p = 2, L < dt, L beta < 2 gives ||sigma|| <= ||g|| / (1 - L beta / 2)."""
    beta, dt, L, Nt = 12.0, 0.1, 0.09, 400
    x = np.array([0.0, L])
    t = np.arange(Nt + 1) * dt
    g = np.stack([np.sin(3 * t) * np.exp(-0.01 * t), np.cos(2 * t) * (t > 0)])
    g[:, 0] = 0.0
    s, _ = volterra.march(x, [beta, beta], False, dt, Nt, 2, [], [], [], g.T.copy(), [])
    assert np.linalg.norm(s) <= np.linalg.norm(g) / (1 - L * beta / 2)


def test_single_spring_stiffness_limit_of_high_order_stencils():
    """The p-point stencil of the newest interval uses the p nearest available samples, i.e. the
    newest sample and p - 1 older ones (Sec. 4.1), so a single spring behaves like an implicit
    Adams method for sigma' = -(beta/2) sigma: p = 2 is unconditionally stable (Sec. 5), high p
    has a bounded interval.  Observed for p = 8: stable at beta dt / 2 = 0.25, growth by many
    orders at 0.5 (where the paper runs its beta = 100, dt = 0.01 array examples); p = 6 is
    still stable at 0.5.  A change of the stencil rule moves these."""
    dt, Nt = 0.01, 1500
    w = 1.0 / math.sqrt(10.0)

    def peak(beta, p):
        _, u = volterra.march([-0.5], [beta], False, dt, Nt, p, [1.0], [-3.0], [w], None, [1.8])
        return float(np.nanmax(np.abs(u)))

    assert peak(50.0, 8) < 1.5
    assert peak(100.0, 8) > 1e6
    assert peak(100.0, 6) < 1.5
    assert peak(100.0, 2) < 1.5


def test_manufactured_solution_order():
    """Sec. 6.1 manufactured solution: error O(dt^{p+1})-ish down to rounding."""
    rng = np.random.default_rng(11)
    M = 6
    x = np.sort(rng.uniform(-1, 1, M))
    beta = rng.uniform(0.1, 3, M)
    mu = rng.uniform(40, 50, M)
    t0 = rng.uniform(1, 3, M)
    sig_ex, u_ex, g_ex = cf.mms(x, beta, mu, t0)
    errs = []
    for dt in (0.04, 0.02):
        Nt = int(round(5.0 / dt))
        t = np.arange(Nt + 1) * dt
        g = g_ex(t)
        s, u = volterra.march(x, beta, False, dt, Nt, 4, [], [], [], g, [0.25])
        errs.append(_rel(s, sig_ex(t)))
        assert _rel(u[:, 0], u_ex(0.25 * np.ones_like(t), t)) < 20 * errs[-1]
    assert math.log2(errs[0] / errs[1]) > 3.7


def test_periodic_equals_replicated_free_space():
    """Periodic images: the periodic march equals a free-space march over the springs and
    their 2 pi translates (driven by the periodised pulse) up to the light-cone horizon."""
    x = np.array([-0.8, 0.35, 1.9])
    beta = np.array([2.0, 6.0, 4.0])
    dt, Nt, p = 0.02, 250, 6        # T = 5 < 4 pi - 2 pi: central copies see every image
    amp, cen, wid = [1.0], [-2.4], [0.15]
    sp, up = volterra.march(x, beta, True, dt, Nt, p, amp, cen, wid, None, [0.0])
    reps = [-2, -1, 0, 1, 2]
    xf = np.concatenate([x + 2 * math.pi * m for m in reps])
    bf = np.concatenate([beta for _ in reps])
    t = np.arange(Nt + 1) * dt
    g = bf[None, :] * cf.periodised_pulse(xf[None, :] - t[:, None], amp, cen, wid)
    g[0] = 0.0
    sf, uf = volterra.march(xf, bf, False, dt, Nt, p, [], [], [], g, [0.0])
    centre = slice(2 * 3, 3 * 3)
    assert _rel(sp, sf[:, centre]) < 1e-12
    assert _rel(up, uf) < 1e-12


def test_self_convergence_periodic():
    """Order p+1-ish self-convergence on a small periodic problem (Sec. 6.1 / Sec. 6.3 practice)."""
    x = np.array([-1.3, -0.2, 0.05, 1.1, 2.5])
    beta = np.array([3.0, 8.0, 1.5, 6.0, 9.0])
    amp, cen, wid = [1.0], [-2.2], [0.2]
    p = 4
    sols = []
    for dt in (0.04, 0.02, 0.01):
        Nt = int(round(4.0 / dt))
        s, _ = volterra.march(x, beta, True, dt, Nt, p, amp, cen, wid, None, [])
        sols.append(s[:: int(round(0.04 / dt))])
    e1 = _rel(sols[0], sols[2])
    e2 = _rel(sols[1], sols[2])
    assert math.log2(e1 / e2) > p - 0.5
