"""Pins for Oracle B (the discrete WFP scheme) against mathematics fixed by the paper."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import closed_forms as cf
from oracle import volterra, wfp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------------------------------- parameters
def test_paper_parameter_values():
    """Sec. 3.1: eps = 1e-12, gamma = 1/2 gives W ~ 35 (2b/(pi gamma) = 35.18, ceil -> 36);
    K = pi/dt (eq. Kdt); m_max = W + ceil(p/2) (Sec. 4.1)."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        gold = json.load(f)
    P = wfp.params(0.01, 1e-12, 8)
    assert abs(2 * P.b / (math.pi * P.gamma) - gold["W_eps1e-12_gamma0.5"]["value"]) < 0.5
    assert P.W == 36 and P.K == 314 and P.m_max == 40 and P.NF == 629
    assert abs(P.delta - 0.36) < 1e-15


# ----------------------------------------------------------------------------- window
def test_window_normalisation_and_symmetry():
    """eq. KB at omega = 0: int_{-1}^{1} I0(b sqrt(1-t^2)) dt = 2 sinh(b)/b, hence phi(delta) = 1."""
    for eps, dt in ((1e-6, 0.01), (1e-10, 1e-3), (1e-12, 0.01), (1e-14, 5e-4)):
        P = wfp.params(dt, eps, 8)
        win = wfp.Window(P.delta, P.b)
        assert abs(win.phi_quadrature(np.array(P.delta)) - 1.0) < 2e-14
        t = np.linspace(0, P.delta, 101)
        assert np.max(np.abs(win.dphi(t) - win.dphi(P.delta - t))) < 1e-12 * np.max(win.dphi(t))
        assert np.max(np.abs(win.phi(t) + win.phi(P.delta - t) - 1.0)) < 5e-14
        assert np.all(np.diff(win.phi(t)) >= -1e-15)
        # jump of phi' at the ends is O(eps): b/(delta sinh b)
        assert win.dphi(np.array(0.0)) * P.delta < 3 * eps * P.b


def test_window_against_high_precision():
    """phi(t) = int_0^t phi' against a 40-digit mpmath quadrature."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    P = wfp.params(0.01, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    d, b = P.delta, P.b
    sc = mp.mpf(b) / (mp.mpf(d) * mp.sinh(b))

    def f(s):
        return sc * mp.besseli(0, b * mp.sqrt(max(0, 1 - (2 * s / d - 1) ** 2)))

    ts = np.array([0.013, 0.05, 0.11, 0.18, 0.2, 0.29, 0.35, 0.3599])
    ref = np.array([float(mp.quad(f, [0, t])) for t in ts])
    assert np.max(np.abs(win.phi(ts) - ref)) < 5e-14


def test_window_second_derivative_by_differences():
    P = wfp.params(0.01, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    t = np.linspace(0.01, 0.35, 35)
    hh = 1e-6
    fd = (win.dphi(t + hh) - win.dphi(t - hh)) / (2 * hh)
    assert np.max(np.abs(fd - win.ddphi(t))) < 1e-6 * np.max(np.abs(win.ddphi(t)))


# ----------------------------------------------------------------------------- history part
def test_history_recurrence_matches_direct_quadrature():
    """eq. alphakEvolutionFormulas + eq. hkcompdisc reproduce eq. alphak for a smooth S_k(tau)."""
    dt, eps = 0.01, 1e-12
    P = wfp.params(dt, eps, 8)
    win = wfp.Window(P.delta, P.b)
    pk, qk = wfp.pk_qk(P, win)
    rot = wfp.rotation(P)
    kk = np.arange(P.K + 1)

    def S(tau, k):
        return np.exp(-(tau - 1.0) ** 2 / 0.02) * np.cos(0.3 * k * tau) + 0.5j * np.exp(-(tau - 1.2) ** 2 / 0.05)

    alpha = np.zeros(P.K + 1, complex)
    ap = np.zeros(P.K + 1, complex)
    ring = np.zeros((P.W, P.K + 1), complex)
    hist = []
    for n in range(250):
        ring = np.roll(ring, 1, axis=0)
        ring[0] = S(n * dt, kk)
        h, g = wfp.fir(pk, qk, ring, dt)
        alpha, ap = wfp.mode_update(alpha, ap, h, g, rot)
        hist.append(alpha.copy())
    hist = np.array(hist)
    scale = np.max(np.abs(hist))
    for k in (0, 1, 5, 40, 150, 314):
        for n1 in (100, 160, 250):
            t = n1 * dt

            def f(tau, part):
                kern = math.sin(k * (t - tau)) / k if k else (t - tau)
                v = kern * S(tau, k) * float(win.phi(t - tau))
                return v.real if part == 0 else v.imag

            ex = complex(integrate.quad(f, 0, t, args=(0,), limit=400, epsabs=1e-15, points=[t - P.delta])[0],
                         integrate.quad(f, 0, t, args=(1,), limit=400, epsabs=1e-15, points=[t - P.delta])[0])
            assert abs(ex - hist[n1 - 1, k]) < 1e-10 * scale, (k, n1)


def test_pk_qk_vanish_at_window_ends_and_converge_in_Ng():
    """p_k, q_k (eq. pkqkcomp) vanish beyond [-dt, delta]; the Ng-node rule is converged."""
    P = wfp.params(0.01, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    pk32, qk32 = wfp.pk_qk(P, win)
    P64 = wfp.params(0.01, 1e-12, 8, Ng=64)
    pk64, qk64 = wfp.pk_qk(P64, win)
    assert np.max(np.abs(pk32 - pk64)) < 1e-15 * np.max(np.abs(pk64)) * 10
    assert np.max(np.abs(qk32 - qk64)) < 1e-15 * np.max(np.abs(qk64)) * 10
    # Psi_k vanishes outside [0, delta]
    assert np.all(wfp.psi_k(np.arange(5.0)[:, None], np.array([-1e-3, P.delta + 1e-9]), win) == 0.0)


# ----------------------------------------------------------------------------- local part
@pytest.mark.parametrize("deg", [0, 3, 7])
def test_local_weights_exact_on_polynomials(deg):
    """Sec. 4.1: the p-point interpolant reproduces degree < p polynomials, so
    sum_m Q_m(d) sigma(t_{n+1-m}) = int_d^delta (1 - phi(s)) sigma(t_{n+1} - s) ds."""
    P = wfp.params(0.01, 1e-12, 8)
    win = wfp.Window(P.delta, P.b)
    d = np.array([0.0, 0.003, 0.0099, 0.01, 0.0137, 0.05, 0.2, 0.3555, 0.36, 0.5])
    Q = wfp.local_weights(d, P, win)
    m = np.arange(P.m_max + 1)

    def poly(s):
        return (1 + s / 0.1) ** deg

    for i, dd in enumerate(d):
        if dd >= P.delta:
            assert np.all(Q[i] == 0.0)
            continue
        ex = integrate.quad(lambda s: (1 - float(win.phi(s))) * poly(s), dd, P.delta,
                            epsabs=1e-16, epsrel=1e-14, limit=200)[0]
        assert abs(np.sum(Q[i] * poly(m * P.dt)) - ex) < 1e-13 * max(1.0, abs(ex))
        if dd >= P.dt:
            assert Q[i, 0] == 0.0           # intermediate sources use only known samples


def test_local_weights_use_window_of_width_delta():
    """sum_m Q_m(0) = int_0^delta (1 - phi) = delta/2 (phi(t) + phi(delta - t) = 1)."""
    for dt in (0.01, 1e-3):
        P = wfp.params(dt, 1e-12, 8)
        win = wfp.Window(P.delta, P.b)
        Q = wfp.local_weights(np.array([0.0]), P, win)
        assert abs(Q.sum() - P.delta / 2) < 1e-15 * 50


# ----------------------------------------------------------------------------- Fourier sums
def test_type1_type2_on_uniform_points_reduce_to_fft():
    """On x_j = -pi + 2 pi j / N the sums of eqs. densco / historySol1 are FFTs."""
    N, K = 64, 20
    rng = np.random.default_rng(3)
    x = -math.pi + 2 * math.pi * np.arange(N) / N
    sigma = rng.standard_normal(N)
    S = wfp.type1(sigma, x, K)
    F = np.fft.ifft(sigma) * N                      # sum_j sigma_j e^{+2 pi i k j / N}
    ref = F[:K + 1] * np.exp(-1j * math.pi * np.arange(K + 1)) / (2 * math.pi)
    assert np.max(np.abs(S - ref)) < 1e-13
    alpha = rng.standard_normal(K + 1) + 1j * rng.standard_normal(K + 1)
    alpha[0] = alpha[0].real
    u = wfp.type2(alpha, x)
    full = np.zeros(N, complex)
    full[:K + 1] = alpha
    full[N - np.arange(1, K + 1)] = np.conj(alpha[1:])
    ref_u = np.real(np.fft.fft(full * np.exp(1j * math.pi * np.fft.fftfreq(N, 1.0 / N))))
    assert np.max(np.abs(u - ref_u)) < 1e-12


# ----------------------------------------------------------------------------- RBC
def test_rbc_projection_leaves_interior_unchanged():
    """Sec. 4.4: the projected coefficients represent the same field in |x| < pi - 2 delta."""
    P = wfp.params(0.01, 1e-12, 8)
    swin = wfp.Window(P.delta_s, P.b)
    rng = np.random.default_rng(5)
    k = np.arange(P.K + 1)
    # a smooth field with content well inside the band, spread over the whole box
    alpha = (rng.standard_normal(P.K + 1) + 1j * rng.standard_normal(P.K + 1)) * np.exp(-(k / 60.0) ** 2)
    alpha[0] = alpha[0].real
    ap = 1j * k * alpha
    a2, ap2 = wfp.rbc_project(alpha, ap, P, swin)
    xi = np.linspace(-math.pi + 2 * P.delta_s + 0.01, math.pi - 2 * P.delta_s - 0.01, 301)
    assert np.max(np.abs(wfp.type2(a2, xi) - wfp.type2(alpha, xi))) < 1e-10 * np.max(np.abs(wfp.type2(alpha, xi)))
    xo = np.linspace(math.pi - P.delta_s + 0.02, math.pi, 20)
    assert np.max(np.abs(wfp.type2(a2, xo))) < 1e-9 * np.max(np.abs(wfp.type2(alpha, xi)))
    assert a2[-1] == 0.0 and ap2[-1] == 0.0


# ----------------------------------------------------------------------------- whole march
def test_periodic_march_matches_direct_volterra():
    """The WFP march converges to the same solution as the direct all-to-all march."""
    x = np.array([-0.5, 0.1, 0.35, 1.1, 2.0])
    beta = np.array([3.0, 8.0, 1.5, 6.0, 9.0])
    amp, cen, wid = [1.0], [-2.2], [0.15]
    dt, Nt = 0.01, 500
    sA, uA = volterra.march(x, beta, True, dt, Nt, 8, amp, cen, wid, None, [0.3, -2.0])
    o = wfp.WFP(x, beta, True, dt, 1e-12, 8, amp, cen, wid, [0.3, -2.0])
    sB, uB = o.run(Nt)
    assert _rel(sB, sA) < 3e-10
    assert _rel(uB, uA) < 3e-10


def test_planted_half_history_factor_is_caught():
    """The printed beta_j/2 in front of the history sum would not reproduce eq. periodicIE."""
    x = np.array([-0.5, 0.1, 0.35, 1.1, 2.0])
    beta = np.array([3.0, 8.0, 1.5, 6.0, 9.0])
    amp, cen, wid = [1.0], [-2.2], [0.15]
    dt, Nt = 0.01, 400
    sA, _ = volterra.march(x, beta, True, dt, Nt, 8, amp, cen, wid, None, [])
    o = wfp.WFP(x, beta, True, dt, 1e-12, 8, amp, cen, wid, [])
    real_t2 = o._type2_springs
    o._type2_springs = lambda a: 0.5 * real_t2(a)      # the mistake, planted in the oracle
    sB, _ = o.run(Nt)
    assert _rel(sB, sA) > 1e-3


def test_free_space_march_matches_direct_volterra():
    """Free space (Sec. 4.4 RBC every ceil(1.5 W) steps) against the direct free-space march."""
    x = np.array([-1.5, -0.5, 0.1, 0.35, 1.1, 1.9])
    beta = np.array([3.0, 8.0, 1.5, 6.0, 9.0, 2.0])
    amp, cen, wid = [1.0, 0.5], [-3.0, -3.4], [0.12, 0.2]
    dt, Nt = 0.01, 1200
    xr = [0.3, -1.9, 2.0]
    sA, uA = volterra.march(x, beta, False, dt, Nt, 8, amp, cen, wid, None, xr)
    o = wfp.WFP(x, beta, False, dt, 1e-12, 8, amp, cen, wid, xr)
    sB, uB = o.run(Nt)
    assert _rel(sB, sA) < 5e-10
    assert _rel(uB, uA) < 5e-10
    o2 = wfp.WFP(x, beta, False, dt, 1e-12, 8, amp, cen, wid, xr, rbc_period=10 ** 9)
    sC, _ = o2.run(Nt)
    assert _rel(sC, sA) > 1e-2          # without the projection waves wrap around the box


def test_free_space_single_spring_closed_form():
    beta, x1, x0, w = 6.0, 0.3, -3.0, 0.1
    sig_ex, u_ex = cf.single_spring_free(beta, x1, 1.0, x0, w)
    dt, Nt = 0.005, 2000
    o = wfp.WFP([x1], [beta], False, dt, 1e-12, 8, [1.0], [x0], [w], [1.0, -0.5])
    s, u = o.run(Nt)
    t = np.arange(Nt + 1) * dt
    assert _rel(s[:, 0], sig_ex(t)) < 1e-10
    assert _rel(u[:, 0], u_ex(1.0, t)) < 1e-10
    assert _rel(u[:, 1], u_ex(-0.5, t)) < 1e-10


def test_zero_stiffness_gives_zero():
    o = wfp.WFP([-0.3, 0.4, 0.40001], [0.0, 0.0, 0.0], True, 0.01, 1e-10, 8, [1.0], [-2.0], [0.1], [0.0])
    s, u = o.run(200)
    assert np.all(s == 0.0) and np.all(u == 0.0)


def test_self_convergence_order():
    x = np.array([-0.5, 0.1, 0.35, 1.1, 2.0])
    beta = np.array([3.0, 8.0, 1.5, 6.0, 9.0])
    amp, cen, wid = [1.0], [-2.2], [0.15]
    sols = []
    for dt in (0.04, 0.02, 0.01):
        o = wfp.WFP(x, beta, True, dt, 1e-13, 4, amp, cen, wid, [])
        s, _ = o.run(int(round(3.0 / dt)))
        sols.append(s[:: int(round(0.04 / dt))])
    e1, e2 = _rel(sols[0], sols[2]), _rel(sols[1], sols[2])
    assert math.log2(e1 / e2) > 3.5
