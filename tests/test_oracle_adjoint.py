"""Pins for the adjoint oracle (oracle/adjoint.py): the gradient of the receiver misfit with
respect to the stiffnesses, from the reverse-time transposed march, against central finite
differences of the forward oracle, in the periodic box and in free space (with radiation
projections inside the window), and the gradient with respect to a host forcing against the
linearity of the forward march.  A second, independent pin: the complex-step derivative of the
direct march (oracle/volterra.c, complex build), a different discretisation of the same Volterra
system whose code shares nothing with the adjoint or the WFP oracle."""
import numpy as np
import pytest

from oracle import adjoint, volterra, wfp
from paper_2507_07823_gb300 import workloads as W


def _setup(bc, seed=5):
    rng = np.random.default_rng(seed)
    M = 8
    x = np.sort(rng.uniform(-0.8, 0.8, M))
    x[3] = x[2] + 0.013                       # one pair closer than dt: an implicit block
    beta = rng.uniform(1.0, 6.0, M)
    w = W.Workload(name="adjoint", bc=bc, x=x, beta=beta, amp=np.array([1.0]), center=np.array([-1.6]),
                   width=np.array([0.12]), dt=0.02, Nt=400, tol=1e-10, p=6,
                   xr=np.array([-0.95, 0.1, x[5], 0.95]), seed=seed)   # one receiver on a spring (m = 0 terms)
    # targets: the receivers of the same layout with perturbed stiffnesses
    w_true = w.with_(beta=beta * (1.0 + 0.1 * rng.standard_normal(M)))
    _, d = wfp.from_workload(w_true).run(w.Nt)
    return w, d


def _misfit(w, d):
    _, u = wfp.from_workload(w).run(w.Nt)
    return 0.5 * float(np.sum((u[1:] - d[1:]) ** 2))


@pytest.mark.parametrize("bc", [W.PERIODIC, W.FREE])
def test_gradient_matches_central_differences(bc):
    w, d = _setup(bc)
    o = wfp.from_workload(w)
    if bc == W.FREE:
        assert w.Nt >= o.P.rbc_period                  # projections happen inside the window
    L, grad = adjoint.misfit_and_gradient(o, w.Nt, d)
    assert abs(L - _misfit(w, d)) <= 1e-12 * L
    for j in (0, 2, 3, 7):
        h = 1e-5 * w.beta[j]
        bp, bm = w.beta.copy(), w.beta.copy()
        bp[j] += h
        bm[j] -= h
        fd = (_misfit(w.with_(beta=bp), d) - _misfit(w.with_(beta=bm), d)) / (2 * h)
        assert abs(grad[j] - fd) <= 1e-6 * np.max(np.abs(grad)), (j, grad[j], fd)


def test_forcing_gradient_is_the_transposed_march():
    """With a host forcing g the receivers are linear in g: u = A g.  For L = 1/2 |A g - d|^2,
    <grad_g L, delta> = <A g - d, A delta>; the reverse sweep's rhs adjoints give grad_g L = -rhsbar,
    checked through a directional derivative of the forward march."""
    w, d = _setup(W.FREE, seed=9)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((w.Nt + 1, w.M)) * 0.1
    delta = rng.standard_normal((w.Nt + 1, w.M))
    o = wfp.from_workload(w)
    L, _ = adjoint.misfit_and_gradient(o, w.Nt, d, g=g)
    # directional derivative by linearity: L(g + e delta) is quadratic in e
    def Lg(gg):
        _, u = wfp.from_workload(w).run(w.Nt, gg)
        return 0.5 * float(np.sum((u[1:] - d[1:]) ** 2))
    e = 1e-3
    dd = (Lg(g + e * delta) - Lg(g - e * delta)) / (2 * e)
    assert abs(L - Lg(g)) <= 1e-12 * L
    # the same directional derivative from the transposed march: sum_n <gbar^n, delta^n>
    gbar = adjoint.forcing_gradient(wfp.from_workload(w), w.Nt, d, g)
    assert abs(float(np.sum(gbar[1:] * delta[1:])) - dd) <= 1e-8 * abs(dd)


def _direct_misfit_complex_step(w, d, j, h):
    """L of the direct march with beta_j + i h: complex receivers, misfit without conjugation."""
    b = w.beta.astype(np.complex128)
    b[j] += 1j * h
    _, u = volterra.march_complex_step(w.x, b, w.bc == W.PERIODIC, w.dt, w.Nt, w.p, w.amp,
                                       w.center, w.width, None, w.xr)
    r = u[1:] - d[1:]
    return 0.5 * np.sum(r * r)


def test_complex_step_build_is_the_derivative_of_the_direct_march():
    """The complex build's real part is the real build bit for bit, and Im L / h equals the central
    difference of the real build (step 1e-5 beta_j: truncation about 1e-10 relative)."""
    w, _ = _setup(W.FREE)
    w = w.with_(Nt=200)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])

    def L_real(beta):
        _, u = volterra.march(w.x, beta, False, w.dt, w.Nt, w.p, w.amp, w.center, w.width, None,
                              w.xr)
        return 0.5 * float(np.sum((u[1:] - d[1:]) ** 2))

    _, u = volterra.march(w.x, w.beta, False, w.dt, w.Nt, w.p, w.amp, w.center, w.width, None,
                          w.xr)
    b = w.beta.astype(np.complex128)
    b[2] += 1e-20j
    _, uc = volterra.march_complex_step(w.x, b, False, w.dt, w.Nt, w.p, w.amp, w.center, w.width,
                                        None, w.xr)
    assert np.array_equal(uc.real, u) and np.any(uc.imag != 0.0)
    for j in (1, 3):
        Lc = _direct_misfit_complex_step(w, d, j, 1e-20 * w.beta[j])
        assert abs(Lc.real - L_real(w.beta)) <= 1e-14 * Lc.real
        hh = 1e-5 * w.beta[j]
        bp, bm = w.beta.copy(), w.beta.copy()
        bp[j] += hh
        bm[j] -= hh
        fd = (L_real(bp) - L_real(bm)) / (2 * hh)
        cs = Lc.imag / (1e-20 * w.beta[j])
        assert abs(cs - fd) <= 1e-7 * abs(cs), (j, cs, fd)


@pytest.mark.parametrize("bc", [W.PERIODIC, W.FREE])
def test_gradient_matches_complex_step_of_the_direct_march(bc):
    """dL/dbeta from the transposed WFP march against Im L(beta + i h e_j) / h of the direct march.
    The two forward schemes differ by their discretisation (the history of the WFP scheme goes
    through the Fourier modes' FIR quadrature, eq. alphakEvolutionFormulas); at p = 8 and
    dt = 0.01 on this layout their gradients agree to about 3e-8 of the largest component, while
    a dropped or halved term of the gradient formula, or P in place of P^T, moves it by > 8e-3."""
    w, _ = _setup(bc)
    w = w.with_(p=8, dt=0.01, Nt=800)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])       # targets that do not come from either oracle
    L, grad = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d)
    cs = np.array([_direct_misfit_complex_step(w, d, j, 1e-20 * w.beta[j]).imag
                   / (1e-20 * w.beta[j]) for j in range(w.M)])
    assert np.max(np.abs(grad - cs)) <= 2e-7 * np.max(np.abs(grad)), (grad, cs)
