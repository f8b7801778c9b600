"""Closed forms and the paper's discrete recursions, written out for the oracle pins.

Nothing here is shared with the oracle or the CUDA library: these are independent
formulas from the paper or derived by hand from its equations.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def gaussian_pulse(s, amp, center, width):
    s = np.asarray(s, dtype=np.float64)
    f = np.zeros_like(s)
    for a, c, w in zip(amp, center, width):
        f = f + a * np.exp(-0.5 * ((s - c) / w) ** 2)
    return f


def periodised_pulse(s, amp, center, width, images=12):
    s = np.asarray(s, dtype=np.float64)
    f = np.zeros_like(s)
    for m in range(-images, images + 1):
        f = f + gaussian_pulse(s + 2 * math.pi * m, amp, center, width)
    return f


def single_spring_free(beta, x1, amp, x0, w):
    """Exact single-spring solution in free space (eq. IEfree with M = 1).

    With Sigma(t) = int_0^t sigma and g(t) = beta f(x1 - t), eq. IEfree reads
    Sigma' + (beta/2) Sigma = -beta f(x1 - t), Sigma(0) = 0.  For the Gaussian
    f(s) = amp exp(-(s - x0)^2 / (2 w^2)), with c = x1 - x0, a = beta/2, mu = c + a w^2:

        Sigma(t) = -beta amp w sqrt(pi/2) exp(-a t + a c + a^2 w^2 / 2)
                   * [erf((t - mu)/(sqrt2 w)) + erf(mu/(sqrt2 w))].

    Returns (sigma(t), u(x, t)) callables; sigma = Sigma' and u = Sigma(t - |x - x1|)/2
    (eq. singleLayerSol).
    """
    a = 0.5 * beta
    c = x1 - x0
    mu = c + a * w * w
    r2w = math.sqrt(2.0) * w

    def Sigma(t):
        t = np.asarray(t, dtype=np.float64)
        A = (t - mu) / r2w
        B = mu / r2w
        # erf(A) + erf(B) = erfc(-A) - erfc(B), accurate when A is very negative
        s = special.erfc(-A) - special.erfc(B)
        val = -beta * amp * w * math.sqrt(math.pi / 2) * np.exp(-a * t + a * c + a * a * w * w / 2) * s
        return np.where(t > 0, val, 0.0)

    def sigma(t):
        t = np.asarray(t, dtype=np.float64)
        f = amp * np.exp(-0.5 * ((x1 - t - x0) / w) ** 2)
        return np.where(t > 0, -a * Sigma(t) - beta * f, 0.0)

    def u(x, t):
        return 0.5 * Sigma(np.asarray(t) - abs(x - x1))

    return sigma, u


def reflection_transmission(beta, omega):
    """Time-harmonic single spring: R = beta/(2 i omega - beta), T = 2 i omega/(2 i omega - beta).

    Derived from eqs. WE-kink with u_inc = exp(i omega (x - t)) (e^{-i omega t} time
    convention); energy conservation gives |R|^2 + |T|^2 = 1.
    """
    den = 2j * omega - beta
    return beta / den, 2j * omega / den


def recursion_M1(beta, dt, g, p):
    """Sec. 5.1: one spring, p = 1 (explicit) or p = 2 (implicit) difference equations.

    p = 1:  sigma^{n+1} + (alpha - 1) sigma^n = -(g^{n+1} - g^n)
    p = 2:  (1 + alpha/2) sigma^{n+1} - (1 - alpha/2) sigma^n = -(g^{n+1} - g^n)
    with alpha = beta dt / 2 and sigma^0 = 0, g^0 = 0 (the sign follows eq. IEfree).
    """
    al = 0.5 * beta * dt
    sig = np.zeros_like(g)
    for n in range(len(g) - 1):
        dg = g[n + 1] - g[n]
        if p == 1:
            sig[n + 1] = -(al - 1.0) * sig[n] - dg
        else:
            sig[n + 1] = ((1.0 - al / 2) * sig[n] - dg) / (1.0 + al / 2)
    return sig


def recursion_M2(beta, dt, L, g1, g2, p):
    """Sec. 5.2-5.3: two springs a distance L apart, equal stiffness beta.

    p = 1 (eq. dvie2), kappa = L/dt, s = floor(kappa), at = (s + 1 - kappa) alpha:
      sigma_1^{n+1} + alpha sum_{nu<=n} sigma_1^nu + at sigma_2^{n-s}
                    + alpha sum_{nu<n-s} sigma_2^nu = -g_1^{n+1}
    p = 2, L < dt (eq. dvie3), xi1 = alpha (2 - kappa^2)/2, xi2 = alpha (1 - kappa)^2/2:
      (1 + alpha/2) sigma_1^{n+1} + alpha sum_{nu<=n} sigma_1^nu + alpha sum_{nu<n} sigma_2^nu
                    + xi1 sigma_2^n + xi2 sigma_2^{n+1} = -g_1^{n+1}
    p = 2, L > dt (eq. dvie4), xi1 = alpha/2 [(1-kappa+s)(1+kappa-s) + 1], xi2 = alpha/2 (1-kappa+s)^2:
      (1 + alpha/2) sigma_1^{n+1} + alpha sum_{nu<=n} sigma_1^nu + alpha sum_{nu<n-s} sigma_2^nu
                    + xi1 sigma_2^{n-s} + xi2 sigma_2^{n+1-s} = -g_1^{n+1}
    plus the 1 <-> 2 swapped equations.  Samples with index <= 0 are zero.
    """
    al = 0.5 * beta * dt
    kappa = L / dt
    s = int(math.floor(kappa))
    N = len(g1) - 1
    s1 = np.zeros(N + 1)
    s2 = np.zeros(N + 1)

    def v(arr, i):
        return arr[i] if i >= 1 else 0.0

    for n in range(N):
        if p == 1:
            at = (s + 1 - kappa) * al
            r1 = -g1[n + 1] - al * sum(s1[1:n + 1]) - at * v(s2, n - s) - al * sum(s2[1:max(n - s, 1)])
            r2 = -g2[n + 1] - al * sum(s2[1:n + 1]) - at * v(s1, n - s) - al * sum(s1[1:max(n - s, 1)])
            s1[n + 1], s2[n + 1] = r1, r2
        elif L < dt:
            xi1 = al * (2 - kappa ** 2) / 2
            xi2 = al * (1 - kappa) ** 2 / 2
            r1 = -g1[n + 1] - al * sum(s1[1:n + 1]) - al * sum(s2[1:max(n, 1)]) - xi1 * v(s2, n)
            r2 = -g2[n + 1] - al * sum(s2[1:n + 1]) - al * sum(s1[1:max(n, 1)]) - xi1 * v(s1, n)
            a = 1 + al / 2
            det = a * a - xi2 * xi2
            s1[n + 1] = (a * r1 - xi2 * r2) / det
            s2[n + 1] = (a * r2 - xi2 * r1) / det
        else:
            xi1 = al / 2 * ((1 - kappa + s) * (1 + kappa - s) + 1)
            xi2 = al / 2 * (1 - kappa + s) ** 2
            a = 1 + al / 2
            r1 = (-g1[n + 1] - al * sum(s1[1:n + 1]) - al * sum(s2[1:max(n - s, 1)])
                  - xi1 * v(s2, n - s) - xi2 * v(s2, n + 1 - s))
            r2 = (-g2[n + 1] - al * sum(s2[1:n + 1]) - al * sum(s1[1:max(n - s, 1)])
                  - xi1 * v(s1, n - s) - xi2 * v(s1, n + 1 - s))
            s1[n + 1], s2[n + 1] = r1 / a, r2 / a
    return s1, s2


def mms(x, beta, mu, t0):
    """Manufactured solution of Sec. 6.1: sigma_j(t) = exp(-mu_j (t - t0_j)^2).

    u_ex(x, t) = 1/2 sum_j int_0^{t - |x - x_j|} sigma_j
               = 1/2 sum_j sqrt(pi/(4 mu_j)) [erf(sqrt(mu_j)(t - |x - x_j| - t0_j)) + erf(sqrt(mu_j) t0_j)]
    for t > |x - x_j| (zero before), and g_j(t) = -sigma_j(t) - beta_j u_ex(x_j, t).
    """
    x = np.asarray(x, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    t0 = np.asarray(t0, dtype=np.float64)

    def sigma(t):
        t = np.asarray(t, dtype=np.float64)[..., None]
        return np.exp(-mu * (t - t0) ** 2)

    def u(xe, t):
        xe, t = np.broadcast_arrays(np.asarray(xe, dtype=np.float64), np.asarray(t, dtype=np.float64))
        tt = t[..., None] - np.abs(xe[..., None] - x)
        rm = np.sqrt(mu)
        val = 0.5 * np.sqrt(math.pi / (4 * mu)) * (special.erf(rm * (tt - t0)) + special.erf(rm * t0))
        return np.sum(np.where(tt > 0, val, 0.0), axis=-1)

    def g(t):
        t = np.asarray(t, dtype=np.float64)
        tt = np.broadcast_to(t[:, None], (t.shape[0], x.shape[0]))
        ux = u(np.broadcast_to(x, tt.shape), tt)
        return -sigma(t) - beta * ux

    return sigma, u, g
