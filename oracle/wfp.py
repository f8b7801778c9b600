"""Oracle B: the discrete windowed Fourier projection (WFP) scheme, step by step.

TEST INFRASTRUCTURE ONLY — see the package docstring.  Plain numpy / scipy in FP64;
library primitives (matrix products, sparse LU, FFT, special functions, Gauss-Legendre
nodes) serve as steps.  Every function names the passage it follows.

One time step n -> n+1 (t_{n+1} = (n+1) dt), in the paper's order:

 1. S_k^n = (1/2pi) sum_j sigma_j^n e^{i k x_j}, |k| <= K                  (eq. densco, Sec. 3.1)
 2. h_k^n = dt sum_{m=0}^{W-1} p_k(m dt) S_k^{n-m},  g_k^n likewise with q_k (eq. hkcompdisc)
 3. alpha_k^{n+1} = alpha_k^n cos(k dt) + alpha'_k^n sin(k dt)/k + h_k^n
    alpha'_k^{n+1} = -k alpha_k^n sin(k dt) + alpha'_k^n cos(k dt) + g_k^n (eq. alphakEvolutionFormulas)
 4. free space only, every `rbc_period` steps: (alpha, alpha') <- P (alpha, alpha')     (Sec. 4.4)
 5. u_H(x, t_{n+1}) = sum_k alpha_k^{n+1} e^{-i k x}                       (eq. historySol1)
 6. local explicit sum and the implicit solve                              (eqs. periodicIE_disc,
    -(I + S) sigma^{n+1} = g^{n+1} + sum_m C^(m) sigma^{n+1-m} + E alpha^{n+1}      linearSystem)
 7. receivers: u = u_L + u_H with sigma^{n+1} known                       (eq. localSol2)

Readings where the paper is silent or inconsistent:
 * K = floor(pi/dt) (eq. Kdt assumes pi/dt is an integer); W = ceil(2b/(pi gamma)), b = ln 1/eps.
 * The history term of eqs. periodicIE_AS / periodicIE_disc and E_jk is printed with beta_j/2; the
   representation u = u_L + u_H with eq. periodicIE fixes it as beta_j, which is used here.
 * Only k = 0..K are stored: sigma is real, so S_{-k} = conj S_k and alpha_{-k} = conj alpha_k.
 * The RBC step keeps the field real: modes |k| = K are dropped before the 2K-point transform and
   set to zero afterwards; the spatial window has width delta_s = W h with h = pi/K.
 * FIR range m = 0..W-1 (eq. hkcompdisc).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C
from numpy.polynomial import legendre
from scipy import special

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------------------------
# parameters (eqs. b, Kdt, W and Remark r:gamma; Sec. 4.1 for m_max)
# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    dt: float
    eps: float
    gamma: float
    p: int
    b: float
    K: int
    W: int
    delta: float
    m_max: int
    NL: int
    Ng: int
    rbc_period: int
    h: float            # RBC grid spacing 2 pi / (2K)
    delta_s: float      # spatial window width W h

    @property
    def NF(self):
        return 2 * self.K + 1


def params(dt, eps, p, gamma=0.5, W=None, NL=None, Ng=32, rbc_period=None) -> Params:
    b = math.log(1.0 / eps)
    K = int(math.floor(math.pi / dt))
    if W is None:
        W = int(math.ceil(2.0 * b / (math.pi * gamma)))
    delta = W * dt
    m_max = W + int(math.ceil(p / 2))
    if NL is None:
        NL = W
    h = math.pi / K
    if rbc_period is None:
        rbc_period = int(math.ceil(1.5 * W))
    return Params(dt=dt, eps=eps, gamma=gamma, p=p, b=b, K=K, W=W, delta=delta, m_max=m_max,
                  NL=NL, Ng=Ng, rbc_period=rbc_period, h=h, delta_s=W * h)


# ---------------------------------------------------------------------------------------------
# blending window (eq. phi): phi' is a scaled Kaiser-Bessel bump on [0, delta], phi = int_0^t phi'
# ---------------------------------------------------------------------------------------------
class Window:
    """phi, phi', phi'' of eq. phi for width delta and shape parameter b.

    phi' is symmetric about delta/2, so phi(t) = 1 - phi(delta - t).  phi on [0, delta/2] is a
    Chebyshev interpolant (degree 48) of the Gauss-Legendre integral of phi'; it agrees with a
    40-digit quadrature to about 1e-14 (pinned in tests).
    """
    N_PHI_GL = 96      # Gauss-Legendre nodes for phi(t) = int_0^t phi'
    CHEB_DEG = 48      # Chebyshev degree of phi on [0, delta/2]

    def __init__(self, delta, b):
        self.delta = float(delta)
        self.b = float(b)
        self.scale = self.b / (self.delta * math.sinh(self.b))
        self._gx, self._gw = legendre.leggauss(self.N_PHI_GL)
        self._cheb = C.chebinterpolate(
            lambda z: self.phi_quadrature(0.25 * self.delta * (z + 1.0)), self.CHEB_DEG)

    def dphi(self, t):
        """phi'(t) = b/(delta sinh b) I0(b sqrt(1 - (2t/delta - 1)^2)) on [0, delta], else 0."""
        t = np.asarray(t, dtype=np.float64)
        u = 2.0 * t / self.delta - 1.0
        inside = (t >= 0.0) & (t <= self.delta)
        z = self.b * np.sqrt(np.clip(1.0 - u * u, 0.0, None))
        return np.where(inside, self.scale * special.i0(z), 0.0)

    def ddphi(self, t):
        """phi''(t) = -(2 b^3 u / (delta^2 sinh b)) I1(z)/z with z = b sqrt(1 - u^2), u = 2t/delta - 1."""
        t = np.asarray(t, dtype=np.float64)
        u = 2.0 * t / self.delta - 1.0
        inside = (t >= 0.0) & (t <= self.delta)
        z = self.b * np.sqrt(np.clip(1.0 - u * u, 0.0, None))
        i1_over_z = np.where(z > 1e-8, special.i1(z) / np.where(z > 1e-8, z, 1.0), 0.5)
        val = -(2.0 * self.b ** 3 * u / (self.delta * self.delta * math.sinh(self.b))) * i1_over_z
        return np.where(inside, val, 0.0)

    def phi_quadrature(self, t):
        """phi(t) = int_0^t phi' by a Gauss-Legendre rule on [0, t] (phi' is entire in t)."""
        t = np.clip(np.asarray(t, dtype=np.float64), 0.0, self.delta)
        nodes = 0.5 * t[..., None] * (1.0 + self._gx)
        return 0.5 * t * np.sum(self._gw * self.dphi(nodes), axis=-1)

    def phi(self, t):
        """phi(t): 0 for t <= 0, 1 for t >= delta; Chebyshev on [0, delta/2], reflected above."""
        t = np.asarray(t, dtype=np.float64)
        tc = np.clip(t, 0.0, self.delta)
        low = tc <= 0.5 * self.delta
        tl = np.where(low, tc, self.delta - tc)
        v = C.chebval(4.0 * tl / self.delta - 1.0, self._cheb)
        v = np.where(low, v, 1.0 - v)
        return np.where(t <= 0.0, 0.0, np.where(t >= self.delta, 1.0, v))


# ---------------------------------------------------------------------------------------------
# history kernels (eqs. psidef, pkqkcomp) and rotation (eq. alphakEvolutionFormulas)
# ---------------------------------------------------------------------------------------------
def sin_over_k(k, t):
    """sin(k t)/k with the k = 0 limit t (Remark r:kzero)."""
    k = np.asarray(k, dtype=np.float64)
    safe = np.where(k == 0, 1.0, k)
    return np.where(k == 0, t, np.sin(k * t) / safe)


def psi_k(k, tau, win: Window):
    """Psi_k(tau) = 2 cos(k tau) phi'(tau) + sin(k tau)/k phi''(tau), support [0, delta]."""
    return 2.0 * np.cos(k * tau) * win.dphi(tau) + sin_over_k(k, tau) * win.ddphi(tau)


def pk_qk(P: Params, win: Window):
    """p_k(m dt), q_k(m dt) for m = 0..W-1, k = 0..K by an Ng-node Gauss-Legendre rule:

    p_k(m dt) = int_0^dt sin(k(dt - mu))/k Psi_k(m dt + mu) dmu,
    q_k(m dt) = int_0^dt cos(k(dt - mu))   Psi_k(m dt + mu) dmu.
    Returns two arrays of shape (W, K+1).
    """
    gx, gw = legendre.leggauss(P.Ng)
    mu = 0.5 * P.dt * (1.0 + gx)                   # (Ng,)
    wt = 0.5 * P.dt * gw
    k = np.arange(P.K + 1, dtype=np.float64)[None, :, None]        # (1, K+1, 1)
    m = np.arange(P.W, dtype=np.float64)[:, None, None]            # (W, 1, 1)
    tau = m * P.dt + mu[None, None, :]                             # (W, 1, Ng)
    ps = psi_k(k, tau, win)                                        # (W, K+1, Ng)
    pk = np.sum(wt * sin_over_k(k, P.dt - mu) * ps, axis=-1)
    qk = np.sum(wt * np.cos(k * (P.dt - mu)) * ps, axis=-1)
    return pk, qk


def rotation(P: Params):
    """cos(k dt), sin(k dt)/k, k sin(k dt) for k = 0..K."""
    k = np.arange(P.K + 1, dtype=np.float64)
    return np.cos(k * P.dt), sin_over_k(k, P.dt), k * np.sin(k * P.dt)


def fir(pk, qk, S_ring, dt):
    """eq. hkcompdisc: h_k = dt sum_m p_k(m dt) S_k^{n-m}; S_ring[m] holds S^{n-m}."""
    return dt * np.sum(pk * S_ring, axis=0), dt * np.sum(qk * S_ring, axis=0)


def mode_update(alpha, alpha_p, h, g, rot):
    """eq. alphakEvolutionFormulas."""
    c, s_over_k, k_s = rot
    return alpha * c + alpha_p * s_over_k + h, -alpha * k_s + alpha_p * c + g


# ---------------------------------------------------------------------------------------------
# Fourier sums (eqs. densco and historySol1), computed directly
# ---------------------------------------------------------------------------------------------
def type1(sigma, x, K, chunk=2048):
    """S_k = (1/2pi) sum_j sigma_j e^{i k x_j}, k = 0..K (direct sum)."""
    k = np.arange(K + 1, dtype=np.float64)
    S = np.zeros(K + 1, dtype=np.complex128)
    for j0 in range(0, len(x), chunk):
        xs = x[j0:j0 + chunk]
        S += np.exp(1j * xs[:, None] * k[None, :]).T @ sigma[j0:j0 + chunk]
    return S / TWO_PI


def type2(alpha, x, chunk=2048):
    """u_H(x) = sum_{|k|<=K} alpha_k e^{-i k x} = alpha_0 + 2 Re sum_{k>=1} alpha_k e^{-i k x}."""
    K = len(alpha) - 1
    k = np.arange(K + 1, dtype=np.float64)
    out = np.empty(len(x))
    wts = np.full(K + 1, 2.0)
    wts[0] = 1.0
    for j0 in range(0, len(x), chunk):
        xs = x[j0:j0 + chunk]
        out[j0:j0 + chunk] = np.real(np.exp(-1j * xs[:, None] * k[None, :]) @ (wts * alpha))
    return out


# ---------------------------------------------------------------------------------------------
# local part (Sec. 4.1): Q_m(d) by an N_L-node Gauss-Legendre rule on [t_{n+1}-delta, t_{n+1}-d]
# ---------------------------------------------------------------------------------------------
def distance(xa, xb, periodic):
    """dist of Definition lambdadef (nearest image) in the periodic box; |xa - xb| in free space."""
    d = np.abs(xa - xb)
    if periodic:
        d = np.mod(d, TWO_PI)
        d = np.minimum(d, TWO_PI - d)
    return d


def local_weights(d, P: Params, win: Window, chunk=100_000):
    """Q_m(d), m = 0..m_max, for an array of distances d (shape (npairs,)).

    Nodes s_i = t_{n+1} - xi_i run over [d, delta] (time before t_{n+1}); the interpolant at xi
    uses the p nearest grid times t_{n+1-m} with m_min <= m <= m_max, where m_min = 0 for nearby
    pairs (d < dt) and 1 otherwise; weights by the Lagrange formula.  Q_m = 0 for d >= delta.
    For each stencil offset r the node contributions w_i (1 - phi(s_i)) v_{lo+r}(s_i) are summed
    over the nodes with one bincount.
    """
    d = np.asarray(d, dtype=np.float64)
    npairs = d.shape[0]
    ncol = P.m_max + 1
    Q = np.zeros((npairs, ncol))
    gx, gw = legendre.leggauss(P.NL)
    for c0 in range(0, npairs, chunk):
        dc = d[c0:c0 + chunk]
        live = dc < P.delta
        dd = dc[live]
        if dd.size == 0:
            continue
        idx = np.nonzero(live)[0]
        s = dd[:, None] + 0.5 * (P.delta - dd)[:, None] * (1.0 + gx[None, :])   # (n, NL)
        w = 0.5 * (P.delta - dd)[:, None] * gw[None, :]
        one_minus_phi = 1.0 - win.phi(s)
        y = s / P.dt                                                          # time in steps
        m_min = np.where(dd < P.dt, 0, 1)[:, None]
        lo = np.floor(y).astype(np.int64) - P.p // 2 + 1
        lo = np.maximum(lo, m_min)
        lo = np.minimum(lo, P.m_max - P.p + 1)
        rowbase = (idx * ncol)[:, None]
        block = np.zeros(len(dc) * ncol)
        # Lagrange basis L_r(y) = prod_{q != r} (y - lo - q) / (r - q), via prefix/suffix products
        diff = [y - (lo + q) for q in range(P.p)]
        prefix = [np.ones_like(y)]
        for q in range(P.p - 1):
            prefix.append(prefix[-1] * diff[q])
        suffix = [np.ones_like(y)] * (P.p + 1)
        for q in range(P.p - 1, 0, -1):
            suffix[q] = suffix[q + 1] * diff[q]
        wphi = w * one_minus_phi
        for r in range(P.p):
            denom = float(np.prod([r - q for q in range(P.p) if q != r]))
            L = prefix[r] * suffix[r + 1] / denom
            val = wphi * L
            block += np.bincount((rowbase + lo + r).ravel(), weights=val.ravel(),
                                 minlength=len(dc) * ncol)
        Q[c0:c0 + chunk] = block.reshape(len(dc), ncol)
    return Q


def neighbour_pairs(xt, xs, radius, periodic):
    """All (target, source, distance) with distance <= radius (brute force, chunked)."""
    T, S_, D = [], [], []
    for t0 in range(0, len(xt), 1024):
        dd = distance(xt[t0:t0 + 1024, None], xs[None, :], periodic)
        ti, si = np.nonzero(dd <= radius)
        T.append(ti + t0)
        S_.append(si)
        D.append(dd[ti, si])
    return np.concatenate(T), np.concatenate(S_), np.concatenate(D)


# ---------------------------------------------------------------------------------------------
# free-space radiation condition P (Sec. 4.4)
# ---------------------------------------------------------------------------------------------
def rbc_project(alpha, alpha_p, P: Params, swin: Window):
    """Roll the field off to zero, outgoing, in |x| > pi - 2 delta_s (Sec. 4.4, eq. vtilde).

    Step 1: grid values u(x_i), v(x_i) on x_i = i h (i < K), (i - 2K) h (i >= K) of the real
            field with modes |k| <= K-1 (FFT of length n = 2K).
    Step 2: at i in {K-2W..K-1}: u~ = phi(pi - ds - x) u, v~ = phi'(pi - ds - x) u + phi(.) v;
            at i in {K..K+2W-1} the mirror image with phi(pi - ds + x).
    Step 3: inverse FFT; alpha_k for k = 0..K-1, alpha_K = 0.
    """
    K, W = P.K, P.W
    n = 2 * K

    def to_grid(a):
        full = np.zeros(n, dtype=np.complex128)
        full[:K] = a[:K]
        full[n - np.arange(1, K)] = np.conj(a[1:K])
        return np.real(np.fft.fft(full))

    u = to_grid(alpha)
    v = to_grid(alpha_p)
    i = np.arange(n)
    xg = np.where(i < K, i, i - n) * P.h
    right = np.arange(K - 2 * W, K)
    left = np.arange(K, K + 2 * W)
    for idx, sign in ((right, -1.0), (left, 1.0)):
        arg = math.pi - P.delta_s + sign * xg[idx]
        ph = swin.phi(arg)
        dph = swin.dphi(arg)
        uu, vv = u[idx].copy(), v[idx].copy()
        u[idx] = ph * uu
        v[idx] = dph * uu + ph * vv
    a_new = np.fft.ifft(u)[:K + 1].copy()
    ap_new = np.fft.ifft(v)[:K + 1].copy()
    a_new[K] = 0.0
    ap_new[K] = 0.0
    return a_new, ap_new


# ---------------------------------------------------------------------------------------------
# incident forcing g_j(t) = beta_j f(x_j - t) (eq. gj), f periodised in the periodic box
# ---------------------------------------------------------------------------------------------
def incident(s, amp, center, width, periodic):
    s = np.asarray(s, dtype=np.float64)
    f = np.zeros_like(s)
    for a, c, w in zip(amp, center, width):
        if not periodic:
            f += a * np.exp(-0.5 * ((s - c) / w) ** 2)
        else:
            mlo = int(np.floor((c - np.max(s) - 40 * w) / TWO_PI)) - 1
            mhi = int(np.ceil((c - np.min(s) + 40 * w) / TWO_PI)) + 1
            for m in range(mlo, mhi + 1):
                f += a * np.exp(-0.5 * ((s + TWO_PI * m - c) / w) ** 2)
    return f


# ---------------------------------------------------------------------------------------------
# the march
# ---------------------------------------------------------------------------------------------
class WFP:
    """The discrete WFP scheme on one workload.  `run(Nt)` returns (sigma, u_receivers)."""

    def __init__(self, x, beta, periodic, dt, eps, p, amp=(), center=(), width=(), xr=(),
                 gamma=0.5, W=None, NL=None, Ng=32, rbc_period=None, dense_modes_limit=1.5e9):
        self.x = np.asarray(x, dtype=np.float64)
        self.beta = np.asarray(beta, dtype=np.float64)
        self.xr = np.asarray(xr, dtype=np.float64).reshape(-1)
        self.periodic = bool(periodic)
        self.amp, self.center, self.width = (np.asarray(a, dtype=np.float64) for a in (amp, center, width))
        self.P = P = params(dt, eps, p, gamma, W, NL, Ng, rbc_period)
        self.win = Window(P.delta, P.b)
        self.swin = Window(P.delta_s, P.b)
        self.pk, self.qk = pk_qk(P, self.win)
        self.rot = rotation(P)
        M, R = len(self.x), len(self.xr)
        self.M, self.R = M, R
        # local weights for springs: explicit stack (m >= 1) and the nearby matrix S (m = 0)
        tj, sl, d = neighbour_pairs(self.x, self.x, P.delta, self.periodic)
        Q = local_weights(d, P, self.win)
        self.pairs = (tj, sl, d, Q)
        rows, cols, vals = [], [], []
        for m in range(1, P.m_max + 1):
            nz = Q[:, m] != 0.0
            rows.append(tj[nz])
            cols.append((m - 1) * M + sl[nz])
            vals.append(Q[nz, m])
        self.Cstack = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                    shape=(M, M * P.m_max))
        near = Q[:, 0] != 0.0
        Smat = sp.csr_matrix((0.5 * self.beta[tj[near]] * Q[near, 0], (tj[near], sl[near])),
                             shape=(M, M))
        self.IS = (sp.identity(M, format="csc") + Smat).tocsc()
        self.lu = spla.splu(self.IS)
        # receivers: full stack including m = 0 (sigma^{n+1} known when they are evaluated)
        if R:
            tr, sr, dr = neighbour_pairs(self.xr, self.x, P.delta, self.periodic)
            Qr = local_weights(dr, P, self.win)
            rows, cols, vals = [], [], []
            for m in range(0, P.m_max + 1):
                nz = Qr[:, m] != 0.0
                rows.append(tr[nz])
                cols.append(m * M + sr[nz])
                vals.append(Qr[nz, m])
            self.Rstack = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                        shape=(R, M * (P.m_max + 1)))
        # dense Fourier matrices when they fit
        self.E = None
        if M * (P.K + 1) * 16 <= dense_modes_limit:
            k = np.arange(P.K + 1, dtype=np.float64)
            self.E = np.exp(1j * self.x[:, None] * k[None, :])      # e^{i k x_j}
        self.reset()

    # -- state ---------------------------------------------------------------------------
    def reset(self):
        P = self.P
        self.n = 0
        self.sig_ring = np.zeros((P.m_max + 1, self.M))    # sig_ring[m] = sigma^{n-m}
        self.S_ring = np.zeros((P.W, P.K + 1), dtype=np.complex128)   # S_ring[m] = S^{n-1-m}
        self.alpha = np.zeros(P.K + 1, dtype=np.complex128)
        self.alpha_p = np.zeros(P.K + 1, dtype=np.complex128)

    def _type1(self, sigma):
        if self.E is not None:
            return (self.E.T @ sigma) / TWO_PI
        return type1(sigma, self.x, self.P.K)

    def _type2_springs(self, alpha):
        if self.E is not None:
            wts = np.full(self.P.K + 1, 2.0)
            wts[0] = 1.0
            return np.real(np.conj(self.E) @ (wts * alpha))
        return type2(alpha, self.x)

    def forcing(self, t):
        return self.beta * incident(self.x - t, self.amp, self.center, self.width, self.periodic)

    def step(self, g_next=None):
        """Advance n -> n+1.  Returns (sigma^{n+1}, u at receivers at t_{n+1})."""
        P = self.P
        n = self.n
        t1 = (n + 1) * P.dt
        # 1. S^n from sigma^n, pushed into the ring
        Sn = self._type1(self.sig_ring[0])
        self.S_ring = np.roll(self.S_ring, 1, axis=0)
        self.S_ring[0] = Sn
        # 2-3. driving terms and the exact rotation
        h, g = fir(self.pk, self.qk, self.S_ring, P.dt)
        self.alpha, self.alpha_p = mode_update(self.alpha, self.alpha_p, h, g, self.rot)
        # 4. radiation condition (free space)
        if not self.periodic and (n + 1) % P.rbc_period == 0:
            self.alpha, self.alpha_p = rbc_project(self.alpha, self.alpha_p, P, self.swin)
        # 5. history part at springs
        self.uH = self._type2_springs(self.alpha)
        # 6. local explicit sum (m >= 1) and the implicit solve
        stack = self.sig_ring[:P.m_max].reshape(-1)           # [sigma^n, ..., sigma^{n+1-m_max}]
        self.c_local = self.Cstack @ stack
        gn = self.forcing(t1) if g_next is None else np.asarray(g_next, dtype=np.float64)
        rhs = -gn - 0.5 * self.beta * self.c_local - self.beta * self.uH
        sig_new = self.lu.solve(rhs)
        self.sig_ring = np.roll(self.sig_ring, 1, axis=0)
        self.sig_ring[0] = sig_new
        self.n = n + 1
        # 7. receivers
        urec = np.zeros(self.R)
        if self.R:
            stack_r = self.sig_ring.reshape(-1)                # [sigma^{n+1}, ..., sigma^{n+1-m_max}]
            self.uH_rec = type2(self.alpha, self.xr)
            urec = 0.5 * (self.Rstack @ stack_r) + self.uH_rec
        return sig_new, urec

    def run(self, Nt, g=None):
        sig = np.zeros((Nt + 1, self.M))
        u = np.zeros((Nt + 1, self.R))
        for n in range(Nt):
            sig[n + 1], u[n + 1] = self.step(None if g is None else g[n + 1])
        return sig, u


def from_workload(w, **kw) -> WFP:
    return WFP(w.x, w.beta, w.bc == 0, w.dt, w.tol, w.p, w.amp, w.center, w.width, w.xr, **kw)
