"""Oracle of the adjoint (reverse-time) march of the discrete WFP scheme: the gradient of a
receiver misfit with respect to the spring stiffnesses.

TEST INFRASTRUCTURE ONLY — like the rest of this package, plain numpy / scipy in FP64; it is never
imported by the library.

For fixed stiffnesses beta, one step of the scheme (oracle/wfp.py, the step of eqs. densco,
hkcompdisc, alphakEvolutionFormulas, the projection of Sec. 4.4, historySol1 and linearSystem, and
the receivers of eq. localSol2) is a linear map of the state

    X^n = (sigma ring [sigma^n .. sigma^{n-m_max}], S ring [S^{n-1} .. S^{n-W}], alpha^n, alpha'^n)

and the forcing g^{n+1}.  For the misfit L = 1/2 sum_{n=1}^{Nt} sum_r (u_r^n - d_r^n)^2 the
gradient follows from the transposed steps taken in reverse order (the adjoint state Xbar^n),
each piece transposed in the real inner product Re <a, b> = sum Re(conj a b):

    type-1  S = E^T sigma / 2 pi            ->  sigmabar += Re(conj(E) Sbar) / 2 pi
    type-2  u = Re(conj(E) (w alpha))       ->  alphabar += w (E^T ubar)      (w = 1, 2, 2, ..)
    FIR     h = dt sum_m p[m] S[m]          ->  Sbar[m] += dt p[m] hbar (likewise q, g)
    rotation (real 2 x 2 per k)             ->  its transpose
    projection P (real-linear, Sec. 4.4)    ->  P^T (as a real matrix; the oracle builds it by
                                                applying P to unit vectors, at test sizes)
    local sum c = C stack                   ->  stackbar += C^T cbar
    solve (I + S) sigma = rhs               ->  rhsbar = (I + S)^{-T} sigmabar

beta enters the step through rhs = -beta f - (beta/2) c - beta u_H (incident forcing g = beta f,
eq. gj) and through S = diag(beta/2) Q0 (eq. linearSystem), so

    dL/dbeta_j = sum_n rhsbar_j^n ( -f_j^{n+1} - c_j^n / 2 - u_H,j^n - (Q0 sigma^{n+1})_j / 2 ).

The forward states are kept in memory (test sizes); a GPU version would recompute them from
checkpoints.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import wfp


def _real_matrix_of_projection(o: wfp.WFP) -> np.ndarray:
    """The projection of Sec. 4.4 as a real matrix on [Re alpha, Im alpha, Re alpha', Im alpha']."""
    K1 = o.P.K + 1
    n = 4 * K1
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        a = e[0:K1] + 1j * e[K1:2 * K1]
        ap = e[2 * K1:3 * K1] + 1j * e[3 * K1:4 * K1]
        a2, ap2 = wfp.rbc_project(a, ap, o.P, o.swin)
        A[:, c] = np.concatenate([a2.real, a2.imag, ap2.real, ap2.imag])
    return A


def misfit_and_gradient(o: wfp.WFP, Nt: int, d: np.ndarray, g: np.ndarray | None = None):
    """L = 1/2 sum_{n=1}^{Nt} |u^n - d^n|^2 over the receivers and dL/dbeta (M values).

    o: a fresh oracle (state at n = 0) with receivers; d: (Nt + 1, R) targets (row 0 unused);
    g: optional (Nt + 1, M) forcing in place of the incident wave (then it does not depend on
    beta)."""
    L, gb, _ = _sweep(o, Nt, d, g)
    return L, gb


def forcing_gradient(o: wfp.WFP, Nt: int, d: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dL/dg^{n} for a host forcing g ((Nt + 1, M); row 0 is not used by the march): since
    rhs = -g - ..., it is minus the adjoint of the right-hand side of each step."""
    return _sweep(o, Nt, d, g)[2]


def _sweep(o: wfp.WFP, Nt: int, d: np.ndarray, g: np.ndarray | None):
    P = o.P
    M, R, K1, mm, W = o.M, o.R, P.K + 1, P.m_max, P.W
    if o.E is None:
        raise ValueError("the adjoint oracle needs the dense Fourier matrices (small sizes)")
    E = o.E
    Er = np.exp(1j * o.xr[:, None] * np.arange(K1, dtype=np.float64)[None, :])
    wts = np.full(K1, 2.0)
    wts[0] = 1.0
    tj, sl, dd, Q = o.pairs
    near = Q[:, 0] != 0.0
    Q0 = sp.csr_matrix((Q[near, 0], (tj[near], sl[near])), shape=(M, M))
    ISt = o.IS.T.tocsc()
    from scipy.sparse.linalg import splu
    lut = splu(ISt)
    CsT = o.Cstack.T.tocsr()
    RsT = o.Rstack.T.tocsr()
    c_rot, s_over_k, k_s = o.rot
    Pmat = _real_matrix_of_projection(o) if not o.periodic else None

    # forward march, recording what the gradient needs
    o.reset()
    rec = []
    L = 0.0
    for n in range(Nt):
        t1 = (n + 1) * P.dt
        f = wfp.incident(o.x - t1, o.amp, o.center, o.width, o.periodic) if g is None else None
        sig, u = o.step(None if g is None else g[n + 1])
        r = u - d[n + 1]
        L += 0.5 * float(np.dot(r, r))
        rec.append((r, f, o.c_local.copy(), o.uH.copy(), sig.copy()))

    # reverse sweep
    sr = np.zeros((mm + 1, M))
    Sr = np.zeros((W, K1), dtype=np.complex128)
    ab = np.zeros(K1, dtype=np.complex128)
    apb = np.zeros(K1, dtype=np.complex128)
    gb = np.zeros(M)
    forcing_b = np.zeros((Nt + 1, M))
    for n in range(Nt - 1, -1, -1):
        r, f, c_loc, uH, sig_new = rec[n]
        # receivers (eq. localSol2): u = 1/2 Rstack [sigma^{n+1} .. ] + Re(conj(Er) (w alpha))
        sr += 0.5 * (RsT @ r).reshape(mm + 1, M)
        ab = ab + wts * (Er.T @ r)
        # ring shift of the densities: sigma^{n+1} is new, the older slots move down
        sig_b = sr[0].copy()
        srn = np.zeros((mm + 1, M))
        srn[:mm] += sr[1:]
        # implicit solve (I + S) sigma^{n+1} = rhs
        rhs_b = lut.solve(sig_b)
        forcing_b[n + 1] = -rhs_b
        gb += rhs_b * (-(f if f is not None else 0.0) - 0.5 * c_loc - uH - 0.5 * (Q0 @ sig_new))
        # rhs = -g - beta/2 c - beta u_H
        c_b = -0.5 * o.beta * rhs_b
        uH_b = -o.beta * rhs_b
        srn[:mm] += (CsT @ c_b).reshape(mm, M)
        ab = ab + wts * (E.T @ uH_b)
        # radiation projection (free space, after the mode update of these steps)
        if Pmat is not None and (n + 1) % P.rbc_period == 0:
            v = Pmat.T @ np.concatenate([ab.real, ab.imag, apb.real, apb.imag])
            ab = v[0:K1] + 1j * v[K1:2 * K1]
            apb = v[2 * K1:3 * K1] + 1j * v[3 * K1:4 * K1]
        # mode update (eq. alphakEvolutionFormulas) and its driving terms
        h_b, g_b = ab, apb
        ab, apb = c_rot * h_b - k_s * g_b, s_over_k * h_b + c_rot * g_b
        Srn = P.dt * (o.pk * h_b[None, :] + o.qk * g_b[None, :])
        Srn = Srn + Sr                                     # S ring of step n+1 after the push
        # the push of S^n into the ring
        Sn_b = Srn[0]
        Sr = np.zeros((W, K1), dtype=np.complex128)
        Sr[:W - 1] = Srn[1:]
        # type-1 of sigma^n (eq. densco)
        srn[0] += np.real(np.conj(E) @ Sn_b) / (2 * np.pi)
        sr = srn
    return L, gb, forcing_b
