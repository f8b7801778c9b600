"""The million-spring clustered workload (periodic box, 16 Gaussian clusters of width 0.05 plus 20 %
uniform springs, beta uniform in [1, 10], dt = 5e-4, tol = 1e-10, p = 4) on the GPU, through the
plan without pair lists (opts.local_weights = 1): 1.3e10 pairs within delta, one block of
931,311 springs closer than dt to a neighbour, neither of which a stored-weight plan can hold.

The springs are those of the benchmark; the incident pulse is narrower (width 0.01) and starts
0.06 from the first springs it meets (the benchmark's pulse, width 0.1 at x = -2, reaches no spring
for about 1300 steps), so the field is live within the first hundred steps.

* First 100 steps against the oracle: until the scattered field has travelled further than the
  pulse's reach, only the springs near it carry a density; the oracle of the discrete scheme
  (direct Fourier sums, FP64 local weights per pair, sparse LU) run on those springs alone (the
  others stay at zero up to the scheme's 1e-10 window error) gives their densities, which the full
  GPU march must reproduce.
* Each stage on the GPU's own state after those steps, at sampled rows and modes: type-1 sums
  S_k against direct sums (eq. densco), u_H against direct type-2 sums (eq. historySol1), the local
  sums c_j against the oracle's weights Q_m(d) (Sec. 4.1) over each row's full neighbour window, and
  the residual of eq. linearSystem with the oracle's Q_0.
* Self-convergence in dt over a live window (dt, dt/2, dt/4)."""
import math

import numpy as np
import pytest

from oracle import wfp
from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PULSE = dict(amp=np.array([1.0]), center=np.array([-1.26]), width=np.array([0.01]))
NSTEPS = 100


def _workload(dt=5e-4, Nt=NSTEPS):
    return W.config2(Nt=Nt).with_(dt=dt, xr=np.array([-1.19, -1.15, 0.5]), **PULSE)


@pytest.fixture(scope="module")
def marched():
    w = _workload()
    plan = wave1d.Plan.from_workload(w, local_weights=1)
    sigma, u = plan.solve(NSTEPS)
    state = {"sigma": sigma, "u": u, "ring": plan.inspect(wave1d.WAVE1D_ARR_SIGMA_RING),
             "local": plan.inspect(wave1d.WAVE1D_ARR_LOCAL), "uH": plan.inspect(wave1d.WAVE1D_ARR_UH),
             "S": plan.inspect(wave1d.WAVE1D_ARR_S_LAST), "alpha": plan.inspect(wave1d.WAVE1D_ARR_ALPHA),
             "info": plan.info}
    plan.close()
    return w, state


def test_first_steps_against_the_oracle_on_the_live_springs(marched):
    w, st = marched
    sigma = st["sigma"]
    live = np.max(np.abs(sigma), axis=0)
    assert live.max() > 1e-2                                   # the field is live
    # outside [-1.21, -1.10] the densities stay at the level of the window tolerance (the history
    # part is band-limited, not exactly causal): the springs there do not act on those inside
    outside = (w.x < -1.21) | (w.x > -1.10)
    print(f"largest density outside the live region: {live[outside].max() / live.max():.1e} of the largest")
    assert live[outside].max() < 1e-8 * live.max()
    sub = np.nonzero((w.x > -1.212) & (w.x < -1.09))[0]
    o = wfp.WFP(w.x[sub], w.beta[sub], True, w.dt, w.tol, w.p, w.amp, w.center, w.width, ())
    s_ref, _ = o.run(NSTEPS)
    got = sigma[:, sub]
    err = float(np.max(np.abs(got - s_ref[1:])) / np.max(np.abs(s_ref)))
    print(f"first {NSTEPS} steps, {sub.size} springs: rel max err {err:.2e}")
    assert err < 1e-9


def _rows(w, rng, n):
    """n sampled springs: half on the live front, half anywhere (sorted order indices)."""
    xs = np.sort(w.x)
    front = np.nonzero((xs > -1.2) & (xs < -1.14))[0]
    return np.unique(np.concatenate([rng.choice(front, n // 2, replace=False), rng.choice(xs.size, n // 2, replace=False)]))


def _neighbours(xs, j, radius):
    """Sources within `radius` of sorted spring j (periodic nearest image): indices, distances."""
    d = np.abs(xs - xs[j]) % (2 * math.pi)
    d = np.minimum(d, 2 * math.pi - d)
    nb = np.nonzero(d < radius)[0]
    return nb, d[nb]


def test_stages_on_the_gpu_state(marched):
    w, st = marched
    n = NSTEPS
    perm = np.argsort(w.x, kind="stable")                      # sorted index -> caller index
    xs, bs = w.x[perm], w.beta[perm]
    ring = st["ring"]                                          # ring[m] = sigma^{n-m}, caller order
    P = wfp.params(w.dt, w.tol, w.p)
    win = wfp.Window(P.delta, P.b)
    rng = np.random.default_rng(11)
    rows = _rows(w, rng, 200)

    # type-1 sums of sigma^{n-1} (the last step's spreading) on sampled modes
    k = np.unique(np.concatenate([np.arange(8), rng.integers(0, P.K + 1, 56)]))
    s_prev = ring[1]
    S_ref = (np.exp(1j * np.outer(k, w.x)) @ s_prev) / (2 * math.pi)
    e_S = np.max(np.abs(st["S"][k] - S_ref)) / np.max(np.abs(S_ref))
    # u_H at sampled springs from alpha^n (eq. historySol1): weights 1 for k = 0, 2 otherwise
    kk = np.arange(P.K + 1)
    wk = np.where(kk == 0, 1.0, 2.0)
    xr = xs[rows]
    uH_ref = np.real(np.exp(-1j * np.outer(xr, kk)) @ (wk * st["alpha"]))
    uH_got = st["uH"][perm[rows]]
    e_uH = np.max(np.abs(uH_got - uH_ref)) / np.max(np.abs(st["uH"]))
    # local sums c_j (m >= 1) with the oracle's weights over the full window, and the residual of
    # the implicit equation with the oracle's Q_0
    c_err, c_scale, r_err, r_scale = 0.0, 0.0, 0.0, 0.0
    t1 = n * w.dt
    for j in rows:
        nb, d = _neighbours(xs, j, P.delta)
        Q = wfp.local_weights(d, P, win)
        # the last step (n-1 -> n) summed sigma^{n-m}, m = 1..m_max, of the sources
        terms = Q[:, 1:].T * ring[1:P.m_max + 1][:, perm[nb]]
        c_ref = terms.sum()
        c_err = max(c_err, abs(st["local"][perm[j]] - c_ref))
        c_scale = max(c_scale, np.abs(terms).sum())
        near = d < P.dt
        g = bs[j] * wfp.incident(xs[j] - t1, w.amp, w.center, w.width, True)
        rhs = -g - 0.5 * bs[j] * st["local"][perm[j]] - bs[j] * st["uH"][perm[j]]
        lhs = ring[0][perm[j]] + 0.5 * bs[j] * np.dot(Q[near, 0], ring[0][perm[nb[near]]])
        r_err = max(r_err, abs(lhs - rhs))
        r_scale = max(r_scale, abs(ring[0][perm[j]]))
    print(f"type-1 {e_S:.2e}  u_H {e_uH:.2e}  local {c_err / c_scale:.2e}  residual {r_err / r_scale:.2e}")
    assert e_S < 1e-9 and e_uH < 1e-9
    assert c_err < 1e-11 * c_scale
    assert r_err < 1e-12 * r_scale


@pytest.mark.slow
def test_self_convergence_in_dt():
    """sigma on the live springs at t = 0.05 .. 0.1 from marches at dt, dt/2, dt/4: the differences
    fall with dt (p = 8) until the window tolerance's floor."""
    T = 0.1
    out = {}
    for r in (1, 2, 4):
        w = _workload(dt=5e-4 / r, Nt=int(round(T / (5e-4 / r))))
        plan = wave1d.Plan.from_workload(w, local_weights=1)
        try:
            s, _ = plan.solve(w.Nt)
        finally:
            plan.close()
        live = (w.x > -1.21) & (w.x < -1.10)
        out[r] = s[r - 1::r][100:, live]                      # common times t = 0.05 .. 0.1
    e12 = np.max(np.abs(out[1] - out[2])) / np.max(np.abs(out[2]))
    e24 = np.max(np.abs(out[2] - out[4])) / np.max(np.abs(out[4]))
    print(f"self-convergence: |dt - dt/2| {e12:.2e}, |dt/2 - dt/4| {e24:.2e}")
    assert e12 < 1e-6 and e24 < e12
