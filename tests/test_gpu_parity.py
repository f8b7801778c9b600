"""Parity of the CUDA path (through the C-ABI) with the discrete WFP oracle (Oracle B).

Tolerance: relative max error <= 1e-9 over the whole recorded array (densities over springs x
steps, fields over receivers x steps), the bar set for FP64 mode.  Per-row checks at the full
free-space workload (M = 1e4) compare each stage with oracle functions applied to the GPU's own
state, so a failure names the stage.
"""
import math

import numpy as np
import pytest

from oracle import volterra, wfp
from paper_2507_07823_gb300 import build, wave1d, workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wave1d.lib()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _gpu_run(w, nsteps=None, **opt):
    plan = wave1d.Plan.from_workload(w, **opt)
    s, u = plan.solve(nsteps or w.Nt)
    info = plan.info
    plan.close()
    return s, u, info


def _oracle_run(w, nsteps=None, **kw):
    o = wfp.from_workload(w, **kw)
    s, u = o.run(nsteps or w.Nt)
    return s[1:], u[1:], o


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
def test_config0_full_run(tol):
    """Periodic box, M = 64, dt = 0.01, 1000 steps: every density and receiver value."""
    w = W.config0(tol=tol)
    sg, ug, info = _gpu_run(w)
    so, uo, o = _oracle_run(w)
    assert info.K == o.P.K and info.W == o.P.W and info.m_max == o.P.m_max
    assert _rel(sg, so) < TOL
    assert np.max(np.abs(uo)) > 1e-6          # the comparison is not on noise
    assert _rel(ug, uo) < TOL
    # and against the direct Volterra march (the truth the scheme approximates, ~1e-8 here)
    sa, ua = volterra.march_workload(w)
    assert _rel(sg, sa[1:]) < 1e-6


def test_free_space_with_radiation_projection():
    """Free space (Sec. 4.4): several projections, waves leaving the box."""
    w = W.make("free_small", M=40, bc=W.FREE, dt=0.005, Nt=1500, tol=1e-12, p=8, seed=99,
               beta_range=(0.5, 20.0), beta_dist="loguniform", amp=(1.0, 0.5),
               center=(-math.pi - 0.5, -math.pi - 0.9), width=(0.05, 0.1), R=5, margin=0.6)
    sg, ug, info = _gpu_run(w)
    so, uo, o = _oracle_run(w)
    assert info.rbc_period == o.P.rbc_period
    assert _rel(sg, so) < TOL
    assert np.max(np.abs(uo)) > 1e-6          # the comparison is not on noise
    assert _rel(ug, uo) < TOL


def test_ragged_multi_tile_periodic():
    """M = 3001 springs (not a multiple of any block size), nearby blocks, 500 steps (the
    scattered field reaches every receiver)."""
    w = W.make("ragged", M=3001, bc=W.PERIODIC, dt=2e-3, Nt=500, tol=1e-11, p=6, seed=5,
               beta_range=(1.0, 10.0), amp=(1.0,), center=(-2.0,), width=(0.05,), R=7)
    sg, ug, info = _gpu_run(w)
    assert info.blocks < w.M            # some springs closer than dt are coupled
    so, uo, _ = _oracle_run(w)
    assert _rel(sg, so) < TOL
    assert np.max(np.abs(uo)) > 1e-6          # the comparison is not on noise
    assert _rel(ug, uo) < TOL


@pytest.mark.parametrize("p", [2, 4])
def test_low_orders(p):
    w = W.config0(p=p, Nt=400)
    sg, ug, _ = _gpu_run(w)
    so, uo, _ = _oracle_run(w)
    assert _rel(sg, so) < TOL and _rel(ug, uo) < TOL


def test_single_spring_and_zero_stiffness():
    w = W.config0(Nt=300).with_(x=np.array([0.7]), beta=np.array([5.0]))
    sg, ug, _ = _gpu_run(w)
    so, uo, _ = _oracle_run(w)
    assert _rel(sg, so) < TOL and _rel(ug, uo) < TOL
    w0 = W.config0(Nt=200)
    w0 = w0.with_(beta=np.zeros(w0.M))
    sg, ug, _ = _gpu_run(w0)
    assert np.all(sg == 0.0) and np.all(ug == 0.0)


def test_graph_replay_matches_single_steps():
    """Steps replayed from captured graphs equal steps queued one by one, bit for bit."""
    w = W.config0(Nt=200)
    a = wave1d.Plan.from_workload(w)
    s1, u1 = a.solve(200)
    b = wave1d.Plan.from_workload(w)
    s2 = np.zeros((200, w.M))
    u2 = np.zeros((200, w.R))
    for n in range(200):
        b.step()
        s2[n] = b.sigma()
        u2[n] = b.receivers()
    assert np.array_equal(s1, s2) and np.array_equal(u1, u2)
    a.close()
    b.close()


def test_step_kernel_matches_per_stage_launches():
    """The one-launch step kernel and the per-stage kernels run the same phases in the same order
    of summation: equal bit for bit over 250 steps of the M = 1e4 free-space workload (four
    radiation projections, which both paths run as per-stage launches)."""
    w = W.config1()
    n = 250
    a = wave1d.Plan.from_workload(w, step_kernel=1)
    s1, u1 = a.solve(n)
    b = wave1d.Plan.from_workload(w, step_kernel=0)
    s2, u2 = b.solve(n)
    a.close()
    b.close()
    assert np.max(np.abs(s1[-1])) > 0.0
    assert np.array_equal(s1, s2) and np.array_equal(u1, u2)


def test_checkpoint_resume_is_bitwise():
    """wave1d_state_save after 150 steps, wave1d_state_load into a fresh plan built from the same
    inputs, 150 more steps: bit for bit the uninterrupted 300-step march (free space, projection
    steps on both sides of the checkpoint); a buffer from a plan of other sizes is refused."""
    w = W.make("ckpt", M=300, bc=W.FREE, dt=4e-3, Nt=300, tol=1e-10, p=6, seed=11,
               beta_range=(0.5, 20.0), beta_dist="loguniform", amp=(1.0,), center=(-math.pi - 0.4,),
               width=(0.05,), R=3, margin=0.6)
    a = wave1d.Plan.from_workload(w)
    s_all, u_all = a.solve(300)
    b = wave1d.Plan.from_workload(w)
    s1, u1 = b.solve(150)
    buf = np.zeros(wave1d.wave1d_state_size(b.h), dtype=np.uint8)
    wave1d._check(wave1d.wave1d_state_save(b.h, buf), "wave1d_state_save")
    b.close()
    c = wave1d.Plan.from_workload(w)
    wave1d._check(wave1d.wave1d_state_load(c.h, buf), "wave1d_state_load")
    s2, u2 = c.solve(150)
    assert np.array_equal(np.vstack([s1, s2]), s_all) and np.array_equal(np.vstack([u1, u2]), u_all)
    assert np.max(np.abs(s_all[150:])) > 1e-6          # the pulse has reached the springs
    other = wave1d.Plan.from_workload(w.with_(x=w.x[:-1], beta=w.beta[:-1]))
    assert wave1d.wave1d_state_load(other.h, buf) == wave1d.WAVE1D_EINVAL
    other.close()
    a.close()
    c.close()


def test_host_forcing_matches_incident_forcing():
    """wave1d_step with g from the host reproduces the incident-wave forcing (eq. gj)."""
    w = W.config0(Nt=200)
    a = wave1d.Plan.from_workload(w)
    s1, _ = a.solve(200)
    b = wave1d.Plan(w.x, w.beta, w.bc, w.dt, w.Nt, w.tol, xr=w.xr, p=w.p)
    for n in range(200):
        t = (n + 1) * w.dt
        g = w.beta * wfp.incident(w.x - t, w.amp, w.center, w.width, True)
        b.step(g)
    assert _rel(b.sigma(), s1[-1]) < 1e-13
    a.close()
    b.close()


def test_step_past_nt_and_errors():
    w = W.config0(Nt=3)
    a = wave1d.Plan.from_workload(w)
    a.solve(3)
    assert wave1d.wave1d_step(a.h) == wave1d.WAVE1D_EDONE
    a.close()


def test_stages_at_full_free_space_size():
    """M = 1e4 free space (the benchmark workload): each stage against the oracle applied to the
    GPU's own state, 2004 steps in (many projections; the pulse is inside the springs)."""
    w = W.config1()
    plan = wave1d.Plan.from_workload(w)
    o = wfp.params(w.dt, w.tol, w.p)
    n0 = 37 * plan.info.rbc_period + 5          # step n0 -> n0+1 is not a projection step
    assert (n0 + 1) % plan.info.rbc_period != 0
    plan.solve(n0, with_sigma=False)
    ring0 = plan.inspect(wave1d.WAVE1D_ARR_SIGMA_RING)        # sigma^{n0 - m}
    a0 = plan.inspect(wave1d.WAVE1D_ARR_ALPHA)
    ap0 = plan.inspect(wave1d.WAVE1D_ARR_ALPHA_P)
    plan.step()
    S = plan.inspect(wave1d.WAVE1D_ARR_S_LAST)                # S^{n0}
    a1 = plan.inspect(wave1d.WAVE1D_ARR_ALPHA)
    uH = plan.inspect(wave1d.WAVE1D_ARR_UH)
    cl = plan.inspect(wave1d.WAVE1D_ARR_LOCAL)
    sig1 = plan.sigma()
    # type-1 NUFFT (eq. densco): relative to sum |sigma| / 2 pi
    S_ref = wfp.type1(ring0[0], w.x, o.K)
    scale = np.sum(np.abs(ring0[0])) / (2 * math.pi)
    assert np.max(np.abs(S - S_ref)) < 1e-11 * scale
    # FIR + rotation (eqs. hkcompdisc, alphakEvolutionFormulas) from the GPU's S history
    win = wfp.Window(o.delta, o.b)
    pk, qk = wfp.pk_qk(o, win)
    S_ring = np.array([wfp.type1(ring0[m], w.x, o.K) for m in range(o.W)])
    h, g = wfp.fir(pk, qk, S_ring, o.dt)
    a_ref, _ = wfp.mode_update(a0, ap0, h, g, wfp.rotation(o))
    assert np.max(np.abs(a1 - a_ref)) < 1e-10 * np.max(np.abs(a_ref))
    # type-2 NUFFT (eq. historySol1) relative to sum |alpha|
    uH_ref = wfp.type2(a1, w.x)
    assert np.max(np.abs(uH - uH_ref)) < 1e-11 * np.sum(np.abs(a1))
    # local explicit sum on sampled targets (Sec. 4.1)
    rng = np.random.default_rng(0)
    sample = rng.choice(w.M, 200, replace=False)
    tj, sl, d = wfp.neighbour_pairs(w.x[sample], w.x, o.delta, False)
    Q = wfp.local_weights(d, o, win)
    m = np.arange(1, o.m_max + 1)
    # ring0[m - 1] holds sigma^{n0+1-m}
    contrib = np.sum(Q[:, 1:] * ring0[m - 1][:, sl].T, axis=1)
    c_ref = np.bincount(tj, weights=contrib, minlength=len(sample))
    assert np.max(np.abs(cl[sample] - c_ref)) < 1e-12 * max(np.max(np.abs(c_ref)), 1e-300) + 1e-300
    # the solve: sigma^{n0+1} from the GPU's own c, u_H and the forcing
    t1 = (n0 + 1) * w.dt
    gj = w.beta * wfp.incident(w.x - t1, w.amp, w.center, w.width, False)
    rhs = -gj - 0.5 * w.beta * cl - w.beta * uH
    tj2, sl2, d2 = wfp.neighbour_pairs(w.x, w.x, o.dt, False)
    near = d2 < o.dt
    Q0 = wfp.local_weights(d2[near], o, win)[:, 0]
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = sp.identity(w.M, format="csc") + sp.csr_matrix(
        (0.5 * w.beta[tj2[near]] * Q0, (tj2[near], sl2[near])), shape=(w.M, w.M)).tocsc()
    sig_ref = spla.spsolve(A, rhs)
    assert _rel(sig1, sig_ref) < 1e-10
    plan.close()


def test_config1_first_steps_against_oracle():
    """The full M = 1e4 free-space workload against Oracle B, element by element, over the
    first 1100 steps (20 radiation projections; the pulses enter the springs at t ~ 0.26 and the
    scattered field reaches the first receiver at t ~ 0.8)."""
    w = W.config1()
    n = 1100
    sg, ug, _ = _gpu_run(w, n)
    so, uo, _ = _oracle_run(w, n)
    assert _rel(sg, so) < TOL
    assert np.max(np.abs(uo)) > 1e-6          # the comparison is not on noise
    assert _rel(ug, uo) < TOL


def test_pairs_at_distance_dt_within_rounding():
    """Springs spaced exactly dt apart in exact arithmetic (centres of 200 cells of [-1, 1],
    dt = 0.01): rounding puts some neighbour distances just below dt (nearby: the implicit
    coupling) and others at or above it, and pairs 36 spacings apart sit at delta = 0.36 within
    rounding, inside the local part with every weight zero (such a source once broke the
    m-ordered rows of the local sum).  Every density and receiver value against the oracle of the
    scheme over 2000 steps, free space."""
    w = W.uniform_array(200, 1.0, Nt=2000).with_(x=-1.0 + (np.arange(200) + 0.5) * (2.0 / 200),
                                                 xr=np.array([-1.8, -0.95, 0.95, 1.8]))
    d = np.abs(np.diff(w.x))
    assert (d < w.dt).any() and (d >= w.dt).any()     # both kinds of tie are present
    sg, ug, _ = _gpu_run(w)
    so, uo, _ = _oracle_run(w)
    es, eu = _rel(sg, so), _rel(ug, uo)
    print(f"pairs at dt: sigma {es:.2e}, receivers {eu:.2e}")
    assert es < TOL and eu < TOL


def test_large_implicit_blocks():
    """Blocks of springs closer than dt with 300 members (the solve's single-task path above 256
    members) and 40 members (32-row tasks), free space, every density and receiver value against
    the oracle of the scheme over 300 steps."""
    dt = 0.01
    x = np.concatenate([-1.5 + 0.004 * np.arange(300), 0.5 + 0.004 * np.arange(40)])
    beta = np.random.default_rng(8).uniform(0.5, 3.0, x.size)
    w = W.config0().with_(bc=W.FREE, x=x, beta=beta, center=np.array([-2.6]), width=np.array([0.08]),
                          dt=dt, Nt=300, tol=1e-10, xr=np.array([-1.8, 0.0, 1.2]))
    sg, ug, info = _gpu_run(w)
    so, uo, _ = _oracle_run(w)
    print(f"large blocks: max block {info.max_block}, sigma {_rel(sg, so):.2e}, receivers {_rel(ug, uo):.2e}")
    assert info.max_block == 300
    assert np.max(np.abs(so)) > 1e-3
    assert _rel(sg, so) < TOL and _rel(ug, uo) < TOL
