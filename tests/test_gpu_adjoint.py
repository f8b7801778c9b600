"""GPU reverse-time march (wave1d_adjoint): dL/dbeta of a receiver misfit against the adjoint
oracle (oracle/adjoint.py) at 1e-9 of the largest component, the same gradient through the
torch.autograd wrapper, dL/dbeta and dL/dg of a march driven by forcing vectors, bitwise
reproducibility, and central differences of the GPU forward march on a larger free-space layout
(several projections, hundreds of springs).

The kernels' bodies are also checked on the CPU against the same oracle by
tests/test_host_adjoint.py."""
import numpy as np
import pytest

from oracle import adjoint, wfp
from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _layout(bc, seed=5, M=10, p=6, dt=0.02, Nt=400):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(-0.8, 0.8, M))
    x[3] = x[2] + 0.4 * dt                       # an implicit block
    beta = rng.uniform(1.0, 6.0, M)
    xr = np.array([-0.95, 0.1, x[5], 0.95])      # one receiver on a spring (m = 0 terms)
    return W.Workload(name="adjoint", bc=bc, x=x, beta=beta, amp=np.array([1.0]), center=np.array([-1.6]),
                      width=np.array([0.12]), dt=dt, Nt=Nt, tol=1e-10, p=p, xr=xr, seed=seed)


def _targets(w):
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    return 0.3 * np.sin(3.0 * t + w.xr[None, :])


@pytest.mark.parametrize("bc", [W.PERIODIC, W.FREE])
def test_gradient_matches_the_adjoint_oracle(bc):
    w = _layout(bc)
    d = _targets(w)
    _, g_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d)
    plan = wave1d.Plan.from_workload(w)
    try:
        sigma, u = plan.solve_device(w.Nt)
        ubar = u - torch.from_numpy(d[1:]).cuda()
        g = plan.adjoint(sigma, ubar).cpu().numpy()
    finally:
        plan.close()
    assert np.max(np.abs(g - g_oracle)) <= 1e-9 * np.max(np.abs(g_oracle)), (g, g_oracle)


def test_gradient_matches_the_adjoint_oracle_at_64_springs():
    """64 free-space springs with stiffnesses uniform in [1, 10] (the adjoint workload's draw),
    8 receivers, a seeded target trace: dL/dbeta against the adjoint oracle at 1e-9."""
    rng = np.random.default_rng(64)
    M, dt, Nt = 64, 0.01, 300
    x = np.sort(rng.uniform(-1.0, 1.0, M))
    w = W.Workload(name="adjoint-64", bc=W.FREE, x=x, beta=rng.uniform(1.0, 10.0, M), amp=np.array([1.0]),
                   center=np.array([-1.8]), width=np.array([0.1]), dt=dt, Nt=Nt, tol=1e-10, p=6,
                   xr=np.linspace(-1.2, 1.2, 8), seed=64)
    d = 0.01 * rng.standard_normal((Nt + 1, 8))
    _, g_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d)
    plan = wave1d.Plan.from_workload(w)
    try:
        sigma, u = plan.solve_device(w.Nt)
        g = plan.adjoint(sigma, u - torch.from_numpy(d[1:]).cuda()).cpu().numpy()
    finally:
        plan.close()
    assert np.max(np.abs(g - g_oracle)) <= 1e-9 * np.max(np.abs(g_oracle))


def test_gradient_is_bitwise_reproducible():
    """No launch of the reverse march uses atomics: two calls give the same bits."""
    w = _layout(W.FREE, seed=7)
    d = torch.from_numpy(_targets(w)[1:]).cuda()
    plan = wave1d.Plan.from_workload(w)
    try:
        sigma, u = plan.solve_device(w.Nt)
        g1 = plan.adjoint(sigma, u - d)
        g2 = plan.adjoint(sigma, u - d)
    finally:
        plan.close()
    assert torch.equal(g1, g2)


def test_forcing_vector_march_gradients_match_the_oracle():
    """A march driven by forcing vectors (wave1d_step(g)): dL/dbeta and dL/dg against the oracle."""
    w = _layout(W.PERIODIC, seed=13)
    rng = np.random.default_rng(6)
    g = 0.2 * rng.standard_normal((w.Nt + 1, w.M))
    d = _targets(w)
    plan = wave1d.Plan(w.x, w.beta, w.bc, w.dt, w.Nt, w.tol, (), (), (), w.xr, p=w.p)
    try:
        sig, u = np.zeros((w.Nt, w.M)), np.zeros((w.Nt, len(w.xr)))
        for n in range(w.Nt):
            plan.step(np.ascontiguousarray(g[n + 1]))
            sig[n], u[n] = plan.sigma(), plan.receivers()
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
        gb, gg = plan.adjoint(dev(sig), dev(u - d[1:]), g=dev(g[1:]), forcing_gradient=True)
    finally:
        plan.close()
    _, gb_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d, g=g)
    gg_oracle = adjoint.forcing_gradient(wfp.from_workload(w), w.Nt, d, g)[1:]
    gb, gg = gb.cpu().numpy(), gg.cpu().numpy()
    assert np.max(np.abs(gb - gb_oracle)) <= 1e-9 * np.max(np.abs(gb_oracle))
    assert np.max(np.abs(gg - gg_oracle)) <= 1e-9 * np.max(np.abs(gg_oracle))


def test_autograd_wrapper_gives_the_same_gradient():
    w = _layout(W.FREE, seed=9)
    d = torch.from_numpy(_targets(w)[1:]).cuda()
    beta = torch.tensor(w.beta, dtype=torch.float64, device="cuda", requires_grad=True)
    u = wave1d.receiver_fields(beta, w, w.Nt)
    loss = 0.5 * torch.sum((u - d) ** 2)
    loss.backward()
    L, g_oracle = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, _targets(w))
    assert abs(loss.item() - L) <= 1e-9 * L
    g = beta.grad.cpu().numpy()
    assert np.max(np.abs(g - g_oracle)) <= 1e-9 * np.max(np.abs(g_oracle))


def test_gradient_matches_central_differences_of_the_gpu_march():
    """Free space, 400 springs in [-2.5, 2.5], dt = 5e-3, 600 steps (projections every
    ceil(1.5 W) steps), 4 receivers: the adjoint gradient on 8 stiffnesses against central
    differences of the GPU forward march (step 1e-4 beta_j)."""
    rng = np.random.default_rng(2024)
    M, dt, Nt = 400, 5e-3, 600
    x = np.sort(rng.uniform(-2.5, 2.5, M))
    beta = rng.uniform(1.0, 10.0, M)
    xr = np.array([-2.6, -0.3, 0.4, 2.6])                  # inside |x| <= pi - 3 delta (delta = 0.15)
    w = W.Workload(name="adjoint-fd", bc=W.FREE, x=x, beta=beta, amp=np.array([1.0]), center=np.array([-3.3]),
                   width=np.array([0.1]), dt=dt, Nt=Nt, tol=1e-10, p=8, xr=xr, seed=2024)
    d = torch.from_numpy(_targets(w)[1:]).cuda()

    def loss_of(b):
        plan = wave1d.Plan(w.x, b, w.bc, w.dt, w.Nt, w.tol, w.amp, w.center, w.width, w.xr, p=w.p)
        try:
            sigma, u = plan.solve_device(Nt)
            return 0.5 * float(torch.sum((u - d) ** 2)), sigma, u, plan
        except Exception:
            plan.close()
            raise

    L, sigma, u, plan = loss_of(beta)
    try:
        g = plan.adjoint(sigma, u - d).cpu().numpy()
    finally:
        plan.close()
    for j in rng.choice(M, 8, replace=False):
        h = 1e-4 * beta[j]
        bp, bm = beta.copy(), beta.copy()
        bp[j] += h
        bm[j] -= h
        Lp, *rest = loss_of(bp)
        rest[-1].close()
        Lm, *rest = loss_of(bm)
        rest[-1].close()
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[j] - fd) <= 1e-6 * np.max(np.abs(g)), (j, g[j], fd)


@pytest.mark.parametrize("interval", [37, 64, 1000])
def test_checkpointed_gradient_equals_the_stored_density_gradient(interval):
    """wave1d_solve_checkpointed + wave1d_adjoint_checkpointed (the march state kept every
    `interval` steps, each segment marched again in the reverse pass) against wave1d_adjoint from
    the stored densities: the same dL/dbeta and dL/dg bit for bit (intervals that do and do not
    divide the march, one longer than it), and the plan back at the end of its march."""
    w = _layout(W.FREE, seed=21, M=40, dt=0.02, Nt=400)
    rng = np.random.default_rng(3)
    w = w.with_(x=np.sort(rng.uniform(-0.9, 0.9, w.M)), beta=rng.uniform(1.0, 6.0, w.M))
    nsteps = 300
    d = torch.from_numpy(_targets(w)[1:nsteps + 1]).cuda()
    ref = wave1d.Plan.from_workload(w)
    plan = wave1d.Plan.from_workload(w)
    try:
        sigma, u = ref.solve_device(nsteps)
        gb, gg = ref.adjoint(sigma, u - d, forcing_gradient=True)
        u2, ckpt = plan.solve_checkpointed(nsteps, interval)
        assert torch.equal(u, u2)
        gb2, gg2 = plan.adjoint_checkpointed(ckpt, nsteps, interval, u2 - d, forcing_gradient=True)
        assert torch.equal(gb, gb2) and torch.equal(gg, gg2)
        assert float(torch.max(torch.abs(gb))) > 0.0
        # the plan continues from the end of its march as the uninterrupted one does
        for _ in range(5):
            ref.step()
            plan.step()
        assert np.array_equal(ref.sigma(), plan.sigma())
        assert np.array_equal(ref.receivers(), plan.receivers())
    finally:
        ref.close()
        plan.close()


def test_checkpointed_march_rejects_mismatched_calls():
    w = _layout(W.PERIODIC, seed=4, Nt=100)
    plan = wave1d.Plan.from_workload(w)
    try:
        u, ckpt = plan.solve_checkpointed(60, 16)
        ubar = torch.zeros_like(u)
        # other interval or length than the march that wrote the checkpoints
        for n, iv in ((60, 15), (59, 16)):
            gb = torch.empty(w.M, dtype=torch.float64, device="cuda")
            assert wave1d.wave1d_adjoint_checkpointed(plan.h, n, iv, ckpt, ubar, gb, None) == wave1d.WAVE1D_EINVAL
        # a march that does not start at step 0
        assert wave1d.wave1d_solve_checkpointed(plan.h, 10, 5, None, ckpt) == wave1d.WAVE1D_EINVAL
    finally:
        plan.close()


@pytest.mark.parametrize("bc", [W.PERIODIC, W.FREE])
def test_plan_without_pair_lists_gives_the_stored_weight_gradient(bc):
    """The reverse march of a plan without pair lists (transposed local sum from the range tables'
    polynomials, transposed Jacobi solve, transposed receiver read-out) against the stored-weight
    plan's on the same layout: dL/dbeta and dL/dg to 1e-9 of the largest component (the two
    forward marches themselves agree to about 1e-12); and its checkpointed form bit for bit."""
    w = _layout(bc, seed=31, M=60, dt=0.02, Nt=400)
    rng = np.random.default_rng(8)
    w = w.with_(x=np.sort(rng.uniform(-0.9, 0.9, w.M)), beta=rng.uniform(1.0, 6.0, w.M))
    nsteps = 300
    d = torch.from_numpy(_targets(w)[1:nsteps + 1]).cuda()
    out = {}
    for lw in (0, 1):
        plan = wave1d.Plan.from_workload(w, local_weights=lw)
        try:
            sigma, u = plan.solve_device(nsteps)
            out[lw] = (u, *plan.adjoint(sigma, u - d, forcing_gradient=True))
        finally:
            plan.close()
    (u0, gb0, gg0), (u1, gb1, gg1) = out[0], out[1]
    assert float(torch.max(torch.abs(u1 - u0))) <= 1e-10 * float(torch.max(torch.abs(u0)))
    assert float(torch.max(torch.abs(gb1 - gb0))) <= 1e-9 * float(torch.max(torch.abs(gb0)))
    assert float(torch.max(torch.abs(gg1 - gg0))) <= 1e-9 * float(torch.max(torch.abs(gg0)))
    plan = wave1d.Plan.from_workload(w, local_weights=1)
    try:
        u2, ckpt = plan.solve_checkpointed(nsteps, 64)
        gb2, gg2 = plan.adjoint_checkpointed(ckpt, nsteps, 64, u2 - d, forcing_gradient=True)
    finally:
        plan.close()
    assert torch.equal(u2, u1) and torch.equal(gb2, gb1) and torch.equal(gg2, gg1)
