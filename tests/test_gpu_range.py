"""Plans without pair lists (opts.local_weights = 1): the local sum over sorted index windows with
the weights from their polynomials in the distance (compensated FP32 pairs), the implicit part by
Jacobi sweeps.  The march against the stored-weight plan of the same scheme and against the
discrete scheme's oracle, in the periodic box, in free space and on a clustered layout whose blocks
of 256 targets hold many sources (receivers placed where the field is live); the reverse march
of such a plan refuses a zero stiffness.

Bars: 1e-10 against the stored-weight plan (the range tables hold every weight to 1e-12 of
max |Q|; single-float rounding of each source's curvature terms gives local sums within about 2e-11
of the FP64 weights where rows hold few sources), 1e-9 against the oracle."""
import numpy as np
import pytest

from oracle import wfp
from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _march(w, n, **kw):
    plan = wave1d.Plan.from_workload(w, **kw)
    try:
        return plan.solve(n)
    finally:
        plan.close()


def _clustered():
    w = W.config2(M=3000, Nt=300, width=(0.005,))
    # receivers among the springs the pulse reaches first (the pulse starts at x = -2)
    return w.with_(xr=np.array([-1.99, -1.97, -1.9, 2.5]))


@pytest.mark.parametrize("which", ["periodic", "free", "clustered"])
def test_range_march_matches_stored_weights_and_the_oracle(which):
    if which == "periodic":
        w = W.config0(Nt=300)
    elif which == "free":
        w = W.config1(M=400, Nt=300, dt=0.005, margin=0.6)
    else:
        w = _clustered()
    s0, u0 = _march(w, w.Nt)
    s1, u1 = _march(w, w.Nt, local_weights=1)
    assert np.max(np.abs(s0)) > 1e-3 and np.max(np.abs(u0)) > 1e-6
    assert _rel(s1, s0) < 1e-10 and _rel(u1, u0) < 1e-10, (_rel(s1, s0), _rel(u1, u0))
    s_ref, u_ref = wfp.from_workload(w).run(w.Nt)
    assert _rel(s1, s_ref[1:]) < 1e-9 and _rel(u1, u_ref[1:]) < 1e-9


def test_range_plan_reports_its_pairs_and_no_stored_weights():
    w = _clustered()
    p0 = wave1d.Plan.from_workload(w)
    p1 = wave1d.Plan.from_workload(w, local_weights=1)
    try:
        i0, i1 = p0.info, p1.info
        # the same pairs within delta, each spring with itself included (the stored plan lists them,
        # the range plan only counts them)
        assert i1.local_pairs == i0.local_pairs
        assert i1.local_weights == 0 and i1.device_bytes < i0.device_bytes
    finally:
        p0.close()
        p1.close()


def test_reverse_march_of_a_range_plan_refuses_a_zero_stiffness():
    """The transposed Jacobi solve of a plan without pair lists works on beta-scaled data
    ((I + S)^T r = b through (I + S) y = beta o b, r = y / beta), so its reverse march refuses a
    layout with a zero stiffness even for dL/dg alone; the stored-weight plan of the same layout
    takes it."""
    torch = pytest.importorskip("torch")
    w = W.config0(Nt=20)
    beta = w.beta.copy()
    beta[5] = 0.0
    w = w.with_(beta=beta)
    for lw, want in ((1, wave1d.WAVE1D_EINVAL), (0, wave1d.WAVE1D_OK)):
        plan = wave1d.Plan.from_workload(w, local_weights=lw)
        try:
            sigma, u = plan.solve_device(20)
            gg = torch.empty((20, w.M), dtype=torch.float64, device="cuda")
            st = wave1d.wave1d_adjoint(plan.h, 20, sigma, None, u.contiguous(), None, gg)
            assert st == want
        finally:
            plan.close()
