"""The torch.autograd wrapper of the reverse-time march (`wave1d.receiver_fields`) on the CPU: a
stand-in plan answers `solve_device` with the discrete scheme's oracle march and `adjoint` with the
adjoint oracle, so the wrapper's own logic is what is tested.  That logic is the plan built from the
stiffnesses, the receiver fields returned, dL/du handed to the adjoint, the gradient returned for
beta, and the plan closed after the backward pass.  The GPU form of the same test is in
tests/test_gpu_adjoint.py."""
import numpy as np
import pytest

from oracle import adjoint, wfp
from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

torch = pytest.importorskip("torch")


class _OraclePlan:
    closed = []

    def __init__(self, x, beta, bc, dt, Nt, tol, amp, center, width, xr, p):
        self.w = W.Workload(name="stand-in", bc=bc, x=np.asarray(x), beta=np.asarray(beta), amp=np.asarray(amp),
                            center=np.asarray(center), width=np.asarray(width), dt=dt, Nt=Nt, tol=tol, p=p,
                            xr=np.asarray(xr), seed=0)
        self.h = object()

    def solve_device(self, nsteps):
        sigma, u = wfp.from_workload(self.w).run(nsteps)
        self.nsteps, self.u = nsteps, u
        return torch.from_numpy(sigma[1:].copy()), torch.from_numpy(u[1:].copy())

    def adjoint(self, sigma, ubar):
        # targets that make the oracle's residual u - d equal to ubar
        d = self.u.copy()
        d[1:] -= ubar.detach().numpy()
        _, g = adjoint.misfit_and_gradient(wfp.from_workload(self.w), self.nsteps, d)
        return torch.from_numpy(g)

    def close(self):
        _OraclePlan.closed.append(self)


def test_receiver_fields_gradient_and_plan_lifetime(monkeypatch):
    monkeypatch.setattr(wave1d, "Plan", _OraclePlan)
    rng = np.random.default_rng(3)
    M = 6
    x = np.sort(rng.uniform(-0.8, 0.8, M))
    w = W.Workload(name="wrapper", bc=W.FREE, x=x, beta=rng.uniform(1.0, 6.0, M), amp=np.array([1.0]),
                   center=np.array([-1.6]), width=np.array([0.12]), dt=0.02, Nt=200, tol=1e-10, p=6,
                   xr=np.array([-0.9, 0.3, 0.9]), seed=3)
    t = np.arange(w.Nt + 1)[:, None] * w.dt
    d = 0.3 * np.sin(3.0 * t + w.xr[None, :])
    beta = torch.tensor(w.beta, dtype=torch.float64, requires_grad=True)
    u = wave1d.receiver_fields(beta, w, w.Nt)
    assert u.shape == (w.Nt, 3)
    loss = 0.5 * torch.sum((u - torch.from_numpy(d[1:])) ** 2)
    _OraclePlan.closed.clear()
    loss.backward()
    assert len(_OraclePlan.closed) == 1
    L, g = adjoint.misfit_and_gradient(wfp.from_workload(w), w.Nt, d)
    assert abs(loss.item() - L) <= 1e-12 * L
    assert np.max(np.abs(beta.grad.numpy() - g)) <= 1e-12 * np.max(np.abs(g))
