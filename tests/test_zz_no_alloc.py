"""wave1d_nufft1_noalloc: the type-1 NUFFT for callers that cannot allocate device memory.

On two calls in a row it must give the direct sums S_k = (1/2 pi) sum_j c_j e^{i k x_j} of the
oracle (eq. densco) within the parity tolerance, and the spectrum S_k a plan computes inside a step
(the spreading + FFT stages, read back with wave1d_inspect) for the same densities.  Collected last
so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from oracle import wfp
from paper_2507_07823_gb300 import build, wave1d, workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wave1d.lib()
    return t


@pytest.mark.parametrize("cfg", ["periodic_small", "free_1e4"])
def test_noalloc_type1_matches_plan(torch, cfg):
    if cfg == "periodic_small":
        w = W.config0(Nt=400)
        n = 300
    else:
        w = W.config1(Nt=2000)
        n = 1200
    plan = wave1d.Plan.from_workload(w)
    plan.solve(n, with_sigma=False)
    ring = plan.inspect(wave1d.WAVE1D_ARR_SIGMA_RING)        # ring[m] = sigma^{n-m}, caller order
    S_prev = plan.inspect(wave1d.WAVE1D_ARR_S_LAST)          # S^{n-1}, from sigma^{n-1}
    K = plan.info.K
    dev = torch.device("cuda")
    x = torch.tensor(w.x, dtype=torch.float64, device=dev)
    c1 = torch.tensor(ring[1], dtype=torch.float64, device=dev)
    c0 = torch.tensor(ring[0], dtype=torch.float64, device=dev)
    out1 = torch.zeros(2 * (K + 1), dtype=torch.float64, device=dev)
    out2 = torch.zeros(2 * (K + 1), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, the second must not see the first call's intermediates
    assert wave1d.wave1d_nufft1_noalloc(x, c1, w.M, K, w.tol, out1, stream) == 0
    assert wave1d.wave1d_nufft1_noalloc(x, c0, w.M, K, w.tol, out2, stream) == 0
    torch.cuda.synchronize()
    plan.step()
    S_now = plan.inspect(wave1d.WAVE1D_ARR_S_LAST)           # S^n, from sigma^n
    plan.close()
    a1 = out1.cpu().numpy()
    a2 = out2.cpu().numpy()
    r1 = a1[0::2] + 1j * a1[1::2]
    r2 = a2[0::2] + 1j * a2[1::2]
    assert np.max(np.abs(S_prev)) > 0 and np.max(np.abs(S_now)) > 0
    # the oracle's direct sums of the same densities
    d1 = wfp.type1(ring[1], w.x, K)
    d2 = wfp.type1(ring[0], w.x, K)
    assert np.max(np.abs(r1 - d1)) <= TOL * np.max(np.abs(d1))
    assert np.max(np.abs(r2 - d2)) <= TOL * np.max(np.abs(d2))
    # and the plan's own spectrum of them
    assert np.max(np.abs(r1 - S_prev)) <= TOL * np.max(np.abs(S_prev))
    assert np.max(np.abs(r2 - S_now)) <= TOL * np.max(np.abs(S_now))


def test_noalloc_rejects_oversize(torch):
    dev = torch.device("cuda")
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    c = torch.zeros(4, dtype=torch.float64, device=dev)
    K = 20000                                                 # fine grid 131072 > 65536
    S = torch.zeros(2 * (K + 1), dtype=torch.float64, device=dev)
    assert wave1d.wave1d_nufft1_noalloc(x, c, 4, K, 1e-10, S) == wave1d.WAVE1D_EUNSUPPORTED
    assert wave1d.wave1d_nufft1_noalloc(x, c, 4, 0, 1e-10, S) == wave1d.WAVE1D_EINVAL
