"""Failure detection without a GPU fault: a non-finite value injected from the host (a NaN in the
forcing vector of one step) makes the step's densities non-finite; the kernels latch
WAVE1D_ENONFINITE in the plan's status word, the next synchronising call reports it, and the
context stays usable (a new plan marches normally afterwards)."""
import numpy as np
import pytest

from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("step_kernel", [1, 0])
def test_nonfinite_forcing_is_latched_and_reported(step_kernel):
    w = W.config0(Nt=10)
    plan = wave1d.Plan.from_workload(w, step_kernel=step_kernel)
    try:
        g = np.zeros(w.M)
        g[3] = np.nan
        assert wave1d.wave1d_step(plan.h, g, 0) == wave1d.WAVE1D_OK      # queued; the fault is on the device
        assert wave1d.wave1d_sync(plan.h) == wave1d.WAVE1D_ENONFINITE
    finally:
        plan.close()
    other = wave1d.Plan.from_workload(w)
    try:
        s, u = other.solve(5)
    finally:
        other.close()
    assert np.all(np.isfinite(s)) and np.all(np.isfinite(u))
