"""Failure detection without a GPU fault.

* A non-finite value injected from the host (a NaN in the forcing vector of one step) makes the
  step's densities non-finite; the kernels latch WAVE1D_ENONFINITE in the plan's status word, the
  next synchronising call reports it, and the context stays usable (a new plan marches normally
  afterwards).
* A bounded wait of the one-launch step kernel runs out: the plan is opened with a short poll limit
  and the test hook that leaves the column pass's first unit uncounted, so the row pass's wait can
  never be met.  The waiting block latches WAVE1D_ETIMEOUT and returns, every other block gives up
  at its next wait, the kernel ends, the next synchronising call reports the status, and the context
  stays usable.  No wait in the kernel is unbounded."""
import time

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


def test_step_kernel_wait_runs_out_and_is_reported():
    w = W.config0(Nt=10)
    plan = wave1d.Plan.from_workload(w, spin_limit=2000, hold_unit=1)
    try:
        t0 = time.time()
        assert wave1d.wave1d_step(plan.h, None, 0) == wave1d.WAVE1D_OK      # queued
        assert wave1d.wave1d_sync(plan.h) == wave1d.WAVE1D_ETIMEOUT
        assert time.time() - t0 < 30.0
    finally:
        plan.close()
    other = wave1d.Plan.from_workload(w)
    try:
        s, u = other.solve(5)
    finally:
        other.close()
    assert np.all(np.isfinite(s)) and np.all(np.isfinite(u))
