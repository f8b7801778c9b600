"""Without a GPU, the batched plan and the mixed-precision plan must get through every host step
(argument marshalling, each instance's tables, the join, the precision checks) and stop only at the
device: WAVE1D_ECUDA "no CUDA device".  A marshalling or host-table fault would surface as another
status first.  Skipped where a GPU is present (the GPU tests cover those plans there)."""
import pytest

from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="a GPU is present: the GPU tests cover these plans")


def test_batched_plan_host_side_reaches_the_device_step():
    ws = [W.make(f"b{i}", M=M, bc=W.PERIODIC, dt=0.01, Nt=300, tol=1e-10, p=8, seed=100 + i, amp=(1.0,),
                 center=(-2.0,), width=(0.08 + 0.02 * i,), R=2) for i, M in enumerate((1, 5, 40, 200))]
    with pytest.raises(wave1d.Wave1DError) as e:
        wave1d.Batch(ws)
    assert e.value.status == wave1d.WAVE1D_ECUDA and "no CUDA device" in str(e.value)


def test_mixed_plan_host_side_reaches_the_device_step():
    with pytest.raises(wave1d.Wave1DError) as e:
        wave1d.Plan.from_workload(W.config0(Nt=10), precision=1)
    assert e.value.status == wave1d.WAVE1D_ECUDA
