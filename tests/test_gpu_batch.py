"""Batched march (wave1d_batch_plan): independent periodic instances of uneven size, each with its own
incident Gaussian and receivers, advanced together.  Each instance's densities and receiver fields
against its own one-instance plan (the same scheme; the history part's spreading runs through the
batched NUFFT instead of the step's spreading matrix, so agreement is to rounding) and against the
discrete scheme's oracle at 1e-9; bit for bit from run to run."""
import numpy as np
import pytest

from oracle import wfp
from paper_2507_07823_gb300 import wave1d
from paper_2507_07823_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances():
    ws = []
    for i, M in enumerate((1, 5, 40, 200, 17, 90)):
        ws.append(W.make(f"b{i}", M=M, bc=W.PERIODIC, dt=0.01, Nt=300, tol=1e-10, p=8, seed=100 + i,
                         amp=(1.0,), center=(-2.0,), width=(0.08 + 0.02 * i,), R=2))
    return ws


def _rel(a, b):
    # relative to the reference's size, floored at 1e-20: an instance the pulse never reaches carries
    # only Gaussian tails below e^-72 of the amplitude, which the library's forcing cuts to zero
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-20))


def test_each_instance_matches_its_own_plan_and_the_oracle():
    ws = _instances()
    batch = wave1d.Batch(ws)
    try:
        s, u = batch.solve(300)
    finally:
        batch.close()
    for i, w in enumerate(ws):
        sb = s[:, batch.offsets[i]:batch.offsets[i + 1]]
        ub = u[:, batch.r_offsets[i]:batch.r_offsets[i + 1]]
        plan = wave1d.Plan.from_workload(w)
        try:
            s1, u1 = plan.solve(300)
        finally:
            plan.close()
        assert _rel(sb, s1) < 1e-12 and _rel(ub, u1) < 1e-12, i
        s_ref, u_ref = wfp.from_workload(w).run(300)
        assert _rel(sb, s_ref[1:]) < 1e-9 and _rel(ub, u_ref[1:]) < 1e-9, i


def test_batched_march_is_bitwise_reproducible():
    ws = _instances()
    out = []
    for _ in range(2):
        batch = wave1d.Batch(ws)
        try:
            out.append(batch.solve(120))
        finally:
            batch.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_one_launch_step_equals_the_per_pass_launches():
    """The batched step as one cooperative launch (opts.step_kernel = 1, the default) against the
    same step as one launch per pass (step_kernel = 0): the same unit bodies in the same order, so
    the densities and receiver fields agree bit for bit; also a larger instance (M = 3000, its
    implicit blocks up to dozens of springs) among small ones."""
    ws = _instances() + [W.make("big", M=3000, bc=W.PERIODIC, dt=0.01, Nt=300, tol=1e-10, p=8, seed=7,
                                amp=(1.0,), center=(-2.0,), width=(0.1,), R=3)]
    out = []
    for sk in (1, 0):
        batch = wave1d.Batch(ws, step_kernel=sk)
        try:
            assert batch.one_launch == bool(sk)
            out.append(batch.solve(120))
        finally:
            batch.close()
    (s1, u1), (s0, u0) = out
    assert np.max(np.abs(s0)) > 1e-3
    assert np.array_equal(s1, s0) and np.array_equal(u1, u0)


def _dense(name, M, seed):
    return W.make(name, M=M, bc=W.PERIODIC, dt=0.01, Nt=300, tol=1e-10, p=8, seed=seed, amp=(1.0,),
                  center=(-2.0,), width=(0.1,), R=3)


def _own_plan(w, n, lw):
    plan = wave1d.Plan.from_workload(w, local_weights=lw)
    try:
        return plan.solve(n)
    finally:
        plan.close()


def test_instances_chosen_without_pair_lists_equal_their_own_plans():
    """local_weights = 2: an instance whose largest block of springs closer than dt passes
    opts.max_block (two dense ones, M = 3000 and 2000, about five springs per dt) is marched as its
    own plan without pair lists, a branch of the step graph beside the joined instances' one
    launch; its densities and receiver fields equal that plan's own march bit for bit (the same
    kernels in the same order), and the joined instances keep their one-instance agreement."""
    ws = _instances()
    ws = ws[:3] + [_dense("dense0", 3000, 7)] + ws[3:] + [_dense("dense1", 2000, 8)]
    batch = wave1d.Batch(ws, local_weights=2, max_block=64)
    try:
        forms = batch.forms
        assert list(forms) == [0, 0, 0, 1, 0, 0, 0, 1]
        assert batch.one_launch
        s, u = batch.solve(200)
    finally:
        batch.close()
    assert np.max(np.abs(s[:, batch.offsets[3]:batch.offsets[4]])) > 1e-3
    for i, w in enumerate(ws):
        sb = s[:, batch.offsets[i]:batch.offsets[i + 1]]
        ub = u[:, batch.r_offsets[i]:batch.r_offsets[i + 1]]
        s1, u1 = _own_plan(w, 200, int(forms[i]))
        if forms[i]:
            assert np.array_equal(sb, s1) and np.array_equal(ub, u1), i
        else:
            assert _rel(sb, s1) < 1e-12 and _rel(ub, u1) < 1e-12, i


def test_every_instance_without_pair_lists():
    """local_weights = 1: every instance its own plan without pair lists, all of them branches of
    one step graph; each equals its own march bit for bit, the smallest ones also the oracle at
    1e-9, and the batch is reproducible from run to run."""
    ws = _instances()[1:4] + [_dense("dense", 1500, 9)]
    out = []
    for _ in range(2):
        batch = wave1d.Batch(ws, local_weights=1)
        try:
            assert list(batch.forms) == [1] * len(ws) and not batch.one_launch
            out.append(batch.solve(150))
            offs, roffs = batch.offsets, batch.r_offsets
        finally:
            batch.close()
    (s, u), (s2, u2) = out
    assert np.array_equal(s, s2) and np.array_equal(u, u2)
    for i, w in enumerate(ws):
        sb, ub = s[:, offs[i]:offs[i + 1]], u[:, roffs[i]:roffs[i + 1]]
        s1, u1 = _own_plan(w, 150, 1)
        assert np.array_equal(sb, s1) and np.array_equal(ub, u1), i
        if w.M <= 200:
            s_ref, u_ref = wfp.from_workload(w).run(150)
            assert _rel(sb, s_ref[1:]) < 1e-9 and _rel(ub, u_ref[1:]) < 1e-9, i


def test_instances_over_the_weight_budget_go_without_pair_lists():
    """local_weights = 2 with opts.max_local_bytes too small for the larger instances' stored
    weights: an instance whose weights would pass what is left of the budget is planned without
    pair lists instead of failing the plan, and still equals its own plan bit for bit."""
    ws = _instances()
    batch = wave1d.Batch(ws, local_weights=2, max_local_bytes=200_000)
    try:
        forms = batch.forms
        assert forms[0] == 0 and forms.sum() >= 1, forms
        s, u = batch.solve(200)
    finally:
        batch.close()
    for i, w in enumerate(ws):
        sb = s[:, batch.offsets[i]:batch.offsets[i + 1]]
        ub = u[:, batch.r_offsets[i]:batch.r_offsets[i + 1]]
        s1, u1 = _own_plan(w, 200, int(forms[i]))
        if forms[i]:
            assert np.array_equal(sb, s1) and np.array_equal(ub, u1), i
        else:
            assert _rel(sb, s1) < 1e-12 and _rel(ub, u1) < 1e-12, i
