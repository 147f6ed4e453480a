"""Launch plans and the autotuner.

* A plan (levels per work item; one or two time steps per pass in (2+1)D)
  only changes how the work of a step is cut: every plan must give the same
  state bit for bit, and the functional fused into the last step may only
  differ by the FP32 summation order.
* dirac_autotune times the candidates on the simulation's own state: the
  state and the time are unchanged afterwards, the kept plan is one of the
  candidates, and a later simulation of the same grid and field path starts
  with it.
* dirac_set_plan rejects plans the kernels cannot run.
"""
import numpy as np
import pytest

from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def run(D, prob, psi, plan, n):
    with D.Sim(prob, D.FP32) as s:
        if plan is not None:
            s.set_plan(**plan)
        s.set_spinor(psi)
        s.step(n)
        E, _ = s.norm()
        return s.get_spinor(), E


def test_plans_give_identical_states_3d(D):
    prob = W.Problem(3, (40, 36, 45), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.7,
                     W.Fields(step_axis=0, step_x0=20.25, step_V=0.8))
    psi = W.random_state(prob, 5)
    ref, E0 = run(D, prob, psi, None, 21)
    for chunk in (1, 2, 4, 7, 16, 44, 45):
        got, E = run(D, prob, psi, {"chunk": chunk}, 21)
        assert np.array_equal(got, ref), chunk
        assert abs(E - E0) <= 1e-6 * abs(E0), chunk


def test_plans_give_identical_states_2d(D):
    prob = W.Problem(2, (130, 97, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.3,
                     W.Fields(step_axis=0, step_x0=60.25, step_V=0.9))
    psi = W.random_state(prob, 6)
    ref, E0 = run(D, prob, psi, None, 20)  # default: two steps per pass
    plans = [{"two_step": 0}, {"two_step": 0, "chunk": 1}, {"two_step": 0, "chunk": 16},
             {"two_step": 0, "chunk": 97}, {"two_step": 1, "chunk2": 1}, {"two_step": 1, "chunk2": 5},
             {"two_step": 1, "chunk2": 96, "chunk": 3}]
    for plan in plans:
        got, E = run(D, prob, psi, plan, 20)
        assert np.array_equal(got, ref), plan
        assert abs(E - E0) <= 1e-6 * abs(E0), plan


@pytest.mark.parametrize("dims", [2, 3])
def test_autotune_keeps_state_and_is_remembered(D, dims):
    if dims == 3:
        prob = W.Problem(3, (64, 48, 40), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 1.0)
    else:
        prob = W.Problem(2, (512, 300, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.2)
    psi = W.random_state(prob, 7)
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(3)
        before, t_before = s.get_spinor(), s.time
        E_before, _ = s.norm()
        plan = s.autotune()
        assert np.array_equal(s.get_spinor(), before)
        assert s.time == t_before
        assert s.norm()[0] == E_before
        assert plan == s.plan
        extent = prob.N[2] if dims == 3 else prob.N[1]
        assert 1 <= plan["chunk"] <= extent
        assert plan["us_per_step"] > 0.0
        if dims == 2:
            assert plan["two_step"] in (0, 1) and 1 <= plan["chunk2"] <= extent
        s.step(5)
        tuned = s.get_spinor()
    with D.Sim(prob, D.FP32) as s2:  # created after the tuning: starts with the same plan
        assert s2.plan == plan
        s2.set_spinor(psi)
        s2.step(8)
        assert np.array_equal(s2.get_spinor(), tuned)


def test_set_plan_validation(D):
    prob3 = W.Problem(3, (20, 20, 12), (1.0, 1.0, 1.0), 0.5, 0.1)
    prob2 = W.Problem(2, (40, 30, 1), (1.0, 1.0, 1.0), 0.5, 0.1)
    with D.Sim(prob3, D.FP32) as s:
        for bad in ({"chunk": -1}, {"chunk": 13}, {"two_step": 1}, {"chunk2": 4}):
            with pytest.raises(D.DiracError):
                s.set_plan(**bad)
        s.set_plan(chunk=12)
        assert s.plan["chunk"] == 12
    with D.Sim(prob2, D.FP32) as s:
        for bad in ({"two_step": 2}, {"chunk2": 31}, {"chunk": 31}):
            with pytest.raises(D.DiracError):
                s.set_plan(**bad)
    with D.Sim(prob3, D.FP64) as s:  # no fused kernels: only the zero plan
        assert s.plan == {"chunk": 0, "two_step": 0, "chunk2": 0, "us_per_step": 0.0}
        assert s.autotune()["chunk"] == 0
        with pytest.raises(D.DiracError):
            s.set_plan(chunk=4)
