"""Stability diagnostics on the GPU (dirac_check, Props. 2 and 4).

* A stable run with real fields: E stays at its reference (taken when the
  state was set) and the naive norm stays within the bounds E implies.
* Absorbing layers: E falls and the check passes.
* A moving vector potential: E is not conserved, the drift is reported but
  not checked.
* A forced run beyond the stability limit: the check raises the alarm while
  the values are still finite.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def problem(dims, fields, r=0.9, m=0.4):
    N = (40, 34, 1) if dims == 2 else (20, 18, 22)
    return W.Problem(dims, N, (1.0, 1.0, 1.0), r * W.stability_limit(dims), m, fields)


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_check_stable_run(D, dims, precision):
    N = (40, 34) if dims == 2 else (20, 18, 22)
    prob = problem(dims, W.Fields(step_axis=0, step_x0=N[0] / 2 + 0.25, step_V=0.7))
    psi = W.random_state(prob, 12)
    prec, tol = (D.FP64, 1e-12) if precision == "fp64" else (D.FP32, 1e-6)
    E0 = O.observables(prob, psi)["E"]
    with D.Sim(prob, prec) as s:
        s.set_spinor(psi)
        s.step(37)
        ok, r = s.check(tol)
        E, naive = s.norm()
    assert ok, r
    assert r["failed"] == 0
    assert abs(r["E_ref"] - E0) < 1e-12 * E0 if precision == "fp64" else abs(r["E_ref"] - E0) < 1e-6 * E0
    assert abs(r["drift"]) < tol
    assert r["E"] == E and r["naive"] == naive
    lo, hi = D.functional_bounds(dims, prob.dx, prob.dt)
    assert abs(r["lower"] - E / hi) < 1e-14 * E and abs(r["upper"] - E / lo) < 1e-14 * E
    assert r["lower"] <= naive <= r["upper"]


@pytest.mark.parametrize("dims", [2, 3])
def test_check_absorbing_layers(D, dims):
    prob = problem(dims, W.Fields(abs_W=0.8, abs_width=5.0, abs_axes=(1 << dims) - 1))
    psi = W.random_state(prob, 13)
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(30)
        ok, r = s.check(1e-6)
    assert ok, r
    assert r["drift"] < -0.05  # absorbed


def test_check_moving_vector_potential(D):
    f = W.Fields(q=1.0, Apw_amp=0.5, Apw_k=(0.0, 0.0, 2 * math.pi / 22), Apw_omega=0.6, Apw_pol=0)
    prob = problem(3, f)
    psi = W.random_state(prob, 14)
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(25)
        ok, r = s.check(1e-9)
    assert ok, r
    assert abs(r["drift"]) > 1e-9  # not conserved, and not checked
    assert r["lower"] == 0.0 and r["upper"] == math.inf  # r_x + r_y + r_z > 1: no bound


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_check_alarm_beyond_the_stability_limit(D, precision):
    prob = problem(3, W.Fields(), r=1.2, m=0.0)
    psi = W.random_state(prob, 15)
    prec = D.FP64 if precision == "fp64" else D.FP32
    alarm = None
    with D.Sim(prob, prec, flags=D.FLAG_ALLOW_UNSTABLE) as s:
        s.set_spinor(psi)
        for _ in range(100):
            s.step(10)
            ok, r = s.check(1e-6)
            if not ok:
                alarm = r
                break
    assert alarm is not None
    assert alarm["failed"] & D.CHECK_DRIFT
    assert math.isfinite(alarm["E"]) and math.isfinite(alarm["naive"])  # raised before overflow
    assert alarm["naive"] > 10 * alarm["naive_ref"]
