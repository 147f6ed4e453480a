"""Stability estimates of the functional (Props. 2 and 4), host side.

dirac_functional_bounds gives lo, hi with lo sum|psi|^2 <= E <= hi sum|psi|^2.
Here the Hermitian form of E is built from the oracle's functional (by
polarisation on tiny grids) and its spectrum compared with those constants:

* without a vector potential the spectrum is exactly [1 - rho, 1 + rho],
  rho = sqrt(sum_a r_a^2), both ends attained at the zone corner;
* a constant (pure gauge) vector potential keeps it inside;
* a non-uniform one can leave [1 - rho, 1 + rho] but stays inside the
  paper's [1 - sum_a r_a, 1 + sum_a r_a] (Prop. 2 / Prop. 4), which the
  library then uses;
* beyond the stability limit lo < 0 and the form is indefinite.
No GPU is needed: the bounds are host code of the library.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W


@pytest.fixture(scope="module")
def D():
    from paper_1309_3452_gb300 import build as B
    B.build()  # host code only: loads without a GPU
    from paper_1309_3452_gb300 import dirac
    return dirac


def functional_form(prob):
    n = int(np.prod(prob.shape))
    eye = np.eye(n)
    Ed = [O.observables(prob, eye[i].reshape(prob.shape))["E"] for i in range(n)]
    M = np.diag(np.array(Ed, complex))
    for i in range(n):
        for j in range(i + 1, n):
            a = O.observables(prob, (eye[i] + eye[j]).reshape(prob.shape))["E"] - Ed[i] - Ed[j]
            b = O.observables(prob, (eye[i] + 1j * eye[j]).reshape(prob.shape))["E"] - Ed[i] - Ed[j]
            M[i, j] = 0.5 * (a - 1j * b)
            M[j, i] = np.conj(M[i, j])
    return np.linalg.eigvalsh(M)


CASES = [(3, (2, 2, 2), (1.0, 1.0, 1.0), 0.4), (3, (2, 2, 2), (1.0, 1.3, 0.8), 0.35),
         (2, (4, 4, 1), (1.0, 1.0, 1.0), 0.5), (2, (4, 2, 1), (1.0, 1.4, 1.0), 0.5)]


@pytest.mark.parametrize("dims,N,dx,dt", CASES)
def test_sharp_bounds_without_vector_potential(D, dims, N, dx, dt):
    prob = W.Problem(dims, N, dx, dt, 0.3, W.Fields(V_static=None))
    prob = prob.with_fields(V_static=W.random_potential(prob, 3, 0.7))  # V does not enter E
    ev = functional_form(prob)
    lo, hi = D.functional_bounds(dims, dx, dt, False)
    rho = math.sqrt(sum((dt / dx[a]) ** 2 for a in range(dims)))
    assert abs(lo - (1 - rho)) < 1e-15 and abs(hi - (1 + rho)) < 1e-15
    assert abs(ev.min() - lo) < 1e-12 and abs(ev.max() - hi) < 1e-12


@pytest.mark.parametrize("dims,N,dx,dt", CASES)
def test_bounds_with_vector_potentials(D, dims, N, dx, dt):
    base = W.Problem(dims, N, dx, dt, 0.3)
    lo, hi = D.functional_bounds(dims, dx, dt, False)
    ev = functional_form(base.with_fields(q=1.0, A_const=(0.3, -0.2, 0.1)))
    assert ev.min() >= lo - 1e-12 and ev.max() <= hi + 1e-12
    # a plane wave (a magnetic field): the paper's coarser constants hold
    wave = base.with_fields(q=1.0, Apw_amp=0.7, Apw_k=(0.0, 2 * math.pi / (N[1] * dx[1]), 0.0), Apw_pol=0)
    ev = functional_form(wave)
    glo, ghi = D.functional_bounds(dims, dx, dt, True)
    assert abs(glo - (1 - sum(dt / dx[a] for a in range(dims)))) < 1e-15
    assert ev.min() >= glo - 1e-12 and ev.max() <= ghi + 1e-12


def test_plane_wave_vector_potential_can_break_the_sharp_bound(D):
    """Why the library falls back to the paper's constants with a
    non-uniform vector potential."""
    dims, N, dx, dt = 3, (2, 2, 2), (1.0, 1.0, 1.0), 0.4
    lo, _ = D.functional_bounds(dims, dx, dt, False)
    wave = W.Problem(dims, N, dx, dt, 0.3).with_fields(q=1.0, Apw_amp=0.7, Apw_k=(0.0, math.pi, 0.0),
                                                       Apw_pol=0)
    assert functional_form(wave).min() < lo - 1e-3


@pytest.mark.parametrize("dims", [2, 3])
def test_beyond_the_stability_limit(D, dims):
    dt = 1.08 * W.stability_limit(dims)
    lo, _ = D.functional_bounds(dims, (1.0, 1.0, 1.0), dt, False)
    assert lo < 0.0
    N = (2, 2, 2) if dims == 3 else (4, 4, 1)
    assert functional_form(W.Problem(dims, N, (1.0, 1.0, 1.0), dt, 0.0)).min() < 0.0
