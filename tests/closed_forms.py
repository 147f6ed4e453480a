"""Closed forms the paper fixes, restated for the tests (not used by the oracle
or the library).

* Lattice plane waves (Sect. 2.1, Eqs. planeonlattice, substE, substp, substm,
  pwdsip): a value c at position x and time sheet t equals a_c exp(i(k.x - w t)),
  where a is the continuum free spinor with E -> (2/dt) sin(w dt/2),
  p_j -> (2/dx_j) sin(k_j dx_j/2), m -> m cos(w dt/2), and
  w = (2/dt) arcsin X,  X^2 = (m^2 + |P|^2) / (m^2 + (2/dt)^2).
  The (2+1)D relation (Sect. 3) is the same X with two momentum components
  (its printed denominator "(mc^2)^2 + 2 hbar c/dt" is read as
  (mc^2)^2 + (2 hbar/dt)^2, the (3+1)D expression).
* Eigenspinors psi^(1) (Sect. 2.1) and, for two components, (E+m, P_x+iP_y).
"""
import math

import numpy as np

from paper_1309_3452_gb300 import workloads as W


def lattice_P(k, dx, dims):
    return [2.0 / dx[a] * math.sin(k[a] * dx[a] / 2.0) for a in range(dims)]


def lattice_omega(k, dx, dt, m, dims):
    P = lattice_P(k, dx, dims)
    X2 = (m * m + sum(p * p for p in P)) / (m * m + (2.0 / dt) ** 2)
    return 2.0 / dt * math.asin(math.sqrt(X2))


def lattice_spinor(k, dx, dt, m, dims, positive=True):
    P = lattice_P(k, dx, dims) + [0.0] * (3 - dims)
    w = lattice_omega(k, dx, dt, m, dims)
    X = math.sin(w * dt / 2.0)
    Ew = 2.0 / dt * X
    mw = m * math.sqrt(max(0.0, 1.0 - X * X))
    if not positive:
        Ew = -Ew
    if dims == 3:
        if positive:
            a = np.array([1.0, 0.0, P[2] / (Ew + mw), (P[0] + 1j * P[1]) / (Ew + mw)], complex)
        else:  # psi^(3) of Sect. 2.1
            a = np.array([-P[2] / (abs(Ew) + mw), -(P[0] + 1j * P[1]) / (abs(Ew) + mw), 1.0, 0.0],
                         complex)
    else:
        if positive:
            a = np.array([Ew + mw, P[0] + 1j * P[1]], complex)
        else:
            a = np.array([-(P[0] - 1j * P[1]), abs(Ew) + mw], complex)
    return a / np.linalg.norm(a), (w if positive else -w)


def plane_wave_state(prob, n_modes, positive=True):
    """Lattice plane wave with k_a = 2 pi n_a / (N_a dx_a) at t = 0."""
    dims = prob.dims
    k = [2.0 * math.pi * n_modes[a] / (prob.N[a] * prob.dx[a]) for a in range(dims)]
    a, w = lattice_spinor(k + [0.0] * (3 - dims), prob.dx, prob.dt, prob.m, dims, positive)
    _, _, _, comp = W.plane_tables(dims)
    out = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        xyz = W.site_positions(prob, pl)
        ph = sum(k[d] * xyz[d] for d in range(dims))
        out[pl] = a[comp[pl]] * np.exp(1j * (ph - w * W.sheet_time(prob, pl, 0.0)))
    return out, w


def reduced_spectrum(prob):
    """Closed-form eigen-phases of the one-step map on a periodic grid:
    -+ w(k) dt for every reduced k, each with multiplicity 2 ((2+1)D) or
    4 ((3+1)D), the second copy being k + 2 pi/dx_x e_x (P_x -> -P_x)."""
    dims = prob.dims
    mult = 2 if dims == 2 else 4
    phases = []
    grids = [range(prob.N[a]) for a in range(dims)]
    for idx in np.ndindex(*[prob.N[a] for a in range(dims)]):
        k = [2.0 * math.pi * idx[a] / (prob.N[a] * prob.dx[a]) for a in range(dims)]
        w = lattice_omega(k + [0.0] * (3 - dims), prob.dx, prob.dt, prob.m, dims)
        phases += [w * prob.dt] * mult + [-w * prob.dt] * mult
    del grids
    return np.array(phases)
