"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  A plausible mistake in the oracle (a
sign of the y or z coupling, a wrong neighbour, a mass on the wrong
component, the time-average on the wrong term, a link phase of the wrong sign
or place) fails at least one of them:

* conservation of the functional E (Lemma, Sect. 2 Eq. EPM; Lemma, Sect. 3)
  holds only for the Hermitian sign pattern of the scheme;
* a lattice plane wave advances by exactly the phase of Eq. pwdsip;
* the full spectrum of the one-step map equals the closed form (single cone);
* stability below/above r_max (Sect. 2.2, Sect. 3);
* the light cone of the nearest-neighbour stencil (Eq. 3+3Ddis);
* the (3+1)D -> (2+1)D reduction (Sect. 3, opening paragraph);
* gauge covariance of the Peierls substitution (Sect. 4).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W
from tests import closed_forms as CF


def prob2(N=(12, 10), r=0.9, m=0.3, dx=(1.0, 1.0)):
    dt = r * W.stability_limit(2) * min(dx)
    return W.Problem(2, (N[0], N[1], 1), (dx[0], dx[1], 1.0), dt, m)


def prob3(N=(6, 5, 7), r=0.9, m=0.7, dx=(1.0, 1.0, 1.0)):
    dt = r * W.stability_limit(3) * min(dx)
    return W.Problem(3, tuple(N), tuple(dx), dt, m)


def rel_drift(prob, psi0, nsteps, t0=0.0):
    e0 = O.observables(prob, psi0, t0)
    psi = O.step(prob, psi0, nsteps, t0)
    e1 = O.observables(prob, psi, t0 + nsteps * prob.dt)
    return (e1["E"] - e0["E"]) / e0["E"], e0, e1, psi


# ---------------------------------------------------------------- T1
@pytest.mark.parametrize("dims", [2, 3])
def test_conservation_random_static_potential(dims):
    """Lemma of Sect. 2 (Eq. EPM) and of Sect. 3: E is conserved exactly for
    arbitrary real V(x); the naive norm is not (Sect. 3)."""
    prob = prob2() if dims == 2 else prob3()
    prob = prob.with_fields(V_static=W.random_potential(prob, 11, 0.8))
    psi0 = W.random_state(prob, 5)
    d, e0, e1, _ = rel_drift(prob, psi0, 400 if dims == 2 else 200)
    assert abs(d) < 2e-14
    # the naive norm oscillates (not conserved), as the paper states
    assert abs(e1["naive"] - e0["naive"]) > 1e-3
    # upper and lower forms agree for static fields (summation by parts)
    assert abs(e1["E"] - e1["E_upper"]) < 1e-13


@pytest.mark.parametrize("dims", [2, 3])
def test_conservation_time_dependent_potential_and_anisotropic_grid(dims):
    """E is conserved for space- and time-dependent V (Prop. 3 / Prop. 5 hold
    'for arbitrary space- and time-dependent mass and potential'), with
    r_x != r_y != r_z."""
    if dims == 2:
        dx = (1.0, 1.3)
        prob = W.Problem(2, (10, 9, 1), (1.0, 1.3, 1.0), 0.5, 0.4)
    else:
        dx = (1.0, 1.2, 0.9)
        prob = W.Problem(3, (5, 6, 4), dx, 0.45, 0.4)
    r2 = sum((prob.dt / prob.dx[a]) ** 2 for a in range(dims))
    assert r2 < 1.0
    prob = prob.with_fields(V_static=W.random_potential(prob, 3, 1.0), Vmod_amp=0.7,
                            Vmod_omega=1.3, V0=0.2, step_axis=0, step_x0=2.6, step_V=0.9,
                            sc_Z=0.5, sc_a=1.0, sc_center=(2.0, 3.0, 1.5))
    psi0 = W.random_state(prob, 9)
    d, _, _, _ = rel_drift(prob, psi0, 300, t0=0.37)
    assert abs(d) < 2e-14


@pytest.mark.parametrize("dims,kaxis", [(2, 1), (3, 2), (2, 0), (3, 0)])
def test_conservation_static_vector_potential(dims, kaxis):
    """Sect. 4: the Peierls-substituted scheme keeps the norm: E (with link
    factors) is conserved for a static vector potential, constant or a
    static (omega = 0) plane wave that is periodic on the box.  With k along
    the polarisation the link factor varies along its own link, so only a
    phase taken at the same point from both ends (the link midpoint) keeps
    the hopping Hermitian."""
    prob = prob2(N=(8, 8)) if dims == 2 else prob3(N=(4, 6, 8))
    L = [prob.N[a] * prob.dx[a] for a in range(dims)]
    k = [0.0, 0.0, 0.0]
    k[kaxis] = 2 * math.pi / L[kaxis]
    prob = prob.with_fields(A_const=(0.31, -0.2, 0.15), Apw_amp=0.6, Apw_k=tuple(k),
                            Apw_omega=0.0, Apw_phase=0.4, Apw_pol=0,
                            V_static=W.random_potential(prob, 2, 0.5))
    psi0 = W.random_state(prob, 4)
    d, e0, e1, _ = rel_drift(prob, psi0, 300)
    assert abs(d) < 2e-14
    assert abs(e1["E"] - e1["E_upper"]) < 1e-13


def _paper_2d_cross(prob, psi, sign):
    """r Re sum_v conj(v) (delta_x u + sign*i delta_y u), restated on the
    canonical planes (u0,u1,v0,v1) of Sect. 3: v0 at (j+1/2, j) has x
    neighbours u0[j+1], u0[j] and y neighbours u1[j], u1[j-1]; v1 at
    (j, j+1/2) has x neighbours u1[j], u1[j-1] and y neighbours u0[j+1], u0[j]."""
    u0, u1, v0, v1 = (psi[i, 0] for i in range(4))
    r = prob.dt / prob.dx[0]
    sx = lambda a: np.roll(a, -1, axis=1)  # a[j+1] along x
    sy = lambda a: np.roll(a, -1, axis=0)
    mx = lambda a: np.roll(a, 1, axis=1)   # a[j-1] along x
    my = lambda a: np.roll(a, 1, axis=0)
    d0 = (sx(u0) - u0) + sign * 1j * (u1 - my(u1))
    d1 = (u1 - mx(u1)) + sign * 1j * (sy(u0) - u0)
    return r * np.real(np.sum(np.conj(v0) * d0) + np.sum(np.conj(v1) * d1))


def test_2d_functional_sign_reading():
    """Sect. 3 Lemma prints the cross term with delta_- u; the scheme as
    printed (Eqs. scheme2ndline, scheme4thline) updates v with
    delta_x u + i delta_y u = delta_+ u, and only the delta_+ form is
    conserved.  The oracle's E equals the delta_+ form."""
    prob = W.Problem(2, (10, 10, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.2)
    psi0 = W.random_state(prob, 21)
    psi1 = O.step(prob, psi0, 150)
    naive = lambda s: float(np.sum(np.abs(s) ** 2))
    Ep = [naive(s) + _paper_2d_cross(prob, s, +1) for s in (psi0, psi1)]
    Em = [naive(s) + _paper_2d_cross(prob, s, -1) for s in (psi0, psi1)]
    assert abs(Ep[1] - Ep[0]) / Ep[0] < 1e-13
    assert abs(Em[1] - Em[0]) / Em[0] > 1e-3
    assert abs(O.observables(prob, psi1, 150 * prob.dt)["E"] - Ep[1]) < 1e-13


# ---------------------------------------------------------------- T2
@pytest.mark.parametrize("dims,m,modes", [(2, 0.0, (5, 3)), (2, 0.5, (5, 3)), (2, 0.5, (-2, 7)),
                                          (3, 0.0, (2, -1, 3)), (3, 1.0, (2, -1, 3)),
                                          (3, 1.0, (0, 0, 0))])
def test_plane_wave_phase(dims, m, modes):
    """Eq. pwdsip with the eigenspinor of Sect. 2.1: a lattice plane wave is
    an exact eigenmode and advances by exp(-i w n dt)."""
    if dims == 2:
        prob = W.Problem(2, (16, 12, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), m)
        n = 200
    else:
        prob = W.Problem(3, (8, 6, 10), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), m)
        n = 100
    psi0, w = CF.plane_wave_state(prob, modes)
    psi = O.step(prob, psi0, n)
    ref = psi0 * np.exp(-1j * w * n * prob.dt)
    err = np.linalg.norm(psi - ref) / np.linalg.norm(ref)
    assert err < 1e-12


def test_plane_wave_negative_energy_3d():
    prob = W.Problem(3, (6, 6, 6), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.6)
    psi0, w = CF.plane_wave_state(prob, (1, 2, -1), positive=False)
    assert w < 0
    psi = O.step(prob, psi0, 60)
    err = np.linalg.norm(psi - psi0 * np.exp(-1j * w * 60 * prob.dt)) / np.linalg.norm(psi0)
    assert err < 1e-12


# ---------------------------------------------------------------- T3 / T4
def one_step_matrix(prob):
    n = int(np.prod(prob.shape))
    G = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1.0
        G[:, i] = O.step(prob, e.reshape(prob.shape), 1).reshape(-1)
    return G


@pytest.mark.parametrize("dims,N,m", [(2, (4, 4), 0.3), (2, (4, 4), 0.0), (3, (2, 2, 2), 0.5)])
def test_exact_spectrum(dims, N, m):
    """Single cone (Sect. 2.1, Fig. 2; Sect. 3): the eigen-phases of the
    one-step map are exactly -+ w(k) dt over the reduced zone, each with the
    multiplicity of the staggered copy, and all have modulus one."""
    prob = W.Problem(dims, tuple(N) + ((1,) if dims == 2 else ()), (1.0, 1.0, 1.0),
                     0.9 * W.stability_limit(dims), m)
    lam = np.linalg.eigvals(one_step_matrix(prob))
    assert np.max(np.abs(np.abs(lam) - 1.0)) < 1e-12
    got = np.sort(np.angle(lam))
    want = np.sort(-CF.reduced_spectrum(prob))  # exp(-i w dt)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) < 1e-10


@pytest.mark.parametrize("dims", [2, 3])
def test_stability_bound(dims):
    """Stability condition r_x^2 + r_y^2 (+ r_z^2) <= 1 (Sect. 2.2, Sect. 3):
    |lambda| = 1 at 0.9 r_max, also with a random real potential (Prop. 3 /
    Prop. 5); |lambda| > 1 at 1.1 r_max."""
    N = (4, 4, 1) if dims == 2 else (2, 2, 2)
    for r, stable in ((0.9, True), (1.1, False)):
        prob = W.Problem(dims, N, (1.0, 1.0, 1.0), r * W.stability_limit(dims), 0.3)
        for V in (None, W.random_potential(prob, 1, 0.7)):
            lam = np.linalg.eigvals(one_step_matrix(prob.with_fields(V_static=V)))
            if stable:
                assert np.max(np.abs(lam)) - 1.0 < 1e-12
            else:
                assert np.max(np.abs(lam)) > 1.05


@pytest.mark.parametrize("dims,N,dx", [(3, (2, 2, 2), (1.0, 1.3, 0.8)), (2, (4, 4, 1), (1.0, 0.7, 1.0))])
def test_stability_bound_anisotropic(dims, N, dx):
    """The stability condition with r_a = dt/dx_a per axis (Sect. 2.2:
    r_x^2 + r_y^2 + r_z^2 <= 1; Sect. 3: r_x^2 + r_y^2 <= 1) on an anisotropic
    grid: |lambda| = 1 at 0.97 of the largest stable dt, |lambda| > 1 at 1.03
    (a mistaken r_a on any axis moves the edge away from 1)."""
    dt_max = 1.0 / math.sqrt(sum(1.0 / dx[a] ** 2 for a in range(dims)))
    for f, stable in ((0.97, True), (1.03, False)):
        prob = W.Problem(dims, N, dx, f * dt_max, 0.3)
        lam = np.abs(np.linalg.eigvals(one_step_matrix(prob)))
        if stable:
            assert np.max(lam) - 1.0 < 1e-12
        else:
            assert np.max(lam) > 1.1


def test_functional_positive_definite_3d():
    """Appendix A / Prop. 3: at r <= 1/sqrt(3) the functional E is a norm;
    above the bound it is indefinite (its Hermitian form gets a negative
    eigenvalue)."""
    def min_eig(r):
        prob = W.Problem(3, (2, 2, 2), (1.0, 1.0, 1.0), r * W.stability_limit(3), 0.0)
        n = int(np.prod(prob.shape))
        Ed = [O.observables(prob, np.eye(n)[i].reshape(prob.shape))["E"] for i in range(n)]
        M = np.diag(np.array(Ed, complex))
        for i in range(n):
            for j in range(i + 1, n):
                ei, ej = np.eye(n)[i], np.eye(n)[j]
                a = O.observables(prob, (ei + ej).reshape(prob.shape))["E"] - Ed[i] - Ed[j]
                b = O.observables(prob, (ei + 1j * ej).reshape(prob.shape))["E"] - Ed[i] - Ed[j]
                M[i, j] = 0.5 * (a - 1j * b)
                M[j, i] = np.conj(M[i, j])
        return np.min(np.linalg.eigvalsh(M))
    assert min_eig(0.99) > 0.0
    assert min_eig(1.05) < 0.0


# ---------------------------------------------------------------- T7
@pytest.mark.parametrize("dims", [2, 3])
def test_light_cone(dims):
    """Nearest-neighbour stencil (Eq. 3+3Ddis): after n steps a single
    nonzero value spreads at most 2n half-lattice steps per axis (one per
    half-step); everything outside is exactly zero."""
    N = (15, 13, 11)
    prob = W.Problem(dims, N if dims == 3 else (15, 13, 1), (1.0, 1.0, 1.0),
                     0.9 * W.stability_limit(dims), 0.5)
    src_cell = (7, 6, 5)
    n = 2
    _, offs, _, _ = W.plane_tables(dims)
    for plane in range(prob.n_planes):
        psi = O.step(prob, W.delta_state(prob, plane, src_cell), n)
        so = [2 * src_cell[a] + offs[plane][a] for a in range(dims)]
        for pl in range(prob.n_planes):
            xyz = W.site_positions(prob, pl)
            dist = sum(np.abs(2 * xyz[a] - so[a]) for a in range(dims))  # half-lattice L1
            outside = dist > 2 * n
            assert np.all(psi[pl][outside] == 0.0)
        assert np.count_nonzero(psi) > 1


# ---------------------------------------------------------------- T6
def test_3d_reduces_to_2d_bitwise():
    """Sect. 3: with z-independent data and B = C = 0 the (3+1)D scheme
    carries A, D exactly like u, v of the (2+1)D scheme (the z differences
    vanish), for any V(x, y)."""
    N = (9, 7)
    Nz = 4
    p2 = W.Problem(2, (N[0], N[1], 1), (1.0, 1.0, 1.0), 0.5, 0.35)
    p3 = W.Problem(3, (N[0], N[1], Nz), (1.0, 1.0, 1.0), 0.5, 0.35)
    V2 = W.random_potential(p2, 7, 0.6)
    V3 = np.zeros(p3.shape)
    psi2 = W.random_state(p2, 8)
    psi3 = np.zeros(p3.shape, complex)
    for z in range(Nz):  # A0,A1 <- u0,u1 ; D0,D1 <- v0,v1
        psi3[0, z], psi3[1, z], psi3[6, z], psi3[7, z] = psi2[0, 0], psi2[1, 0], psi2[2, 0], psi2[3, 0]
        V3[0, z], V3[1, z], V3[6, z], V3[7, z] = V2[0, 0], V2[1, 0], V2[2, 0], V2[3, 0]
    out2 = O.step(p2.with_fields(V_static=V2), psi2, 37)
    out3 = O.step(p3.with_fields(V_static=V3), psi3, 37)
    for z in range(Nz):
        assert np.array_equal(out3[0, z], out2[0, 0]) and np.array_equal(out3[1, z], out2[1, 0])
        assert np.array_equal(out3[6, z], out2[2, 0]) and np.array_equal(out3[7, z], out2[3, 0])
        assert not np.any(out3[2:6, z])


# ---------------------------------------------------------------- T9
@pytest.mark.parametrize("dims", [2, 3])
def test_gauge_covariance_constant_vector_potential(dims):
    """Sect. 4 (Peierls substitution): a constant A with q A_a L_a = 2 pi n_a
    is a pure gauge; psi_A(t) = exp(i q A.x) psi_0(t) at every site."""
    N = (8, 6, 5)
    prob = W.Problem(dims, N if dims == 3 else (8, 6, 1), (1.0, 1.0, 1.0),
                     0.9 * W.stability_limit(dims), 0.4)
    prob = prob.with_fields(V_static=W.random_potential(prob, 5, 0.5))
    q = 0.7
    A = [2 * math.pi * n / (q * prob.N[a] * prob.dx[a]) for a, n in zip(range(dims), (1, -2, 3))]
    A += [0.0] * (3 - dims)
    psi0 = W.random_state(prob, 3)
    gauge = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        xyz = W.site_positions(prob, pl)
        gauge[pl] = np.exp(1j * q * sum(A[a] * xyz[a] for a in range(dims)))
    out0 = O.step(prob, psi0, 40)
    outA = O.step(prob.with_fields(q=q, A_const=tuple(A)), gauge * psi0, 40)
    assert np.max(np.abs(outA - gauge * out0)) < 1e-12


@pytest.mark.parametrize("dims,axis", [(2, 0), (2, 1), (3, 2)])
def test_gauge_covariance_longitudinal_plane_wave(dims, axis):
    """Sect. 4: the Peierls phase of a link is q times the line integral of
    A along it.  A static longitudinal wave A_a = amp cos(k x_a + ph) along
    axis a is the pure gauge grad chi, chi = (amp/k) sin(k x_a + ph), so
    psi_A(t) = exp(i q chi) psi_0(t) holds exactly at every value; evaluating
    A at the link midpoint instead misses this by O((k dx)^2)."""
    N = (8, 6, 10)
    prob = W.Problem(dims, N if dims == 3 else (8, 6, 1), (1.0, 1.0, 1.0),
                     0.9 * W.stability_limit(dims), 0.4)
    prob = prob.with_fields(V_static=W.random_potential(prob, 6, 0.5))
    q, amp, ph = 0.8, 0.9, 0.35
    k = 2 * math.pi * 2 / (prob.N[axis] * prob.dx[axis])
    kvec = [0.0, 0.0, 0.0]
    kvec[axis] = k
    psi0 = W.random_state(prob, 4)
    gauge = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        x = W.site_positions(prob, pl)[axis]
        gauge[pl] = np.exp(1j * q * amp / k * np.sin(k * x + ph))
    out0 = O.step(prob, psi0, 30)
    f = dict(q=q, Apw_amp=amp, Apw_k=tuple(kvec), Apw_omega=0.0, Apw_phase=ph, Apw_pol=axis)
    outA = O.step(prob.with_fields(**f), gauge * psi0, 30)
    assert np.max(np.abs(outA - gauge * out0)) < 1e-12


def test_uniform_time_dependent_vector_potential_2d():
    """Sect. 4 with a spatially uniform A(t): a lattice plane wave stays a
    plane wave whose momentum is shifted, P_a = (2/dx) sin((k_a - q A_a(t))
    dx/2) (the link factor multiplies exp(i k h) by exp(-i q A h)).  The
    oracle must agree with this per-mode 2x2 recursion, each half-step at the
    time sheet of its neighbours."""
    N = (8, 8)
    dt = 0.9 * W.stability_limit(2)
    amp, om, q, m = 0.4, 0.3, 1.0, 0.25
    prob = W.Problem(2, (N[0], N[1], 1), (1.0, 1.0, 1.0), dt, m,
                     W.Fields(q=q, Apw_amp=amp, Apw_k=(0.0, 0.0, 0.0), Apw_omega=om, Apw_phase=0.2,
                              Apw_pol=1))
    k = (2 * math.pi * 1 / N[0], 2 * math.pi * 2 / N[1])
    u, v = 0.6 + 0.1j, -0.3 + 0.7j
    # state: u at t=-dt/2, v at t=0, amplitudes times exp(i k.x)
    psi0 = np.zeros(prob.shape, complex)
    for pl in range(4):
        xyz = W.site_positions(prob, pl)
        psi0[pl] = (u if pl < 2 else v) * np.exp(1j * (k[0] * xyz[0] + k[1] * xyz[1]))
    n = 30
    t = 0.0
    for _ in range(n):
        # upper half-step: A at time t
        Ay = amp * math.cos(-om * t + 0.2)
        Px, Py = 2 * math.sin(k[0] / 2), 2 * math.sin((k[1] - q * Ay) / 2)
        th = dt * m / 2
        S = dt * 1j * (Px - 1j * Py) * v   # r(delta_x - i delta_y) v with delta -> 2i sin
        u = ((1 - 1j * th) * u - S) / (1 + 1j * th)
        Ay = amp * math.cos(-om * (t + dt / 2) + 0.2)
        Py = 2 * math.sin((k[1] - q * Ay) / 2)
        th = -dt * m / 2
        S = dt * 1j * (Px + 1j * Py) * u
        v = ((1 - 1j * th) * v - S) / (1 + 1j * th)
        t += dt
    out = O.step(prob, psi0, n)
    ref = np.zeros(prob.shape, complex)
    for pl in range(4):
        xyz = W.site_positions(prob, pl)
        ref[pl] = (u if pl < 2 else v) * np.exp(1j * (k[0] * xyz[0] + k[1] * xyz[1]))
    assert np.max(np.abs(out - ref)) < 1e-12


def test_uniform_time_dependent_scalar_potential_2d():
    """Eqs. ss1-ss4 with a spatially uniform V(t) (a constant static array
    modulated by 1 + a cos(w t)): a lattice plane wave stays a plane wave
    and each half-step is a 2x2 Cayley map of its two amplitudes, with
    theta = dt (m + V(t))/2 on the upper half-step and dt (V(t + dt/2) - m)/2
    on the lower one (each at its own sheet's midpoint time).  The oracle must
    agree with this per-mode recursion."""
    N = (8, 6)
    dt = 0.9 * W.stability_limit(2)
    V1, amp, om, m = 0.35, 0.7, 0.5, 0.3
    prob = W.Problem(2, (N[0], N[1], 1), (1.0, 1.0, 1.0), dt, m)
    prob = prob.with_fields(V0=-0.1, V_static=np.full(prob.shape, V1), Vmod_amp=amp, Vmod_omega=om)
    k = (2 * math.pi * 3 / N[0], 2 * math.pi * -1 / N[1])
    u, v = 0.2 - 0.5j, 0.8 + 0.1j
    psi0 = np.zeros(prob.shape, complex)
    for pl in range(4):
        xyz = W.site_positions(prob, pl)
        psi0[pl] = (u if pl < 2 else v) * np.exp(1j * (k[0] * xyz[0] + k[1] * xyz[1]))
    Px, Py = 2 * math.sin(k[0] / 2), 2 * math.sin(k[1] / 2)
    V = lambda t: -0.1 + V1 * (1 + amp * math.cos(om * t))
    n, t0 = 40, 0.35
    t = t0
    for _ in range(n):
        th = dt * (m + V(t)) / 2
        u = ((1 - 1j * th) * u - dt * 1j * (Px - 1j * Py) * v) / (1 + 1j * th)
        th = dt * (V(t + dt / 2) - m) / 2
        v = ((1 - 1j * th) * v - dt * 1j * (Px + 1j * Py) * u) / (1 + 1j * th)
        t += dt
    out = O.step(prob, psi0, n, t0)
    ref = np.zeros(prob.shape, complex)
    for pl in range(4):
        xyz = W.site_positions(prob, pl)
        ref[pl] = (u if pl < 2 else v) * np.exp(1j * (k[0] * xyz[0] + k[1] * xyz[1]))
    assert np.max(np.abs(out - ref)) < 1e-12


def test_uniform_time_dependent_fields_3d():
    """Eqs. ss1-ss4 in (3+1)D with a spatially uniform V(t) and A(t) (a
    constant A_x plus A_z = amp cos(phase - w t)): a lattice plane wave keeps
    one amplitude per component A, B, C, D, and a step is the per-mode
    recursion S_A = i dt (P_z c + (P_x - i P_y) d), S_B = i dt ((P_x + i P_y) c
    - P_z d), S_C = i dt (P_z a + (P_x - i P_y) b), S_D = i dt ((P_x + i P_y) a
    - P_z b), with P_a = (2/dx) sin((k_a - q A_a) dx/2) and every field taken
    at its half-step's time sheet (upper t, lower t + dt/2)."""
    N = (6, 5, 8)
    dt = 0.9 * W.stability_limit(3)
    m, q, V1, vamp, vom = 0.4, 0.9, 0.3, 0.5, 0.6
    Ax, amp, om, ph = 0.25, 0.45, 0.35, 0.3
    prob = W.Problem(3, N, (1.0, 1.0, 1.0), dt, m)
    prob = prob.with_fields(V0=0.05, V_static=np.full(prob.shape, V1), Vmod_amp=vamp, Vmod_omega=vom,
                            q=q, A_const=(Ax, 0.0, 0.0), Apw_amp=amp, Apw_k=(0.0, 0.0, 0.0), Apw_omega=om,
                            Apw_phase=ph, Apw_pol=2)
    k = (2 * math.pi * 1 / N[0], 2 * math.pi * -2 / N[1], 2 * math.pi * 3 / N[2])
    amps = [0.3 + 0.2j, -0.5 + 0.1j, 0.2 - 0.6j, 0.4 + 0.4j]  # a, b, c, d
    comp = [0, 0, 1, 1, 2, 2, 3, 3]  # planes A0 A1 B0 B1 C0 C1 D0 D1

    def wave(ampl):
        out = np.zeros(prob.shape, complex)
        for pl in range(8):
            xyz = W.site_positions(prob, pl)
            out[pl] = ampl[comp[pl]] * np.exp(1j * sum(k[i] * xyz[i] for i in range(3)))
        return out

    V = lambda t: 0.05 + V1 * (1 + vamp * math.cos(vom * t))
    P = lambda t: [2 * math.sin((k[0] - q * Ax) / 2), 2 * math.sin(k[1] / 2),
                   2 * math.sin((k[2] - q * amp * math.cos(ph - om * t)) / 2)]
    a, b, c, d = amps
    n, t0 = 25, 0.15
    t = t0
    for _ in range(n):
        Px, Py, Pz = P(t)
        th = dt * (m + V(t)) / 2
        a = ((1 - 1j * th) * a - 1j * dt * (Pz * c + (Px - 1j * Py) * d)) / (1 + 1j * th)
        b = ((1 - 1j * th) * b - 1j * dt * ((Px + 1j * Py) * c - Pz * d)) / (1 + 1j * th)
        Px, Py, Pz = P(t + dt / 2)
        th = dt * (V(t + dt / 2) - m) / 2
        c = ((1 - 1j * th) * c - 1j * dt * (Pz * a + (Px - 1j * Py) * b)) / (1 + 1j * th)
        d = ((1 - 1j * th) * d - 1j * dt * ((Px + 1j * Py) * a - Pz * b)) / (1 + 1j * th)
        t += dt
    out = O.step(prob, wave(amps), n, t0)
    assert np.max(np.abs(out - wave([a, b, c, d]))) < 1e-12


def test_time_reversal_3d():
    """Eqs. ss1-ss4 are explicit Cayley maps, each half-step reading only the
    other time sheet, so the scheme runs backwards exactly: shifting the
    lattice by dx/2 along z swaps the upper and lower sheets (A,B <-> C,D
    without changing any value's sign class (x+y parity)), and stepping the
    shifted state with -dt and -m applies the inverse half-steps in reverse
    order.  n steps forward and n back recover the initial state to
    rounding; an update that read its own sheet, or values of the other
    sheet from the wrong step, would not."""
    N = (6, 5, 7)
    prob = W.Problem(3, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.5)
    Vs = W.random_potential(prob, 31, 0.5)
    prob = prob.with_fields(V_static=Vs, q=0.8, A_const=(0.3, -0.2, 0.1))
    # plane -> (plane after the shift, cell shift along z): A0->C0, A1->C1,
    # B0->D0(+1), B1->D1(+1), C0->A0(+1), C1->A1(+1), D0->B0, D1->B1
    moves = {0: (4, 0), 1: (5, 0), 2: (6, 1), 3: (7, 1), 4: (0, 1), 5: (1, 1), 6: (2, 0), 7: (3, 0)}

    def shift(a):
        out = np.empty_like(a)
        for p, (q, dz) in moves.items():
            out[q] = np.roll(a[p], dz, axis=0)
        return out

    def unshift(a):
        out = np.empty_like(a)
        for p, (q, dz) in moves.items():
            out[p] = np.roll(a[q], -dz, axis=0)
        return out

    psi0 = W.random_state(prob, 32)
    n = 30
    fwd = O.step(prob, psi0, n)
    back = W.Problem(3, N, prob.dx, -prob.dt, -prob.m, prob.fields).with_fields(V_static=shift(Vs))
    out = unshift(O.step(back, shift(fwd), n))
    assert np.max(np.abs(fwd - psi0)) > 0.05
    assert np.max(np.abs(out - psi0)) < 1e-13


def test_klein_step_normal_incidence_nearly_transparent():
    """Sect. 5 (soft check): at normal incidence with m = 0 a packet passes a
    Klein step almost completely (in the continuum exactly: chirality
    conservation).  On the lattice the abrupt step reflects a little; with
    V dx = 0.5 and k0 dx = 0.25 the transmitted fraction, once the packet has
    passed, exceeds 0.98 (measured 0.984), and halving V reduces the
    reflection at least threefold."""
    def transmitted(V):
        N = 320
        x0 = N / 2 + 0.25
        prob = W.Problem(2, (N, 2, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.0,
                         W.Fields(step_axis=0, step_x0=x0, step_V=V))
        sigma, kx = 16.0, 0.25
        w = W.continuum_spinor(2, (kx, 0.0), 0.0)
        _, _, _, comp = W.plane_tables(2)
        psi = np.zeros(prob.shape, complex)
        for pl in range(4):  # a packet uniform along y: normal incidence only
            x = W.site_positions(prob, pl)[0]
            ts = W.sheet_time(prob, pl, 0.0)
            psi[pl] = w[comp[pl]] * np.exp(-(x - (x0 - 4 * sigma)) ** 2 / (2 * sigma ** 2)) * \
                np.exp(1j * (kx * x - kx * ts))
        psi /= np.linalg.norm(psi)
        out = O.step(prob, psi, int(8 * sigma / (0.95 * prob.dt)))
        right = sum(np.sum(np.abs(out[pl][W.site_positions(prob, pl)[0] > x0]) ** 2) for pl in range(4))
        return right / np.sum(np.abs(out) ** 2)

    T1, T2 = transmitted(0.5), transmitted(0.25)
    assert T1 > 0.98
    assert (1 - T2) < (1 - T1) / 3


@pytest.mark.parametrize("dims", [2, 3])
def test_potential_values_at_every_site(dims):
    """Eqs. ss1-ss4: with every lower value zero, the upper half-step sees no
    difference part, so one step multiplies every upper value F by its own
    Cayley factor (1 - i theta)/(1 + i theta), theta = dt (m + V(x, t))/2, and
    the lower half-step leaves it alone.  This fixes the value of V at every
    upper site's own position: a Klein step H(x_a - x0) with a site exactly on
    x0 (strict '>'), an off-grid soft core -Z/sqrt(|x - c|^2 + a^2) (plain
    distance), a modulated static array and absorbing layers (Im V)."""
    N = (7, 6, 5) if dims == 3 else (7, 6, 1)
    prob = W.Problem(dims, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.3)
    Vs = W.random_potential(prob, 21, 0.4)
    c = (2.3, 3.65, 1.8)
    f = dict(V0=0.1, step_axis=1, step_x0=2.5, step_V=0.6, sc_Z=0.8, sc_a=1.1, sc_center=c, V_static=Vs,
             Vmod_amp=0.3, Vmod_omega=0.7, V0_imag=-0.01, abs_W=0.5, abs_width=2.0, abs_axes=(1 << dims) - 1)
    prob = prob.with_fields(**f)
    P_up = prob.n_planes // 2  # upper planes come first
    psi = W.random_state(prob, 22)
    psi[P_up:] = 0.0
    t0 = 0.4
    out = O.step(prob, psi, 1, t0)
    L = [prob.N[a] * prob.dx[a] for a in range(3)]
    for pl in range(P_up):
        x = W.site_positions(prob, pl)
        V = 0.1 + 0.6 * (x[1] > 2.5) + Vs[pl] * (1 + 0.3 * math.cos(0.7 * t0))
        V = V - 0.8 / np.sqrt(sum((x[a] - c[a]) ** 2 for a in range(dims)) + 1.1 ** 2)
        Wl = np.zeros(V.shape)
        for a in range(dims):
            d = np.minimum(x[a], L[a] - x[a])
            Wl += np.where(d < 2.0, (1 - d / 2.0) ** 2, 0.0)
        th = prob.dt * (prob.m + V + 1j * (-0.01 - 0.5 * Wl)) / 2
        assert np.max(np.abs(out[pl] - psi[pl] * (1 - 1j * th) / (1 + 1j * th))) < 1e-14
    ys = np.concatenate([W.site_positions(prob, pl)[1].ravel() for pl in range(P_up)])
    assert np.any(ys == 2.5) and np.any(ys == 3.0)  # upper sites on and just beyond the step


# ---------------------------------------------------------------- T10
def test_proposition_2_bound():
    """Prop. 2: for r_x + r_y + r_z < 1 the naive norm stays below
    E0 / (1 - r_x - r_y - r_z) for all time, for arbitrary V(x,t)."""
    prob = W.Problem(3, (5, 4, 6), (1.0, 1.0, 1.0), 0.3, 0.2)
    prob = prob.with_fields(V_static=W.random_potential(prob, 4, 2.0), Vmod_amp=0.5, Vmod_omega=0.9)
    psi = W.random_state(prob, 6)
    E0 = O.observables(prob, psi)["E"]
    bound = E0 / (1 - 3 * 0.3)
    t = 0.0
    for _ in range(40):
        psi = O.step(prob, psi, 5, t)
        t += 5 * prob.dt
        assert O.observables(prob, psi, t)["naive"] <= bound


def _appendix_sums_3d(prob, psi):
    """The appendix's sum of squares around the A and B sites at
    r = 1/sqrt(3) (E-tilde) and the grid-averaged norm of (C, D) of Prop. 3,
    evaluated on the half lattice (neighbours at +-1 with the periodic wrap)."""
    M = [2 * prob.N[a] for a in range(3)]
    f = np.zeros((M[2], M[1], M[0]), complex)
    for pl in range(prob.n_planes):
        X, Y, Z = W.half_lattice_points(prob, pl)
        f[Z, Y, X] = psi[pl]
    at = lambda d, ax: np.roll(f, -d, axis=2 - ax)  # the value at F + d e_ax
    Z, Y, X = np.meshgrid(*[np.arange(n) for n in f.shape], indexing="ij")
    A = ((X + Y) % 2 == 0) & (Z % 2 == 0)
    B = ((X + Y) % 2 == 1) & (Z % 2 == 1)
    s3 = math.sqrt(3.0)
    aA = (at(1, 2) + at(1, 0) - 1j * at(1, 1)) / s3    # (C_{z+} + D_{x+} - i D_{y+}) / sqrt(3)
    bA = (at(-1, 2) + at(-1, 0) - 1j * at(-1, 1)) / s3
    aB = (at(1, 2) - at(1, 0) - 1j * at(1, 1)) / s3    # (D_{z+} - C_{x+} - i C_{y+}) / sqrt(3)
    bB = (at(-1, 2) - at(-1, 0) - 1j * at(-1, 1)) / s3
    E_tilde = 0.5 * np.sum(np.abs(aA - f)[A] ** 2 + np.abs(bA + f)[A] ** 2) + \
        0.5 * np.sum(np.abs(aB + f)[B] ** 2 + np.abs(bB - f)[B] ** 2)
    cd_avg = 0.25 * np.sum(np.abs(aA + bA)[A] ** 2) + 0.25 * np.sum(np.abs(aB + bB)[B] ** 2)
    return E_tilde, cd_avg


def test_appendix_sum_of_squares_and_proposition_3():
    """Appendix A: at r = 1/sqrt(3) the functional equals a sum of squares
    around the A and B sites (E-tilde, an algebraic identity for every
    state), so E >= 0 and the grid-averaged norm of (C, D) of Prop. 3 never
    exceeds E.  Checked on random states (identity to rounding) and along a
    run with a random, time-dependent potential and a mass (the averaged
    norm stays below the conserved E0)."""
    N = (5, 4, 6)
    prob = W.Problem(3, N, (1.0, 1.0, 1.0), 1 / math.sqrt(3), 0.7)
    for seed in (3, 4):
        psi = W.random_state(prob, seed)
        ob = O.observables(prob, psi)
        E_tilde, _ = _appendix_sums_3d(prob, psi)
        assert abs(E_tilde - ob["E_upper"]) < 1e-14 and abs(E_tilde - ob["E"]) < 1e-14
    prob = prob.with_fields(V_static=W.random_potential(prob, 5, 0.8), Vmod_amp=0.6, Vmod_omega=0.9,
                            step_axis=0, step_x0=2.25, step_V=0.5)
    psi = W.random_state(prob, 6)
    E0 = O.observables(prob, psi)["E"]
    t = 0.0
    for _ in range(8):
        psi = O.step(prob, psi, 25, t)
        t += 25 * prob.dt
        E = O.observables(prob, psi, t)["E"]
        E_tilde, cd_avg = _appendix_sums_3d(prob, psi)
        assert abs(E - E0) < 1e-12 and abs(E_tilde - E) < 1e-12
        assert cd_avg <= E0 * (1 + 1e-12)


def test_2d_functional_is_a_sum_of_squares_at_the_bound():
    """Prop. 5's proof (Sect. 3): at r = 1/sqrt(2) the (2+1)D functional equals
    the auxiliary E~ = sum over v sites G of 1/2 |a_G + v_G|^2 + 1/2 |b_G - v_G|^2,
    a_G = (u_{G+x} + i u_{G+y})/sqrt(2), b_G = (u_{G-x} + i u_{G-y})/sqrt(2),
    for every state (the u-u cross terms telescope).  With the delta_+ reading
    of the functional the signs are +i; the printed -i would not reproduce E.
    Checked on random states with the oracle's E."""
    N = (7, 6)
    prob = W.Problem(2, (N[0], N[1], 1), (1.0, 1.0, 1.0), 1.0 / math.sqrt(2.0), 0.4)
    M = (2 * N[0], 2 * N[1])
    for seed in (8, 9):
        psi = W.random_state(prob, seed)
        f = np.zeros((M[1], M[0]), complex)
        for pl in range(4):
            X, Y, _ = W.half_lattice_points(prob, pl)
            f[Y[0], X[0]] = psi[pl, 0]
        at = lambda d, ax: np.roll(f, -d, axis=1 - ax)  # the value at G + d e_ax
        Y, X = np.meshgrid(np.arange(M[1]), np.arange(M[0]), indexing="ij")
        v = (X + Y) % 2 == 1
        a = (at(1, 0) + 1j * at(1, 1)) / math.sqrt(2)
        b = (at(-1, 0) + 1j * at(-1, 1)) / math.sqrt(2)
        E_tilde = 0.5 * np.sum(np.abs(a + f)[v] ** 2 + np.abs(b - f)[v] ** 2)
        ob = O.observables(prob, psi)
        assert abs(E_tilde - ob["E"]) < 1e-14 and abs(E_tilde - ob["E_upper"]) < 1e-14
        printed = 0.5 * np.sum(np.abs((at(1, 0) - 1j * at(1, 1)) / math.sqrt(2) + f)[v] ** 2 +
                               np.abs((at(-1, 0) - 1j * at(-1, 1)) / math.sqrt(2) - f)[v] ** 2)
        assert abs(printed - ob["E"]) > 1e-3


def test_proposition_5_averaged_norm_2d():
    """Prop. 5 (Sect. 3): at r = 1/sqrt(2) the grid-averaged norm of u stays
    below E0 (so ||u~||^2 + ||v~||^2 <= 2 E0) for arbitrary V.  With the
    delta_+ reading of the (2+1)D functional the averaging carries +i:
    ||u~||^2 = sum_j |(u_{j+(1,0)} + i u_{j+(1/2,1/2)} + u_j + i u_{j+(1/2,-1/2)}) / (2 sqrt 2)|^2
    over j in Z^2 u (Z+1/2)^2; the proof's auxiliary E~ then expands to the
    conserved E (the u-u cross terms telescope for either sign)."""
    N = 8
    prob = W.Problem(2, (N, N, 1), (1.0, 1.0, 1.0), 1.0 / math.sqrt(2.0), 0.3)
    prob = prob.with_fields(V_static=W.random_potential(prob, 1, 1.5))
    psi = W.random_state(prob, 2)
    E0 = O.observables(prob, psi)["E"]

    def unorm(s):
        u0, u1 = s[0, 0], s[1, 0]
        sx = lambda a: np.roll(a, -1, axis=1)
        sy = lambda a: np.roll(a, -1, axis=0)
        my = lambda a: np.roll(a, 1, axis=0)
        # j on u0 sites (integer): j+(1,0) -> u0[x+1], j+(1/2,1/2) -> u1[j], j+(1/2,-1/2) -> u1[y-1]
        a0 = (sx(u0) + 1j * u1 + u0 + 1j * my(u1)) / (2 * math.sqrt(2))
        # j on u1 sites (half-integer): j+(1,0) -> u1[x+1], j+(1/2,1/2) -> u0[x+1,y+1], j+(1/2,-1/2) -> u0[x+1]
        a1 = (sx(u1) + 1j * sx(sy(u0)) + u1 + 1j * sx(u0)) / (2 * math.sqrt(2))
        return float(np.sum(np.abs(a0) ** 2) + np.sum(np.abs(a1) ** 2))

    t = 0.0
    for _ in range(30):
        psi = O.step(prob, psi, 7, t)
        t += 7 * prob.dt
        assert unorm(psi) <= E0 * (1 + 1e-12)


def test_partial_density_splits_naive_norm():
    prob = W.Problem(2, (12, 8, 1), (1.0, 1.0, 1.0), 0.5, 0.1)
    psi = W.random_state(prob, 1)
    x0 = 5.25
    right = O.partial_density(prob, psi, 0, x0)
    xs = [W.site_positions(prob, pl)[0] for pl in range(4)]
    want = sum(float(np.sum(np.abs(psi[pl][xs[pl] > x0]) ** 2)) for pl in range(4))
    assert abs(right - want) < 1e-14


# ---------------------------------------------------------------- complex potential, absorbing layers
def growth_matrix_2d(kx, ky, m, V, dt, dx=1.0, dy=1.0):
    """Amplification matrix G = -S^-1 T of the (2+1)D scheme for constant m
    and complex V (Sect. 3, Eq. stabilityeq, hbar = c = 1).  The mass and
    potential enter as (m +- V)/(2 i), the time average of the scheme: the
    printed S and T drop the 1/2, while the printed det G = Q and N keep it."""
    a = 2j / dx * math.sin(kx * dx / 2.0)
    b = 2j / dy * math.sin(ky * dy / 2.0)
    S = np.array([[1.0 / dt - (m + V) / 2j, 0.0], [a + 1j * b, 1.0 / dt + (m - V) / 2j]])
    T = np.array([[-1.0 / dt - (m + V) / 2j, a - 1j * b], [0.0, -1.0 / dt + (m - V) / 2j]])
    return -np.linalg.solve(S, T)


def match_eigenvalues(got, want):
    """Largest distance of a greedy one-to-one matching of two multisets."""
    got = list(got)
    worst = 0.0
    for w in want:
        i = int(np.argmin([abs(g - w) for g in got]))
        worst = max(worst, abs(got.pop(i) - w))
    return worst


@pytest.mark.parametrize("V", [0.2 - 0.3j, -0.1 + 0.15j, -0.4j])
def test_growth_factors_complex_potential_2d(V):
    """Sect. 3 (growth factors): for a constant complex V the eigenvalues of
    the oracle's one-step map are the eigenvalues of G(k) over the grid's k,
    each twice (the staggered copy); det G equals the printed
    Q = (4 + (m^2 - V^2) dt^2 - 4 i V dt) / N, N = 4 + (m^2 - V^2) dt^2 + 4 i V dt,
    for every k; |lambda| < 1 where Im V < 0 (absorbing) and > 1 where Im V > 0."""
    m = 0.3
    prob = W.Problem(2, (4, 4, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), m,
                     W.Fields(V0=V.real, V0_imag=V.imag))
    dt = prob.dt
    lam = np.linalg.eigvals(one_step_matrix(prob))
    Nn = 4 + (m * m - V * V) * dt * dt + 4j * V * dt
    Q = (4 + (m * m - V * V) * dt * dt - 4j * V * dt) / Nn
    want = []
    for nx, ny in np.ndindex(4, 4):
        g = growth_matrix_2d(2 * math.pi * nx / 4, 2 * math.pi * ny / 4, m, V, dt)
        assert abs(np.linalg.det(g) - Q) < 1e-13
        want += list(np.linalg.eigvals(g)) * 2
    assert len(want) == lam.size
    assert match_eigenvalues(lam, want) < 1e-10
    if V.imag < 0:
        assert np.max(np.abs(lam)) < 1.0
    else:
        assert np.max(np.abs(lam)) > 1.0


@pytest.mark.parametrize("dims", [2, 3])
def test_uniform_state_complex_potential(dims):
    """A spatially constant state has S = 0, so every upper value is
    multiplied by (1 - i th_u)/(1 + i th_u) and every lower one by
    (1 - i th_l)/(1 + i th_l) per step, th_u = dt (m + V)/2, th_l = dt (V - m)/2,
    with V complex (Eqs. ss1-ss4)."""
    V = 0.15 - 0.25j
    m = 0.6
    prob = prob2(N=(3, 4)) if dims == 2 else prob3(N=(2, 3, 2))
    prob = W.Problem(prob.dims, prob.N, prob.dx, prob.dt, m, W.Fields(V0=V.real, V0_imag=V.imag))
    rng = np.random.default_rng(3)
    c = rng.standard_normal(prob.n_planes) + 1j * rng.standard_normal(prob.n_planes)
    psi = np.broadcast_to(c[:, None, None, None], prob.shape).copy()
    n = 7
    out = O.step(prob, psi, n)
    th_u, th_l = prob.dt * (m + V) / 2, prob.dt * (V - m) / 2
    upper = 4 if dims == 3 else 2
    for pl in range(prob.n_planes):
        th = th_u if pl < upper else th_l
        want = c[pl] * ((1 - 1j * th) / (1 + 1j * th)) ** n
        assert np.max(np.abs(out[pl] - want)) < 1e-13 * abs(want) + 1e-15


@pytest.mark.parametrize("dims", [2, 3])
def test_absorbing_layer_functional_decreases(dims):
    """Absorbing layers (Im V <= 0 near the box faces, Sect. 3): E never
    grows from one step to the next and falls once the state reaches the
    layers; abs_W = 0 reproduces the run without layers bit for bit."""
    prob = prob2(N=(14, 12)) if dims == 2 else prob3(N=(8, 7, 9))
    axes = 0b11 if dims == 2 else 0b101
    V = W.random_potential(prob, 2, 0.5)
    lay = prob.with_fields(V_static=V, abs_W=0.6, abs_width=2.5, abs_axes=axes)
    psi = W.random_state(prob, 8)
    E = [O.observables(lay, psi, 0.0)["E"]]
    cur = psi
    for s in range(12):
        cur = O.step(lay, cur, 1, s * prob.dt)
        E.append(O.observables(lay, cur, (s + 1) * prob.dt)["E"])
    d = np.diff(E)
    assert np.all(d <= 1e-13 * E[0])
    assert E[-1] < 0.9 * E[0]
    off = prob.with_fields(V_static=V, abs_W=0.0, abs_width=2.5, abs_axes=axes)
    assert np.array_equal(O.step(off, psi, 5), O.step(prob.with_fields(V_static=V), psi, 5))


@pytest.mark.parametrize("dims", [2, 3])
def test_absorbing_layer_placement(dims):
    """The layer acts only within abs_width of the box faces along the
    selected axes: a state supported in the middle evolves bit for bit as
    without layers while its light cone stays clear of them, and differs
    once it has reached them."""
    N = (30, 26) if dims == 2 else (22, 20, 18)
    prob = prob2(N=N) if dims == 2 else prob3(N=N)
    lay = prob.with_fields(abs_W=0.8, abs_width=4.0, abs_axes=(1 << dims) - 1)
    psi = np.zeros(prob.shape, complex)
    rng = np.random.default_rng(4)
    mid = [n // 2 for n in prob.N[:dims]]
    sl = [slice(None)]
    sl += [slice(mid[2] - 1, mid[2] + 2)] if dims == 3 else [slice(0, 1)]
    sl += [slice(mid[1] - 1, mid[1] + 2), slice(mid[0] - 1, mid[0] + 2)]
    block = psi[tuple(sl)]
    psi[tuple(sl)] = rng.standard_normal(block.shape) + 1j * rng.standard_normal(block.shape)
    # the support reaches mid +- 2 cells; one step spreads it by one cell per axis
    clear = min(prob.N[a] // 2 for a in range(dims)) - 2 - 5  # cells to the layer edge (width 4 + 1)
    assert np.array_equal(O.step(lay, psi, clear), O.step(prob, psi, clear))
    assert not np.array_equal(O.step(lay, psi, clear + 6), O.step(prob, psi, clear + 6))


# ---------------------------------------------------------------- Klein refraction (Sect. 5)
def test_klein_step_negative_refraction():
    """Sect. 5, oblique incidence on a Klein step with m = 0 and V = 2E: the
    transmitted packet is refracted to the other side of the normal (negative
    angle, specular for a single plane wave since |k| is the same on both
    sides), the reflected one leaves at the specular angle, and on the far
    side phase and group velocity point in opposite directions while on the
    near side they agree."""
    from tests import klein_refraction as K
    prob, psi, _ = W.workload_klein_oblique(N=384, sigma=16.0, kabs=0.5, offset=4.0)
    x0 = prob.fields.step_x0
    inc = math.radians(90.0 - 37.0)
    p1 = O.step(prob, psi, 250)
    p2 = O.step(prob, p1, 100, 250 * prob.dt)
    v, part = K.velocity(prob, p1, p2, 100, x0)
    ang_t = math.degrees(math.atan2(v["T"][1], v["T"][0]))
    ang_r = math.degrees(math.atan2(v["R"][1], v["R"][0]))
    assert -60.0 < ang_t < -40.0                      # negative refraction (53 deg incidence)
    assert abs(ang_r - (180.0 - math.degrees(inc))) < 3.0  # specular reflection
    assert part["T"][0] > 0.2 and part["R"][0] > 0.5
    kt, kr = part["T"][2], part["R"][2]
    cos_t = kt @ v["T"] / (np.linalg.norm(kt) * np.linalg.norm(v["T"]))
    cos_r = kr @ v["R"] / (np.linalg.norm(kr) * np.linalg.norm(v["R"]))
    assert cos_t < -0.9 and cos_r > 0.9


# ---------------------------------------------------------------- arbitrary vector potentials (Sect. 4)
@pytest.mark.parametrize("dims", [2, 3])
def test_gauge_covariance_arbitrary_lattice_gauge(dims):
    """Sect. 4: phases given as line integrals on every link.  For the pure
    gauge of an arbitrary (random) lattice function chi, link (F -> F + e_a)
    carrying chi(F + e_a) - chi(F), the evolution is exactly covariant:
    psi_A(t) = exp(i q chi) psi_0(t), which checks every link's start and end."""
    prob = prob2(N=(6, 5)) if dims == 2 else prob3(N=(4, 3, 5))
    prob = prob.with_fields(V_static=W.random_potential(prob, 8, 0.4))
    q = 0.9
    chi = W.random_lattice_gauge(prob, 12, 3.0)
    at = lambda P: chi[P[2], P[1], P[0]]
    links = W.link_integrals(prob, lambda a, S, E: at(E) - at(S))
    gauge = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        gauge[pl] = np.exp(1j * q * at(W.half_lattice_points(prob, pl)))
    psi0 = W.random_state(prob, 13)
    out0 = O.step(prob, psi0, 25)
    outA = O.step(prob.with_fields(q=q, A_links=links), gauge * psi0, 25)
    assert np.max(np.abs(outA - gauge * out0)) < 1e-12


@pytest.mark.parametrize("dims", [2, 3])
def test_link_integrals_equal_the_analytic_plane_wave(dims):
    """The array path and the analytic path are the same Peierls substitution:
    line integrals of a plane wave (with a constant part and a time
    modulation) tabulated per link reproduce the analytic fields."""
    prob = prob2(N=(8, 6)) if dims == 2 else prob3(N=(4, 6, 5))
    k = [2 * math.pi / (prob.N[a] * prob.dx[a]) * n for a, n in zip(range(dims), (1, 2, 1))] + [0.0] * (3 - dims)
    A0, amp, om, pol = 0.3, 0.8, 0.45, 1
    h = prob.dx[pol] / 2

    def integral(a, S, E):  # a constant A0 along pol: every link carries A0 h
        return np.full(S[0].shape, A0 * h if a == pol else 0.0)

    links = W.link_integrals(prob, integral)
    f_arr = dict(q=1.0, A_links=links, Alink_amp=amp, Alink_omega=om)
    # A_pol(t) = A0 (1 + amp cos(om t)): a constant plus a k = 0 wave of amplitude A0 amp
    f_ana = dict(q=1.0, A_const=tuple(A0 if b == pol else 0.0 for b in range(3)), Apw_amp=A0 * amp,
                 Apw_k=(0.0, 0.0, 0.0), Apw_omega=om, Apw_phase=0.0, Apw_pol=pol)
    psi0 = W.random_state(prob, 14)
    a = O.step(prob.with_fields(**f_arr), psi0, 30, 0.2)
    b = O.step(prob.with_fields(**f_ana), psi0, 30, 0.2)
    assert np.max(np.abs(a - b)) < 1e-12
    # a static wave along k (analytic line integrals per link) against the analytic path
    def wave(a_, S, E):
        if a_ != pol:
            return np.zeros(S[0].shape)
        mid = [(S[b] + 0.5 * (b == a_)) * prob.dx[b] / 2 for b in range(3)]
        ph = sum(k[b] * mid[b] for b in range(dims)) + 0.3
        u = 0.5 * k[a_] * h
        return amp * h * np.cos(ph) * (np.sin(u) / u if u != 0 else 1.0)
    links = W.link_integrals(prob, wave)
    a = O.step(prob.with_fields(q=1.0, A_links=links), psi0, 30)
    b = O.step(prob.with_fields(q=1.0, Apw_amp=amp, Apw_k=tuple(k), Apw_omega=0.0, Apw_phase=0.3, Apw_pol=pol),
               psi0, 30)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("dims", [2, 3])
def test_conservation_arbitrary_static_links(dims):
    """Lemma of Sect. 2 / Sect. 3 with an arbitrary static vector potential
    (random link integrals, not a pure gauge) and a random V: E is conserved
    exactly."""
    prob = prob2(N=(6, 5)) if dims == 2 else prob3(N=(4, 3, 5))
    prob = prob.with_fields(V_static=W.random_potential(prob, 9, 0.5))
    prob = prob.with_fields(q=0.7, A_links=W.random_links(prob, 15, 1.0))
    psi0 = W.random_state(prob, 16)
    d, e0, e1, psi = rel_drift(prob, psi0, 40)
    assert abs(d) < 1e-13
    assert abs(e1["naive"] - e0["naive"]) > 1e-6 * e0["naive"]  # a real field: the naive norm moves
