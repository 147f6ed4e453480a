"""Seeded synthetic inputs for the staggered leap-frog Dirac stepper.

This module builds problem descriptions and initial spinor states.  It is the
one module that both the CUDA path (tests, benchmark) and the CPU oracle read,
so it holds no arithmetic of the scheme itself: no stencil, no update, no
conserved functional and no lattice dispersion.  Wave packets use the
*continuum* free Dirac spinor (Sect. 2, Eq. 3+3D with constant m), evaluated
at every value's own position and time sheet.

Layout ("canonical", the library's host format): a complex128 array of shape
(P, Nz, Ny, Nx), x fastest.  (3+1)D has P = 8 planes A0,A1,B0,B1,C0,C1,D0,D1;
(2+1)D has P = 4 planes u0,u1,v0,v1 and Nz = 1.  Plane positions inside cell
j follow the grid definitions of Sect. 2 (and Sect. 3 for u, v):

    A0 j            A1 j+(1/2,1/2,0)     B0 j+(1/2,0,1/2)   B1 j+(0,1/2,1/2)
    C0 j+(0,0,1/2)  C1 j+(1/2,1/2,1/2)   D0 j+(1/2,0,0)     D1 j+(0,1/2,0)
    u0 j            u1 j+(1/2,1/2)       v0 j+(1/2,0)       v1 j+(0,1/2)

Upper planes (A, B, u) hold values at time t - dt/2, lower planes (C, D, v)
at time t.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

PLANES_3D = ("A0", "A1", "B0", "B1", "C0", "C1", "D0", "D1")
PLANES_2D = ("u0", "u1", "v0", "v1")
# offsets in half lattice constants
OFFSETS_3D = ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1), (0, 0, 1), (1, 1, 1), (1, 0, 0), (0, 1, 0))
OFFSETS_2D = ((0, 0, 0), (1, 1, 0), (1, 0, 0), (0, 1, 0))
UPPER_3D = (True, True, True, True, False, False, False, False)
UPPER_2D = (True, True, False, False)
# spinor component carried by each plane: A,B,C,D = 0..3 ; u,v = 0,1
COMPONENT_3D = (0, 0, 1, 1, 2, 2, 3, 3)
COMPONENT_2D = (0, 0, 1, 1)


@dataclass
class Fields:
    """External fields.  Scalar potential
    V(x,t) = V0 + step_V*H(x_axis - step_x0) - sc_Z/sqrt(|x-c|^2 + sc_a^2)
             + V_static(x)*(1 + Vmod_amp*cos(Vmod_omega*t)),
    vector potential A(x,t) = A_const + e_pol*Apw_amp*cos(k.x - Apw_omega*t + Apw_phase),
    coupled with charge q (Sect. 4), and an imaginary part of V for absorbing
    boundary layers (Sect. 3, growth factors).  V_static is one real per site
    in canonical layout (shape (P, Nz, Ny, Nx)) or None."""

    V0: float = 0.0
    step_axis: int = -1
    step_x0: float = 0.0
    step_V: float = 0.0
    sc_Z: float = 0.0
    sc_a: float = 1.0
    sc_center: Sequence[float] = (0.0, 0.0, 0.0)
    V_static: Optional[np.ndarray] = None
    Vmod_amp: float = 0.0
    Vmod_omega: float = 0.0
    q: float = 1.0
    A_const: Sequence[float] = (0.0, 0.0, 0.0)
    Apw_amp: float = 0.0
    Apw_k: Sequence[float] = (0.0, 0.0, 0.0)
    Apw_omega: float = 0.0
    Apw_phase: float = 0.0
    Apw_pol: int = 0
    # imaginary part of V: V0_imag - abs_W * sum over the axes in the bit mask
    # abs_axes of (1 - d/abs_width)^2 within abs_width of a box face (d = the
    # distance to the nearer face); Im V < 0 absorbs
    V0_imag: float = 0.0
    abs_W: float = 0.0
    abs_width: float = 0.0
    abs_axes: int = 0
    # an arbitrary vector potential by its line integrals (Sect. 4): shape
    # (dims, P, Nz, Ny, Nx), entry [a, plane, cell] = integral of A_a along the
    # link from that value's point to its neighbour at +dx_a/2, scaled at time
    # t by 1 + Alink_amp cos(Alink_omega t); None: none
    A_links: Optional[np.ndarray] = None
    Alink_amp: float = 0.0
    Alink_omega: float = 0.0


@dataclass
class Problem:
    """dims in {2, 3}; N = cells per axis; dx = lattice constants; dt = time
    step (hbar = c = 1); m = mass."""

    dims: int
    N: Sequence[int]
    dx: Sequence[float]
    dt: float
    m: float
    fields: Fields = field(default_factory=Fields)

    @property
    def n_planes(self) -> int:
        return 8 if self.dims == 3 else 4

    @property
    def shape(self) -> tuple:
        nz = self.N[2] if self.dims == 3 else 1
        return (self.n_planes, nz, self.N[1], self.N[0])

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape[1:]))

    def with_fields(self, **kw) -> "Problem":
        return dataclasses.replace(self, fields=dataclasses.replace(self.fields, **kw))


def stability_limit(dims: int) -> float:
    """Largest r = dt/dx (isotropic) the paper proves stable: 1/sqrt(3) in
    (3+1)D (Sect. 2, Stability) and 1/sqrt(2) in (2+1)D (Sect. 3)."""
    return 1.0 / math.sqrt(3.0) if dims == 3 else 1.0 / math.sqrt(2.0)


def plane_tables(dims: int):
    if dims == 3:
        return PLANES_3D, OFFSETS_3D, UPPER_3D, COMPONENT_3D
    return PLANES_2D, OFFSETS_2D, UPPER_2D, COMPONENT_2D


def site_positions(prob: Problem, plane: int):
    """Physical coordinates (x, y, z) of every site of one plane, each an
    array of shape (Nz, Ny, Nx)."""
    _, offs, _, _ = plane_tables(prob.dims)
    o = offs[plane]
    nz = prob.N[2] if prob.dims == 3 else 1
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(prob.N[1]), np.arange(prob.N[0]), indexing="ij")
    x = (jx + 0.5 * o[0]) * prob.dx[0]
    y = (jy + 0.5 * o[1]) * prob.dx[1]
    z = (jz + 0.5 * o[2]) * prob.dx[2] if prob.dims == 3 else np.zeros_like(x, dtype=float)
    return x, y, z


def sheet_time(prob: Problem, plane: int, t: float = 0.0) -> float:
    _, _, upper, _ = plane_tables(prob.dims)
    return t - 0.5 * prob.dt if upper[plane] else t


def continuum_spinor(dims: int, k: Sequence[float], m: float) -> np.ndarray:
    """Positive-energy free spinor of the continuum Dirac Hamiltonian with
    momentum k (standard representation, Sect. 2; Sect. 3 for 2 components)."""
    kx, ky = float(k[0]), float(k[1])
    kz = float(k[2]) if dims == 3 else 0.0
    E = math.sqrt(m * m + kx * kx + ky * ky + kz * kz)
    if E + m == 0.0:
        w = np.array([1, 0, 0, 0], complex) if dims == 3 else np.array([1, 1], complex)
    elif dims == 3:
        w = np.array([1.0, 0.0, kz / (E + m), (kx + 1j * ky) / (E + m)], complex)
    else:
        w = np.array([E + m, kx + 1j * ky], complex)
    return w / np.linalg.norm(w)


def gaussian_packet(prob: Problem, sigma: float, k0: Sequence[float], center: Sequence[float],
                    t: float = 0.0) -> np.ndarray:
    """Gaussian packet exp(-|x-xc|^2/(2 sigma^2)) times the continuum plane
    wave w(k0) exp(i(k0.x - E t_sheet)), sampled at every value's own
    position and time sheet, periodic (minimum image) and normalised to
    sum |psi|^2 = 1."""
    dims = prob.dims
    k = [float(v) for v in k0] + [0.0] * (3 - len(k0))
    E = math.sqrt(prob.m ** 2 + k[0] ** 2 + k[1] ** 2 + (k[2] ** 2 if dims == 3 else 0.0))
    w = continuum_spinor(dims, k, prob.m)
    _, _, _, comp = plane_tables(dims)
    L = [prob.N[a] * prob.dx[a] for a in range(3 if dims == 3 else 2)]
    out = np.zeros(prob.shape, np.complex128)
    for pl in range(prob.n_planes):
        xyz = site_positions(prob, pl)
        r2 = np.zeros(xyz[0].shape)
        phase = np.zeros(xyz[0].shape)
        for a in range(dims):
            d = xyz[a] - center[a]
            d = d - L[a] * np.round(d / L[a])
            r2 += d * d
            phase += k[a] * xyz[a]
        ts = sheet_time(prob, pl, t)
        out[pl] = w[comp[pl]] * np.exp(-r2 / (2 * sigma * sigma)) * np.exp(1j * (phase - E * ts))
    out /= math.sqrt(float(np.sum(np.abs(out) ** 2)))
    return out


def gaussian_packet_separable(prob: Problem, sigma: float, k0: Sequence[float], center: Sequence[float],
                              out: Optional[np.ndarray] = None, t: float = 0.0,
                              origin: Sequence[int] = (0, 0, 0), box: Optional[Sequence[int]] = None,
                              normalise: bool = True) -> np.ndarray:
    """The packet of gaussian_packet, built as a product of one-dimensional
    factors per axis (the Gaussian and the plane wave both separate), so a
    512^3 state (17 GB) is written plane by plane into `out` (complex128,
    shape prob.shape; allocated if None) without full-size temporaries.
    origin (cells) places the grid inside a periodic box of `box` cells per
    axis (default: the grid itself) for a window of a larger workload; the
    minimum-image distance is taken in that box.  Values agree with
    gaussian_packet to rounding (products of factors instead of one
    exponential)."""
    dims = prob.dims
    k = [float(v) for v in k0] + [0.0] * (3 - len(k0))
    E = math.sqrt(prob.m ** 2 + k[0] ** 2 + k[1] ** 2 + (k[2] ** 2 if dims == 3 else 0.0))
    w = continuum_spinor(dims, k, prob.m)
    _, offs, _, comp = plane_tables(dims)
    B = list(box) if box is not None else list(prob.N)
    L = [B[a] * prob.dx[a] for a in range(dims)]
    nz = prob.N[2] if dims == 3 else 1
    if out is None:
        out = np.empty(prob.shape, np.complex128)
    for pl in range(prob.n_planes):
        o = offs[pl]
        fac = []
        for a, n in enumerate((prob.N[0], prob.N[1], nz)):
            if a >= dims:
                fac.append(np.ones(1, np.complex128))
                continue
            x = (np.arange(n) + origin[a] + 0.5 * o[a]) * prob.dx[a]
            d = x - center[a]
            d = d - L[a] * np.round(d / L[a])
            fac.append(np.exp(-d * d / (2 * sigma * sigma)) * np.exp(1j * k[a] * x))
        ts = sheet_time(prob, pl, t)
        fz = fac[2] * (w[comp[pl]] * np.exp(-1j * E * ts))
        fyx = np.multiply.outer(fac[1], fac[0])
        for z in range(nz):
            np.multiply(fyx, fz[z], out=out[pl, z])
    if normalise:
        out /= math.sqrt(float(np.vdot(out.reshape(-1), out.reshape(-1)).real))
    return out


def gaussian_packet_torch(prob: Problem, sigma: float, k0: Sequence[float], center: Sequence[float],
                          device, t: float = 0.0):
    """The same packet as gaussian_packet, built plane by plane with torch in
    complex128 on `device` (for grids whose host copy would be tens of GB).
    Returns a tensor of shape (P, Nz, Ny, Nx)."""
    import torch
    dims = prob.dims
    k = [float(v) for v in k0] + [0.0] * (3 - len(k0))
    E = math.sqrt(prob.m ** 2 + k[0] ** 2 + k[1] ** 2 + (k[2] ** 2 if dims == 3 else 0.0))
    w = continuum_spinor(dims, k, prob.m)
    _, offs, _, comp = plane_tables(dims)
    L = [prob.N[a] * prob.dx[a] for a in range(3 if dims == 3 else 2)]
    nz = prob.N[2] if dims == 3 else 1
    out = torch.empty(prob.shape, dtype=torch.complex128, device=device)
    axes = [torch.arange(n, dtype=torch.float64, device=device) for n in (prob.N[0], prob.N[1], nz)]
    for pl in range(prob.n_planes):
        o = offs[pl]
        r2 = torch.zeros((nz, prob.N[1], prob.N[0]), dtype=torch.float64, device=device)
        phase = torch.zeros_like(r2)
        for a in range(dims):
            c = (axes[a] + 0.5 * o[a]) * prob.dx[a]
            d = c - center[a]
            d = d - L[a] * torch.round(d / L[a])
            shape = [1, 1, 1]
            shape[2 - a] = -1
            r2 = r2 + (d * d).view(shape)
            phase = phase + (k[a] * c).view(shape)
        ts = sheet_time(prob, pl, t)
        amp = torch.exp(-r2 / (2 * sigma * sigma))
        out[pl] = complex(w[comp[pl]]) * torch.polar(amp, phase - E * ts)
    out /= math.sqrt(float(torch.sum(torch.abs(out) ** 2)))
    return out


def random_state(prob: Problem, seed: int) -> np.ndarray:
    """Uniformly random complex values (PCG64), normalised to sum |psi|^2 = 1."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(prob.shape)
    im = rng.standard_normal(prob.shape)
    out = (re + 1j * im).astype(np.complex128)
    out /= math.sqrt(float(np.sum(np.abs(out) ** 2)))
    return out


def random_potential(prob: Problem, seed: int, amplitude: float) -> np.ndarray:
    """Static real potential, one value per site, uniform in [-a, a]."""
    rng = np.random.default_rng(seed)
    return amplitude * (2.0 * rng.random(prob.shape) - 1.0)


def half_lattice_points(prob: Problem, plane: int):
    """Integer half-lattice coordinates (X, Y, Z) (units of dx/2) of every
    value of a plane, each an int array of shape (Nz, Ny, Nx); Z = 0 in
    (2+1)D."""
    _, offs, _, _ = plane_tables(prob.dims)
    o = offs[plane]
    nz = prob.N[2] if prob.dims == 3 else 1
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(prob.N[1]), np.arange(prob.N[0]), indexing="ij")
    Z = 2 * jz + o[2] if prob.dims == 3 else np.zeros_like(jx)
    return 2 * jx + o[0], 2 * jy + o[1], Z


def link_integrals(prob: Problem, fn) -> np.ndarray:
    """An A_links array (dims, P, Nz, Ny, Nx) from fn(a, S, E) -> array: the
    value for the link along axis a from the half-lattice points S to E = S +
    e_a (coordinate tuples as from half_lattice_points; E wraps at the far
    face)."""
    M = [2 * prob.N[a] if a < prob.dims else 1 for a in range(3)]
    out = np.zeros((prob.dims,) + tuple(prob.shape))
    for pl in range(prob.n_planes):
        S = half_lattice_points(prob, pl)
        for a in range(prob.dims):
            E = list(S)
            E[a] = (S[a] + 1) % M[a]
            out[a, pl] = fn(a, S, tuple(E))
    return out


def random_links(prob: Problem, seed: int, amplitude: float) -> np.ndarray:
    """Link integrals of an arbitrary (not pure gauge) static vector
    potential, uniform in [-a, a] per link."""
    rng = np.random.default_rng(seed)
    return amplitude * (2.0 * rng.random((prob.dims,) + tuple(prob.shape)) - 1.0)


def random_lattice_gauge(prob: Problem, seed: int, amplitude: float) -> np.ndarray:
    """A random real function chi on the half lattice, shape (2Nz or 1, 2Ny,
    2Nx), uniform in [-a, a]; its lattice gradient chi(E) - chi(S) is a pure
    gauge."""
    M = [2 * prob.N[a] if a < prob.dims else 1 for a in range(3)]
    rng = np.random.default_rng(seed)
    return amplitude * (2.0 * rng.random((M[2], M[1], M[0])) - 1.0)


def delta_state(prob: Problem, plane: int, cell: Sequence[int]) -> np.ndarray:
    """A single unit value at one site."""
    out = np.zeros(prob.shape, np.complex128)
    jz = cell[2] if prob.dims == 3 else 0
    out[plane, jz, cell[1], cell[0]] = 1.0
    return out


def random_k0(seed: int) -> np.ndarray:
    """k0 = u*d with d uniform on the unit sphere and u ~ U[0,1] (PCG64)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    return rng.random() * d


# --------------------------------------------------------------------------
# The workloads.  dt = 0.9 x the stability limit for every one of them.

def workload_2d64(m: float = 0.0):
    """(2+1)D, 64^2 periodic, dx = 1, packet sigma = 6, k0 = (0.5, 0) centred
    at (32, 32); 200 steps, FP64."""
    N = 64
    prob = Problem(2, (N, N, 1), (1.0, 1.0, 1.0), 0.9 * stability_limit(2), m)
    psi = gaussian_packet(prob, 6.0, (0.5, 0.0), (32.0, 32.0))
    return prob, psi, 200


def workload_3d(N: int = 128, steps: int = 1000, seed: int = 0, m: float = 1.0, sigma: float = 10.0,
                packet: bool = True):
    """(3+1)D, N^3 periodic, m = 1, no fields, packet sigma = 10 at the box
    centre with seeded k0 (|k0| <= 1).  packet=False: no state (None)."""
    prob = Problem(3, (N, N, N), (1.0, 1.0, 1.0), 0.9 * stability_limit(3), m)
    c = N / 2.0
    psi = gaussian_packet(prob, sigma, random_k0(seed), (c, c, c)) if packet else None
    return prob, psi, steps


def klein_fields(N: int, m: float, k0x: float) -> Fields:
    """Klein step along x at x0 = N/2 + 1/4 (no site on the step) with height
    V0 = 2 E + m, E the continuum packet energy sqrt(m^2 + k0^2)."""
    E = math.sqrt(m * m + k0x * k0x)
    return Fields(step_axis=0, step_x0=N / 2.0 + 0.25, step_V=2.0 * E + m)


def workload_klein(N: int = 4096, steps: int = 5000, m: float = 0.2, sigma: float = 40.0):
    """(2+1)D Klein-step scattering: packet at (N/4, N/2), k0 = (0.25, 0)
    (normal incidence), step at x0 = N/2 + 1/4."""
    k0 = (0.25, 0.0)
    prob = Problem(2, (N, N, 1), (1.0, 1.0, 1.0), 0.9 * stability_limit(2), m,
                   klein_fields(N, m, k0[0]))
    psi = gaussian_packet(prob, sigma, k0, (N / 4.0, N / 2.0))
    return prob, psi, steps


def workload_klein_oblique(N: int = 4096, steps: int = 3000, sigma: float = 64.0, kabs: float = 0.25,
                           angle_to_step_deg: float = 37.0, offset: float = 4.0):
    """(2+1)D Klein refraction (Sect. 5, the oblique-incidence example): m = 0,
    step height V = 2E (E = |k0|, the continuum packet energy) at x0 = N/2 + 1/4,
    a packet whose momentum makes angle_to_step_deg with the step (the y-axis),
    i.e. an incidence angle of 90 - angle_to_step_deg from the step's normal,
    centred offset*sigma before the step along its direction of motion."""
    inc = math.radians(90.0 - angle_to_step_deg)
    k0 = (kabs * math.cos(inc), kabs * math.sin(inc))
    x0 = N / 2.0 + 0.25
    f = Fields(step_axis=0, step_x0=x0, step_V=2.0 * kabs)
    prob = Problem(2, (N, N, 1), (1.0, 1.0, 1.0), 0.9 * stability_limit(2), 0.0, f)
    c = (x0 - offset * sigma * math.cos(inc), N / 2.0 - offset * sigma * math.sin(inc))
    psi = gaussian_packet(prob, sigma, k0, c)
    return prob, psi, steps


def workload_links(dims: int = 3, N: int = 128, steps: int = 200, seed: int = 2, amplitude: float = 0.3):
    """A static vector potential given only by its link integrals (Sect. 4),
    drawn uniformly in [-a, a] per link (seeded), q = 1, m = 1, on the
    periodic (3+1)D or (2+1)D grid of the free workloads with their packet."""
    if dims == 3:
        prob, psi, _ = workload_3d(N=N, steps=steps)
    else:
        prob = Problem(2, (N, N, 1), (1.0, 1.0, 1.0), 0.9 * stability_limit(2), 1.0)
        psi = gaussian_packet(prob, 10.0, tuple(random_k0(0))[:2], (N / 2.0, N / 2.0))
    prob = prob.with_fields(q=1.0, A_links=random_links(prob, seed, amplitude))
    return prob, psi, steps


def laser_fields(N: int) -> Fields:
    """Soft-core potential -1/sqrt(|x-c|^2 + 1) at the box centre plus a plane
    wave A_x = 0.5 cos(2 pi z / 64 - omega t), omega = 2 pi / 64."""
    c = N / 2.0
    w = 2.0 * math.pi / 64.0
    return Fields(sc_Z=1.0, sc_a=1.0, sc_center=(c, c, c), q=1.0,
                  Apw_amp=0.5, Apw_k=(0.0, 0.0, w), Apw_omega=w, Apw_pol=0)


def workload_laser(N: int = 512, steps: int = 2000, seed: int = 1, sigma: float = 24.0, packet: bool = True):
    """(3+1)D, m = 1, soft core + time-dependent vector potential.
    packet=False: no state (None; large grids build theirs in place)."""
    prob = Problem(3, (N, N, N), (1.0, 1.0, 1.0), 0.9 * stability_limit(3), 1.0, laser_fields(N))
    c = N / 2.0
    psi = gaussian_packet(prob, sigma, random_k0(seed), (c, c, c)) if packet else None
    return prob, psi, steps
