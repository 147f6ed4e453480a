"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (relative L2 over the whole state, and E):
  FP64: 1e-12 (rounding-order differences only);
  FP32: 1e-5 rel L2 and 1e-6 relative drift of E (compensated coefficients).
Sizes span several thread blocks and ragged tails (N not a multiple of any
tile), both dimensions, all field paths.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W
from tests import closed_forms as CF

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5
FP32_EDRIFT = 1e-6


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_gpu(D, prob, psi, n, precision, t0=0.0, chunks=1):
    with D.Sim(prob, precision) as s:
        s.time = t0
        s.set_spinor(psi)
        E0, _ = s.norm()
        for c in range(chunks):
            s.step(n // chunks + (1 if c < n % chunks else 0))
        E1, naive = s.norm()
        out = s.get_spinor()
        t = s.time
    return out, E0, E1, naive, t


def field_cases(dims, N):
    c = [n / 2.0 for n in N]
    L = [float(n) for n in N]
    cases = {
        "free": W.Fields(),
        "V0": W.Fields(V0=0.37),
        "klein": W.Fields(V0=0.05, step_axis=0, step_x0=N[0] / 2 + 0.25, step_V=0.8),
        "klein_y": W.Fields(step_axis=1, step_x0=N[1] / 3 + 0.25, step_V=-0.6),
        "softcore": W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=tuple(c)),
        "A_const": W.Fields(q=0.8, A_const=(0.3, -0.45, 0.2)),
        "A_wave": W.Fields(q=1.0, Apw_amp=0.5, Apw_k=(0, 0, 2 * math.pi / L[dims - 1]) if dims == 3
                           else (0, 2 * math.pi / L[1], 0), Apw_omega=0.3, Apw_pol=0),
        "A_wave_long": W.Fields(q=1.0, Apw_amp=0.4, Apw_k=(2 * math.pi / L[0], 0, 0),
                                Apw_omega=0.0, Apw_pol=0, Apw_phase=0.3),
        # soft core off the half lattice, with a Klein step
        "softcore_offgrid": W.Fields(sc_Z=0.8, sc_a=1.3, sc_center=(c[0] - 0.37, c[1] + 0.61, 2.13),
                                     V0=-0.1, step_axis=1, step_x0=N[1] / 2 + 0.25, step_V=0.3),
        # a deep soft core: |theta| > 1 near the centre
        "softcore_deep": W.Fields(sc_Z=4.0, sc_a=0.5, sc_center=tuple(c)),
        # absorbing layers on every face plus a uniform imaginary part (Sect. 3)
        "absorb": W.Fields(V0=0.05, V0_imag=-0.02, abs_W=0.7, abs_width=3.0, abs_axes=(1 << dims) - 1),
        # the laser workload's fields: soft core plus a moving plane wave
        "laser": W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=tuple(c), q=1.0, Apw_amp=0.5,
                          Apw_k=(0, 0, 2 * math.pi / L[dims - 1]) if dims == 3 else (0, 2 * math.pi / L[1], 0),
                          Apw_omega=0.4, Apw_pol=0),
    }
    return cases


@pytest.mark.parametrize("dims,N", [(2, (37, 29)), (3, (13, 11, 9))])
@pytest.mark.parametrize("case", ["free", "V0", "klein", "klein_y", "softcore", "A_const", "A_wave",
                                  "A_wave_long", "Vstatic", "Vstatic_mod", "softcore_offgrid", "softcore_deep",
                                  "laser", "absorb"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parity_fields(D, dims, N, case, precision):
    full = tuple(N) + ((1,) if dims == 2 else ())
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.45)
    if case == "Vstatic_mod":
        f = W.Fields(V_static=W.random_potential(prob, 4, 0.6), Vmod_amp=0.5, Vmod_omega=0.7)
    elif case == "Vstatic":  # time-independent: tabulated theta in FP32
        f = W.Fields(V_static=W.random_potential(prob, 4, 0.6), sc_Z=0.5, sc_a=1.5, sc_center=(3.0, 4.5, 2.0))
    else:
        f = field_cases(dims, N)[case]
    prob = W.Problem(prob.dims, prob.N, prob.dx, prob.dt, prob.m, f)
    psi = W.random_state(prob, 17)
    n = 60
    t0 = 0.25
    ref = O.step(prob, psi, n, t0)
    ob0 = O.observables(prob, psi, t0)
    ob1 = O.observables(prob, ref, t0 + n * prob.dt)
    prec = D.FP64 if precision == "fp64" else D.FP32
    out, E0, E1, naive, t = run_gpu(D, prob, psi, n, prec, t0, chunks=3)
    assert abs(t - (t0 + n * prob.dt)) < 1e-12
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert rel(out, ref) < tol
    if precision == "fp64":
        assert abs(E0 - ob0["E"]) < 1e-13 * abs(ob0["E"])
        assert abs(E1 - ob1["E"]) < 1e-12 * abs(ob1["E"])
        assert abs(naive - ob1["naive"]) < 1e-12 * ob1["naive"]
    else:
        assert abs(E1 - ob1["E"]) < 1e-5 * abs(ob1["E"])
        if case not in ("A_wave", "laser", "absorb"):  # time-dependent A, absorption: E not conserved
            assert abs(E1 - E0) < FP32_EDRIFT * abs(E0)


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_anisotropic_grid(D, dims, precision):
    if dims == 2:
        prob = W.Problem(2, (21, 18, 1), (1.0, 1.3, 1.0), 0.5, 0.3, W.Fields(V0=0.1))
    else:
        prob = W.Problem(3, (10, 12, 7), (1.0, 1.2, 0.9), 0.45, 0.3, W.Fields(V0=0.1))
    psi = W.random_state(prob, 3)
    ref = O.step(prob, psi, 40)
    out, E0, E1, _, _ = run_gpu(D, prob, psi, 40, D.FP64 if precision == "fp64" else D.FP32)
    assert rel(out, ref) < (FP64_TOL if precision == "fp64" else FP32_TOL)
    assert abs(E1 - E0) < (1e-13 if precision == "fp64" else FP32_EDRIFT) * abs(E0)


@pytest.mark.parametrize("m", [0.0, 0.5])
def test_workload_2d64_fp64(D, m):
    """(2+1)D 64^2 packet, 200 steps, FP64: parity with the oracle and
    conservation of E."""
    prob, psi, n = W.workload_2d64(m)
    ref = O.step(prob, psi, n)
    out, E0, E1, _, _ = run_gpu(D, prob, psi, n, D.FP64)
    assert rel(out, ref) < FP64_TOL
    assert abs(E1 - E0) < 1e-13 * E0


@pytest.mark.parametrize("dims,modes,m", [(2, (5, 3), 0.5), (3, (2, -1, 3), 1.0)])
def test_plane_wave_closed_form(D, dims, modes, m):
    """Eq. pwdsip on the GPU: a lattice plane wave advances by exp(-i w n dt)."""
    if dims == 2:
        prob = W.Problem(2, (64, 64, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), m)
        n = 200
    else:
        prob = W.Problem(3, (16, 12, 20), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), m)
        n = 100
    psi, w = CF.plane_wave_state(prob, modes)
    out, _, _, _, _ = run_gpu(D, prob, psi, n, D.FP64)
    assert rel(out, psi * np.exp(-1j * w * n * prob.dt)) < 1e-12
    out32, _, _, _, _ = run_gpu(D, prob, psi, n, D.FP32)
    assert rel(out32, psi * np.exp(-1j * w * n * prob.dt)) < FP32_TOL


def test_observables_match_oracle(D):
    prob = W.Problem(3, (9, 10, 11), (1.0, 1.0, 1.0), 0.5, 0.2,
                     W.Fields(q=0.9, A_const=(0.2, 0.1, -0.3)))
    psi = W.random_state(prob, 8)
    with D.Sim(prob, D.FP64) as s:
        s.set_spinor(psi)
        E, naive = s.norm()
        pd = s.partial_density(1, 4.6)
        back = s.get_spinor()
    ob = O.observables(prob, psi, 0.0)
    assert np.array_equal(back, psi)
    assert abs(E - ob["E"]) < 1e-14 * abs(ob["E"])
    assert abs(naive - ob["naive"]) < 1e-14
    assert abs(pd - O.partial_density(prob, psi, 1, 4.6)) < 1e-14


def test_fp32_roundtrip_is_float_rounding(D):
    prob = W.Problem(2, (33, 17, 1), (1.0, 1.0, 1.0), 0.5, 0.0)
    psi = W.random_state(prob, 2)
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        back = s.get_spinor()
    want = psi.real.astype(np.float32).astype(np.float64) + 1j * psi.imag.astype(np.float32)
    assert np.array_equal(back, want)


def test_light_cone_on_gpu(D):
    """Nearest-neighbour stencil: exact zeros outside the light cone (catches
    wrong neighbour offsets and wrap-around mistakes at block edges)."""
    prob = W.Problem(3, (40, 36, 20), (1.0, 1.0, 1.0), 0.5, 0.5)
    for plane, cell in ((0, (0, 0, 0)), (5, (39, 35, 19)), (7, (17, 20, 10))):
        psi = W.delta_state(prob, plane, cell)
        n = 3
        out, _, _, _, _ = run_gpu(D, prob, psi, n, D.FP64)
        ref = O.step(prob, psi, n)
        assert rel(out, ref) < FP64_TOL
        _, offs, _, _ = W.plane_tables(3)
        so = [2 * cell[a] + offs[plane][a] for a in range(3)]
        L = [2 * prob.N[a] for a in range(3)]
        for pl in range(prob.n_planes):
            xyz = W.site_positions(prob, pl)
            dist = 0
            for a in range(3):
                d = np.abs(2 * xyz[a] - so[a])
                dist = dist + np.minimum(d, L[a] - d)  # periodic half-lattice distance
            assert np.all(out[pl][dist > 2 * n] == 0.0)


def test_unstable_is_rejected_and_diverges_when_forced(D):
    prob = W.Problem(2, (8, 8, 1), (1.0, 1.0, 1.0), 1.2 * W.stability_limit(2), 0.3)
    with pytest.raises(D.DiracError) as e:
        D.Sim(prob, D.FP64)
    assert e.value.status == D.ERR_UNSTABLE
    psi = W.random_state(prob, 1)
    with D.Sim(prob, D.FP64, flags=D.FLAG_ALLOW_UNSTABLE) as s:
        s.set_spinor(psi)
        E0, _ = s.norm()
        s.step(4000)
        try:
            E1, naive = s.norm()
            grew = not math.isfinite(naive) or naive > 1e6
        except D.DiracError as err:
            grew = err.status == D.ERR_DIVERGED
    assert grew


@pytest.mark.parametrize("dims,N", [(2, (37, 29)), (2, (64, 70)), (3, (13, 11, 9)), (3, (33, 17, 20)),
                                    (3, (2, 3, 2)), (3, (33, 27, 5)), (3, (40, 53, 3))])
@pytest.mark.parametrize("case", ["free", "klein", "klein_y", "softcore", "A_const", "A_wave",
                                  "A_wave_long", "Vstatic", "Vstatic_mod", "softcore_offgrid", "softcore_deep",
                                  "laser", "absorb"])
def test_fused_kernel_bit_identical_to_reference_kernels(D, dims, N, case):
    """The fused time-step kernel (out of place, tiles with recomputed halos,
    z/y marching) uses the same per-value arithmetic as the one-kernel-per-
    half-step path, so the FP32 states agree bit for bit, for every field
    path, ragged tiles and grids smaller than one tile (the (3+1)D tiles hold
    32 x 26 interior cells: 27 and 53 rows leave a last tile of one row)."""
    full = tuple(N) + ((1,) if dims == 2 else ())
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.45)
    if case == "Vstatic_mod":
        f = W.Fields(V_static=W.random_potential(prob, 4, 0.6), Vmod_amp=0.5, Vmod_omega=0.7)
    elif case == "Vstatic":
        f = W.Fields(V_static=W.random_potential(prob, 4, 0.6))
    else:
        f = field_cases(dims, N)[case]
    prob = W.Problem(prob.dims, prob.N, prob.dx, prob.dt, prob.m, f)
    psi = W.random_state(prob, 23)
    outs = []
    for flags in (0, D.FLAG_REFERENCE_KERNELS):
        with D.Sim(prob, D.FP32, flags=flags) as s:
            s.time = 0.1
            s.set_spinor(psi)
            s.step(7)
            s.step(10)
            outs.append(s.get_spinor())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("dims,precision", [(3, "fp32"), (2, "fp32"), (3, "fp64"), (2, "fp64")])
def test_graph_replay_bit_identical_to_plain_launches(D, dims, precision, monkeypatch):
    """Step loops of time-independent fields replay captured CUDA graphs of
    64 steps; the result must equal plain launches bit for bit, for both
    buffer parities (odd step counts in between)."""
    N = (30, 20, 18) if dims == 3 else (70, 50, 1)
    prob = W.Problem(dims, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.6,
                     W.Fields(step_axis=0, step_x0=N[0] / 2 + 0.25, step_V=0.5))
    psi = W.random_state(prob, 5)
    prec = D.FP64 if precision == "fp64" else D.FP32
    outs = []
    for no_graphs in (False, True):
        if no_graphs:
            monkeypatch.setenv("DIRAC_NO_GRAPHS", "1")
        with D.Sim(prob, prec) as s:
            s.set_spinor(psi)
            s.step(150)
            s.step(3)
            s.step(131)
            launches = s.launches
            outs.append(s.get_spinor())
        monkeypatch.delenv("DIRAC_NO_GRAPHS", raising=False)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("N", [(70, 50), (29, 31), (5, 9), (129, 64)])
@pytest.mark.parametrize("case", ["free", "klein", "klein_y", "A_const", "softcore", "softcore_offgrid",
                                  "absorb"])
def test_temporal_blocking_2d_bit_identical(D, N, case, monkeypatch):
    """(2+1)D: two time steps per pass (step 2 runs one row behind step 1 in
    registers) equal two single-step passes bit for bit; odd step counts
    finish with a single-step pass."""
    prob = W.Problem(2, (N[0], N[1], 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.45,
                     field_cases(2, N)[case])
    psi = W.random_state(prob, 9)
    outs = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("DIRAC_NO_TEMPORAL_BLOCKING", "1")
        with D.Sim(prob, D.FP32) as s:
            s.set_spinor(psi)
            s.step(21)
            s.step(6)
            outs.append(s.get_spinor())
        monkeypatch.delenv("DIRAC_NO_TEMPORAL_BLOCKING", raising=False)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("dims,N", [(3, (33, 29, 21)), (2, (70, 45))])
@pytest.mark.parametrize("case", ["free", "klein", "A_const", "A_wave_long", "softcore", "laser"])
@pytest.mark.parametrize("nsteps", [7, 10])
def test_fused_functional_matches_reduction(D, dims, N, case, nsteps, monkeypatch):
    """The last fused launch of dirac_step accumulates E of the new state
    (sum |psi|^2 + r_x Re sum_lower conj(G) S'_G, with the S' its own lower
    half-step formed); it must equal the separate reduction of that state."""
    full = tuple(N) + ((1,) if dims == 2 else ())
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.45,
                     field_cases(dims, N)[case])
    psi = W.random_state(prob, 12)
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(nsteps)
        E_fused, n_fused = s.norm()
        monkeypatch.setenv("DIRAC_NO_FUSED_NORM", "1")
        E_red, n_red = s.norm()
        monkeypatch.delenv("DIRAC_NO_FUSED_NORM")
    assert abs(E_fused - E_red) <= 2e-7 * abs(E_red)
    assert abs(n_fused - n_red) <= 2e-7 * n_red


@pytest.mark.parametrize("dims,N", [(2, (36, 30)), (3, (24, 20, 22))])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_absorbing_layers_functional_never_grows(D, dims, N, precision):
    """Absorbing layers (Im V < 0 near the faces, Sect. 3): E computed after
    every step never grows and falls well below its start once a packet has
    run into a layer; the oracle agrees on the final state."""
    full = tuple(N) + ((1,) if dims == 2 else ())
    f = W.Fields(abs_W=0.8, abs_width=6.0, abs_axes=1)  # layers on the two x faces
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.2, f)
    c = [n / 2.0 for n in N]
    psi = W.gaussian_packet(prob, 3.0, (1.2,) + (0.0,) * (dims - 1), tuple(c))
    prec = D.FP64 if precision == "fp64" else D.FP32
    E = []
    with D.Sim(prob, prec) as s:
        s.set_spinor(psi)
        E.append(s.norm()[0])
        for _ in range(40):
            s.step(1)
            E.append(s.norm()[0])
        out = s.get_spinor()
    d = np.diff(E)
    slack = 1e-13 if precision == "fp64" else 2e-7
    assert np.all(d <= slack * E[0])
    assert E[-1] < 0.8 * E[0]
    ref = O.step(prob, psi, 40)
    assert rel(out, ref) < (FP64_TOL if precision == "fp64" else FP32_TOL)


@pytest.mark.parametrize("dims,axis", [(2, 0), (3, 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gauge_covariance_longitudinal_wave(D, dims, axis, precision):
    """Sect. 4: Peierls phases are line integrals of A, so a static
    longitudinal wave (a pure gauge) only multiplies the state by
    exp(i q chi), chi = (amp/k) sin(k x_a + ph), on the GPU too."""
    N = (24, 20, 18)
    prob = W.Problem(dims, N if dims == 3 else (24, 20, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.4)
    q, amp, ph = 0.8, 0.9, 0.35
    k = 2 * math.pi * 2 / (prob.N[axis] * prob.dx[axis])
    kvec = [0.0, 0.0, 0.0]
    kvec[axis] = k
    psi0 = W.random_state(prob, 4)
    gauge = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        x = W.site_positions(prob, pl)[axis]
        gauge[pl] = np.exp(1j * q * amp / k * np.sin(k * x + ph))
    prec = D.FP64 if precision == "fp64" else D.FP32
    out0, *_ = run_gpu(D, prob, psi0, 40, prec)
    fA = prob.with_fields(q=q, Apw_amp=amp, Apw_k=tuple(kvec), Apw_omega=0.0, Apw_phase=ph, Apw_pol=axis)
    outA, *_ = run_gpu(D, fA, gauge * psi0, 40, prec)
    assert rel(outA, gauge * out0) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_klein_negative_refraction(D, precision):
    """Sect. 5, oblique incidence (m = 0, V = 2E): the GPU state equals the
    oracle's, and the transmitted packet is refracted to negative angles with
    phase and group velocity opposed."""
    from tests import klein_refraction as K
    prob, psi, _ = W.workload_klein_oblique(N=384, sigma=16.0, kabs=0.5, offset=4.0)
    x0 = prob.fields.step_x0
    prec = D.FP64 if precision == "fp64" else D.FP32
    with D.Sim(prob, prec) as s:
        s.set_spinor(psi)
        s.step(250)
        p1 = s.get_spinor()
        s.step(100)
        p2 = s.get_spinor()
        T = s.partial_density(0, x0)
    ref = O.step(prob, psi, 350)
    assert rel(p2, ref) < (FP64_TOL if precision == "fp64" else FP32_TOL)
    v, part = K.velocity(prob, p1, p2, 100, x0)
    ang_t = math.degrees(math.atan2(v["T"][1], v["T"][0]))
    assert -60.0 < ang_t < -40.0
    kt = part["T"][2]
    assert kt @ v["T"] / (np.linalg.norm(kt) * np.linalg.norm(v["T"])) < -0.9
    assert abs(T - part["T"][0]) < 1e-6


def test_algorithmic_bytes_per_path(D, monkeypatch):
    """dirac_algorithmic_bytes: the state read and written once per step,
    plus one 16-byte coefficient per value read with a tabulated potential,
    or one FP64 potential value with the per-site FP64 path."""
    p3 = W.Problem(3, (12, 10, 8), (1.0, 1.0, 1.0), 0.5, 0.3)
    p2 = W.Problem(2, (20, 18, 1), (1.0, 1.0, 1.0), 0.5, 0.3)
    soft = W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=(6.0, 5.0, 4.0))
    soft2 = W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=(10.0, 9.0, 0.0))
    absorb = W.Fields(V0_imag=-0.01, abs_W=0.2, abs_width=2.0, abs_axes=1)
    cases = [(p3, D.FP32, 128.0), (p2, D.FP32, 64.0), (p3, D.FP64, 256.0),
             (p3.with_fields(**vars(absorb)), D.FP32, 128.0 + 128.0),
             (p3.with_fields(step_axis=0, step_x0=6.25, step_V=0.5), D.FP32, 128.0)]
    vstat = p3.with_fields(V_static=W.random_potential(p3, 1, 0.3), Vmod_amp=0.2, Vmod_omega=0.5)
    cases.append((vstat, D.FP64, 256.0 + 64.0))
    for prob, prec, want in cases:
        with D.Sim(prob, prec) as s:
            assert s.algorithmic_bytes == want, (prob.fields, prec)
    # the soft core's evaluations: analytic (the default, nothing per site),
    # FP32 estimate with a 4-byte correction per value, per-site table (16 bytes)
    for how, extra in (("analytic", 0.0), ("corrected", 4.0), ("table", 16.0)):
        monkeypatch.setenv("DIRAC_SOFTCORE", how)
        for prob, np_ in ((p3.with_fields(**vars(soft)), 8), (p2.with_fields(**vars(soft2)), 4)):
            with D.Sim(prob, D.FP32) as s:
                assert s.algorithmic_bytes == 16.0 * np_ + extra * np_, how


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_degenerate_inputs(D, dims, precision):
    """Empty and degenerate work: zero steps change nothing, an empty batch is
    a no-op, the zero state stays zero with E = 0 and passes the stability
    check, and the smallest grid (two cells per axis) matches the oracle."""
    prec = D.FP64 if precision == "fp64" else D.FP32
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    N = (2, 2, 1) if dims == 2 else (2, 2, 2)
    prob = W.Problem(dims, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.6,
                     W.Fields(step_axis=0, step_x0=1.25, step_V=0.4))
    psi = W.random_state(prob, 31)
    with D.Sim(prob, prec) as s:
        s.set_spinor(psi)
        t0, launches = s.time, s.launches
        s.step(0)
        D.batch_step([s], 0)
        D.batch_step([], 5)
        assert s.time == t0 and s.launches == launches
        back = s.get_spinor()
        assert rel(back, psi) < (1e-15 if precision == "fp64" else 2e-7)
        s.step(25)
        assert rel(s.get_spinor(), O.step(prob, psi, 25)) < tol
    with D.Sim(W.Problem(dims, (9, 7, 5) if dims == 3 else (9, 7, 1), (1.0, 1.0, 1.0), 0.5, 0.3), prec) as z:
        z.set_spinor(np.zeros(z.prob.shape, complex))
        z.step(12)
        E, naive = z.norm()
        ok, r = z.check(1e-6)
        assert E == 0.0 and naive == 0.0 and ok and r["failed"] == 0
        assert not np.any(z.get_spinor())
