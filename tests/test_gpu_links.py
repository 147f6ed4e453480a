"""Arbitrary vector potentials given by their link integrals (Sect. 4: the
Peierls phase of a link is q times the line integral of A along it), on the
GPU through the C ABI.

* Parity with the FP64 oracle for random static links and for links with a
  cos(omega t) modulation, on top of a random scalar potential and a constant
  A: FP64 within 1e-12, FP32 within 1e-5 (relative L2 over the state).
* Exact gauge covariance under a random lattice gauge function chi:
  psi_A(t) = exp(i q chi) psi_0(t).
* The functional E stays conserved with static links (FP32 drift below
  1e-6, dirac_check passes) and the fused FP32 kernels agree bit for bit
  with the one-kernel-per-half-step path (static links: FP32 link factors
  tabulated once per simulation; modulated links: per-site FP64 phases).
"""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(dims, N, moving, seed=3, link_amp=0.7):
    full = tuple(N) + ((1,) if dims == 2 else ())
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.45)
    f = dict(V_static=W.random_potential(prob, seed, 0.5), q=0.8, A_const=(0.2, -0.3, 0.1),
             A_links=W.random_links(prob, seed + 1, link_amp))
    if moving:
        f.update(Alink_amp=0.6, Alink_omega=0.9)
    return prob.with_fields(**f)


@pytest.mark.parametrize("dims,N", [(2, (37, 29)), (3, (13, 11, 9))])
@pytest.mark.parametrize("moving", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parity_link_integrals(D, dims, N, moving, precision):
    prob = problem(dims, N, moving)
    psi = W.random_state(prob, 17)
    n, t0 = 60, 0.25
    ref = O.step(prob, psi, n, t0)
    ob0 = O.observables(prob, psi, t0)
    ob1 = O.observables(prob, ref, t0 + n * prob.dt)
    prec = D.FP64 if precision == "fp64" else D.FP32
    with D.Sim(prob, prec) as s:
        s.time = t0
        s.set_spinor(psi)
        E0, _ = s.norm()
        for k in (25, 35):
            s.step(k)
        E1, naive = s.norm()
        out = s.get_spinor()
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rel(out, ref) < tol
    if precision == "fp64":
        assert abs(E0 - ob0["E"]) < 1e-13 * abs(ob0["E"])
        assert abs(E1 - ob1["E"]) < 1e-12 * abs(ob1["E"])
        assert abs(naive - ob1["naive"]) < 1e-12 * ob1["naive"]
    else:
        # the functional of the GPU's own final state: FP32 terms of the size of
        # |psi|^2 summed in FP64, so within 1e-6 of sum |psi|^2.  (Against the
        # oracle's final state E would also carry the state's own error, which a
        # moving field does not conserve and which sum |psi|^2 / E amplifies.)
        own = O.observables(prob, out, t0 + n * prob.dt)
        assert abs(E1 - own["E"]) < 1e-6 * own["naive"]
        assert abs(naive - own["naive"]) < 1e-6 * own["naive"]
    if not moving:  # static links: E conserved (Lemma of Sect. 2)
        assert abs(E1 - E0) < (1e-13 if precision == "fp64" else 1e-6) * abs(E0)
    else:  # a moving field does work on the state: the oracle's E changes too
        assert abs(ob1["E"] - ob0["E"]) > 1e-6 * abs(ob0["E"])


@pytest.mark.parametrize("dims,N", [(2, (24, 20)), (3, (12, 10, 9))])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gauge_covariance_lattice_gauge(D, dims, N, precision):
    full = tuple(N) + ((1,) if dims == 2 else ())
    prob = W.Problem(dims, full, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.4)
    prob = prob.with_fields(V_static=W.random_potential(prob, 5, 0.4))
    q = 0.9
    chi = W.random_lattice_gauge(prob, 12, 3.0)
    at = lambda P: chi[P[2], P[1], P[0]]
    gauge = np.zeros(prob.shape, complex)
    for pl in range(prob.n_planes):
        gauge[pl] = np.exp(1j * q * at(W.half_lattice_points(prob, pl)))
    pA = prob.with_fields(q=q, A_links=W.link_integrals(prob, lambda a, S, E: at(E) - at(S)))
    psi0 = W.random_state(prob, 13)
    prec = D.FP64 if precision == "fp64" else D.FP32
    outs = []
    for p, psi in ((prob, psi0), (pA, gauge * psi0)):
        with D.Sim(p, prec) as s:
            s.set_spinor(psi)
            s.step(40)
            outs.append(s.get_spinor())
    assert rel(outs[1], gauge * outs[0]) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("dims,N", [(2, (37, 29)), (2, (64, 70)), (3, (13, 11, 9)), (3, (33, 17, 20))])
@pytest.mark.parametrize("moving", [False, True])
def test_fused_bit_identical_to_reference_kernels(D, dims, N, moving):
    prob = problem(dims, N, moving, seed=8)
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


@pytest.mark.parametrize("dims,N", [(2, (40, 36)), (3, (16, 14, 12))])
def test_check_and_bytes_with_links(D, dims, N):
    prob = problem(dims, N, False, seed=11, link_amp=0.3)
    P = prob.n_planes
    # FP64: state (16 B each way per value), the static potential (8 B), the
    # up and down link integral per axis (16 B) read by the per-site path
    with D.Sim(prob, D.FP64) as s:
        assert s.algorithmic_bytes == 2 * P * 16 + 8 * P + 16 * dims * P
    # FP32 with a modulation: the per-site path as well (coefficient table 16 B)
    with D.Sim(problem(dims, N, True, seed=11, link_amp=0.3), D.FP32) as s:
        assert s.algorithmic_bytes == 2 * P * 8 + 16 * P + 16 * dims * P
    with D.Sim(prob, D.FP32) as s:
        # static links in FP32: the tabulated factors, up and down link per axis as
        # hi + lo complex floats (32 B per axis and value)
        assert s.algorithmic_bytes == 2 * P * 8 + 16 * P + 32 * dims * P
        # a smooth packet, as in the workloads the 1e-6 drift bound is quoted on
        # (a white-noise state under white-noise links accumulates FP32 rounding
        # in E faster)
        c = [n / 2.0 for n in prob.N[:dims]]
        s.set_spinor(W.gaussian_packet(prob, 3.0, [0.4, -0.3, 0.2][:dims], c))
        s.step(60)
        ok, rep = s.check(1e-6)
        assert ok, rep
        assert abs(rep["drift"]) < 1e-6 and rep["lower"] <= rep["naive"] <= rep["upper"]
