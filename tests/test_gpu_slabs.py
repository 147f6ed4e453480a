"""The sub-domain decomposition (Sect. 6): a grid split along its marching
axis (z in (3+1)D, y in (2+1)D) into slabs with one halo level on either
side, refreshed after every time step from the neighbours.  Every value is computed by the same arithmetic from
the same neighbours as in the whole grid, so the stepped state must equal
the whole grid's bit for bit, for any number of slabs (uneven ones
included), and match the FP64 oracle within the FP32 tolerance; the
functional summed over the slabs equals the whole grid's up to summation
order."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = (40, 36, 34)


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def fields(name):
    c = (N[0] / 2.0, N[1] / 2.0, N[2] / 2.0)
    kz = 2 * math.pi / N[2]
    return {
        "free": W.Fields(),
        "klein_z": W.Fields(V0=0.05, step_axis=2, step_x0=N[2] - 3.75, step_V=0.9),  # near the wrap
        "softcore": W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=(c[0], c[1], 1.5)),       # centre on a slab edge
        "A_const": W.Fields(q=1.0, A_const=(0.3, -0.25, 0.15)),
        "laser": W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=c, q=1.0, Apw_amp=0.5, Apw_k=(0.0, 0.0, kz),
                          Apw_omega=kz, Apw_pol=0),
    }[name]


@pytest.mark.parametrize("name", ["free", "klein_z", "softcore", "A_const", "laser"])
def test_slabs_equal_whole_grid_bitwise_and_oracle(D, name):
    prob = W.Problem(3, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 1.0, fields(name))
    psi = W.gaussian_packet(prob, 5.0, W.random_k0(21), (20.0, 18.0, 3.0))  # packet across the wrap
    n = 37
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(n)
        E_whole, naive_whole = s.norm()
        whole = s.get_spinor()
    ref = O.step(prob, psi, n)
    assert np.linalg.norm(whole - ref) / np.linalg.norm(ref) < 1e-5
    for nslabs in (1, 2, 3, 5):
        with D.Slabs(prob, nslabs) as g:
            parts = [g.info(k) for k in range(nslabs)]
            assert parts == D.slab_partition(N[2], nslabs)
            g.set_spinor(psi)
            E_set, _ = g.norm()
            g.step(n)
            E, naive = g.norm()
            got = g.get_spinor()
            assert abs(g.time - n * prob.dt) < 1e-12
        assert np.array_equal(got, whole), (name, nslabs)
        assert abs(E - E_whole) < 1e-12 * abs(E_whole)
        assert abs(naive - naive_whole) < 1e-12 * naive_whole
        if name != "laser":  # static fields: E conserved
            assert abs(E - E_set) < 1e-6 * abs(E_set)


N2 = (150, 97, 1)


def fields2(name):
    ky = 2 * math.pi / N2[1]
    return {
        "free": W.Fields(),
        "klein_x": W.Fields(step_axis=0, step_x0=N2[0] / 2 + 0.25, step_V=0.9),
        "klein_y": W.Fields(step_axis=1, step_x0=N2[1] - 2.75, step_V=-0.6),       # near the wrap
        "softcore": W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=(70.0, 3.5, 0.0)),
        "A_wave": W.Fields(q=1.0, Apw_amp=0.5, Apw_k=(0.0, ky, 0.0), Apw_omega=ky, Apw_pol=0),
    }[name]


@pytest.mark.parametrize("name", ["free", "klein_x", "klein_y", "softcore", "A_wave"])
def test_row_slabs_2d_equal_whole_grid_bitwise_and_oracle(D, name):
    """(2+1)D: y-slabs stepped one time step per pass against the whole grid
    (which takes two steps per pass where it can: the same values)."""
    prob = W.Problem(2, N2, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.4, fields2(name))
    psi = W.gaussian_packet(prob, 9.0, (0.3, 0.2), (60.0, 5.0))  # across the wrap in y
    n = 41
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        s.step(n)
        E_whole, _ = s.norm()
        whole = s.get_spinor()
    ref = O.step(prob, psi, n)
    assert np.linalg.norm(whole - ref) / np.linalg.norm(ref) < 1e-5
    for nslabs in (1, 2, 4, 7):
        with D.Slabs(prob, nslabs) as g:
            assert [g.info(k) for k in range(nslabs)] == D.slab_partition(N2[1], nslabs)
            g.set_spinor(psi)
            g.step(n)
            E, _ = g.norm()
            got = g.get_spinor()
        assert np.array_equal(got, whole), (name, nslabs)
        assert abs(E - E_whole) < 1e-12 * abs(E_whole)


def test_slabs_reject_what_they_do_not_decompose(D):
    p3 = W.Problem(3, (16, 16, 12), (1.0, 1.0, 1.0), 0.5, 0.5)
    bad = [(p3, 2, D.FP64), (W.Problem(2, (16, 16, 1), (1.0, 1.0, 1.0), 0.5, 0.5), 17, D.FP32),
           (p3.with_fields(V_static=W.random_potential(p3, 1, 0.1)), 2, D.FP32),
           (p3.with_fields(abs_W=0.3, abs_width=2.0, abs_axes=1), 2, D.FP32),
           (p3.with_fields(Apw_amp=0.2, Apw_k=(0.3, 0.2, 0.0), Apw_pol=2), 2, D.FP32),  # a static table of links
           (p3, 13, D.FP32)]
    for prob, n, prec in bad:
        with pytest.raises(D.DiracError):
            D.Slabs(prob, n, prec)
