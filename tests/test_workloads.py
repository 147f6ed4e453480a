"""The seeded input generators (CPU): the separable packet generator the
benchmark uses for grids whose host state is tens of GB agrees with the
direct one, and a window of it (origin inside a larger periodic box) is the
same packet sampled on that window."""
import numpy as np

from paper_1309_3452_gb300 import workloads as W


def test_separable_packet_matches_direct_3d_and_2d():
    prob, _, _ = W.workload_laser(N=20, steps=1)
    k0 = W.random_k0(1)
    a = W.gaussian_packet(prob, 4.0, k0, (10.0, 9.5, 11.0))
    b = W.gaussian_packet_separable(prob, 4.0, k0, (10.0, 9.5, 11.0))
    assert np.max(np.abs(a - b)) < 1e-14 * np.max(np.abs(a))
    p2 = W.Problem(2, (30, 21, 1), (1.0, 1.2, 1.0), 0.4, 0.3)
    a = W.gaussian_packet(p2, 3.0, (0.3, -0.2), (5.0, 17.0))  # near a face: the periodic image counts
    b = W.gaussian_packet_separable(p2, 3.0, (0.3, -0.2), (5.0, 17.0))
    assert np.max(np.abs(a - b)) < 1e-14 * np.max(np.abs(a))


def test_separable_packet_window_is_a_slice_of_the_full_state():
    prob, _, _ = W.workload_laser(N=24, steps=1)
    k0 = W.random_k0(2)
    full = W.gaussian_packet_separable(prob, 5.0, k0, (12.0, 12.0, 12.0), normalise=False)
    wp = W.Problem(3, (10, 12, 8), prob.dx, prob.dt, prob.m, prob.fields)
    origin = (7, 3, 9)
    win = W.gaussian_packet_separable(wp, 5.0, k0, (12.0, 12.0, 12.0), origin=origin, box=prob.N,
                                      normalise=False)
    want = full[:, 9:17, 3:15, 7:17]
    assert np.max(np.abs(win - want)) < 1e-14 * np.max(np.abs(full))
