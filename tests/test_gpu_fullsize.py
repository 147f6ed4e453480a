"""Parity at the full workload sizes, in the launch configuration the
benchmark times (FP32 fused kernels; FP64 split kernels for the FP64 line).

* (3+1)D 128^3, 1000 steps: sampled values and E against stored oracle
  results (tests/golden/workload_3d128_1000.json, written by
  tests/golden/make_golden.py from the oracle only).
* (2+1)D 4096^2 Klein step, the oblique Klein refraction workload and (3+1)D
  512^3 soft core + plane-wave vector potential: light-cone windows.  After n steps a value depends only on the
  values within n cells (one half-lattice site per half-step), so the oracle
  run on a periodic window of half-width n + 2 around a cell, placed at the
  same position (origin), reproduces that cell exactly; windows are kept
  away from the domain wrap so the fields see the same positions.
* Properties at full size: E conserved (static fields), FP32 drift <= 1e-6.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "workload_3d128_1000.json")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac as D
    return torch, D


def window(psi, prob, cell, w):
    """Cells [cell - w, cell + w] per axis of a (P, Nz, Ny, Nx) state (numpy or torch)."""
    sl = [slice(None)]
    if prob.dims == 3:
        sl.append(slice(cell[2] - w, cell[2] + w + 1))
    else:
        sl.append(slice(0, 1))
    sl += [slice(cell[1] - w, cell[1] + w + 1), slice(cell[0] - w, cell[0] + w + 1)]
    out = psi[tuple(sl)]
    return out.cpu().numpy() if hasattr(out, "cpu") else np.array(out)


def window_problem(prob, w):
    n = 2 * w + 1
    N = (n, n, n) if prob.dims == 3 else (n, n, 1)
    return W.Problem(prob.dims, N, prob.dx, prob.dt, prob.m, prob.fields)


def check_windows(prob, psi0, out, cells, n, tol):
    w = n + 2
    wp = window_problem(prob, w)
    for cell in cells:
        origin = [c - w for c in cell] + [0] * (3 - len(cell))
        ref = O.step(wp, window(psi0, prob, cell, w), n, 0.0, origin=origin)
        got = window(out, prob, cell, 0)
        want = ref[(slice(None),) + ((slice(w, w + 1),) if prob.dims == 3 else (slice(0, 1),))
                   + (slice(w, w + 1), slice(w, w + 1))]
        scale = max(float(np.max(np.abs(ref))), 1e-30)
        err = float(np.max(np.abs(got - want))) / scale
        assert err < tol, (cell, err)


def test_workload_3d128_against_golden(env):
    torch, D = env
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file not generated")
    g = json.load(open(GOLDEN))
    prob, psi, n = W.workload_3d(N=128, steps=1000)
    assert n == g["steps"] and abs(prob.dt - g["dt"]) < 1e-15
    sites = tuple(np.array(g["sites"]).T)
    want = np.array([complex(a, b) for a, b in g["values"]])
    for prec, tol, etol in ((D.FP64, 1e-12, 1e-12), (D.FP32, 1e-5, 1e-6)):
        with D.Sim(prob, prec) as s:
            s.set_spinor(psi)
            s.step(n)
            E, naive = s.norm()
            out = s.get_spinor()
        got = out[sites]
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
        assert abs(E - g["E"]) < etol * abs(g["E"])
        assert abs(E - g["E0"]) < etol * abs(g["E0"])  # conserved over the 1000 steps


def test_workload_klein4096_windows_and_conservation(env):
    torch, D = env
    prob, psi, _ = W.workload_klein(N=4096, steps=5000)
    n = 10
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        E0, _ = s.norm()
        s.step(n)
        out = s.get_spinor()
        x0 = prob.fields.step_x0
        cells = [(1024, 2048), (1030, 2041), (2048, 2048), (2049, 1000), (3000, 2050), (40, 4000)]
        check_windows(prob, psi, out, cells, n, 2e-6)
        s.step(490)
        E1, _ = s.norm()
        T = s.partial_density(0, x0)
    assert abs(E1 - E0) < 1e-6 * abs(E0)
    assert 0.0 <= T <= 1.0


def test_workload_laser512_windows(env):
    torch, D = env
    prob, _, _ = W.workload_laser(N=512, steps=2000, seed=1, sigma=24.0, packet=False)
    c = 256.0
    psi0 = W.gaussian_packet_torch(prob, 24.0, W.random_k0(1), (c, c, c), "cuda")
    n = 5
    w = n + 2
    cells = [(256, 256, 256), (250, 270, 259), (230, 250, 300), (300, 200, 222), (20, 480, 100)]
    wins = [(cell, window(psi0, prob, cell, w)) for cell in cells]
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor_device(psi0.data_ptr())
        s.step(n)
        s.get_spinor_device(psi0.data_ptr())  # reuse the buffer for the result
        torch.cuda.synchronize()
    wp = window_problem(prob, w)
    for cell, win in wins:
        ref = O.step(wp, win, n, 0.0, origin=[v - w for v in cell])
        got = window(psi0, prob, cell, 0)
        want = ref[:, w:w + 1, w:w + 1, w:w + 1]
        scale = max(float(np.max(np.abs(ref))), 1e-30)
        assert float(np.max(np.abs(got - want))) / scale < 2e-6, cell


def test_workload_klein_oblique4096_windows_and_conservation(env):
    torch, D = env
    prob, psi, _ = W.workload_klein_oblique(N=4096)
    n = 10
    x0 = prob.fields.step_x0
    with D.Sim(prob, D.FP32) as s:
        s.set_spinor(psi)
        E0, _ = s.norm()
        s.step(n)
        out = s.get_spinor()
        # around the packet (centred 4 sigma before the step), on both sides of the step, far away
        c = (int(x0 - 4 * 64 * math.cos(math.radians(53))), int(2048 - 4 * 64 * math.sin(math.radians(53))))
        cells = [c, (c[0] + 9, c[1] - 17), (2048, 2000), (2049, 2100), (3500, 600), (100, 4000)]
        check_windows(prob, psi, out, cells, n, 2e-6)
        s.step(490)
        ok, r = s.check(1e-6)
    assert ok, r
    assert abs(r["E"] - E0) < 1e-6 * abs(E0)
