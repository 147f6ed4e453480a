"""dirac_set_spinor / dirac_get_spinor from host buffers of every kind.

An FP32 simulation converts a page-locked, device-mapped, 16-byte aligned
buffer in place (the conversion kernels read and write host memory); a
pageable buffer, a page-locked one at an 8-byte offset and any buffer under
DIRAC_HOST_COPY=staged go through the device staging plane.  The conversion
is the same rounding either way, so every route must give the same state to
the last bit, and the state read back must equal the FP32 rounding of what
was set (the canonical layout, plane by plane).
"""
import numpy as np
import pytest

from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def pinned(shape, offset_bytes=0):
    """A page-locked complex128 array of `shape` starting offset_bytes into
    its allocation (the torch buffer is returned to keep it alive)."""
    import torch
    n = int(np.prod(shape))
    buf = torch.empty(2 * n + 2, dtype=torch.float64, pin_memory=True)
    raw = buf.numpy().view(np.uint8)[offset_bytes:offset_bytes + 16 * n]
    return raw.view(np.complex128).reshape(shape), buf


def rounded(psi):
    """The FP32 rounding of every real and imaginary part (what the state holds)."""
    return (psi.real.astype(np.float32).astype(np.float64)
            + 1j * psi.imag.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("dims", [3, 2])
def test_set_get_routes_agree_bitwise(D, dims, monkeypatch):
    N = (37, 29, 19) if dims == 3 else (133, 71, 1)
    prob = W.Problem(dims, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), 0.6,
                     W.Fields(step_axis=0, step_x0=N[0] / 2 + 0.25, step_V=0.5))
    psi = W.random_state(prob, 41 + dims)
    want = rounded(psi)
    host_al, keep_al = pinned(prob.shape)        # mapped, aligned: converted in place
    host_off, keep_off = pinned(prob.shape, 8)   # mapped, 8-byte offset: staged
    host_al[...] = psi
    host_off[...] = psi
    states, stepped = [], []
    for route in ("pageable", "mapped", "offset", "staged"):
        if route == "staged":
            monkeypatch.setenv("DIRAC_HOST_COPY", "staged")
        with D.Sim(prob, D.FP32) as s:
            if route == "pageable":
                s.set_spinor(psi)
            elif route == "offset":
                s.set_spinor_ptr(host_off.ctypes.data)
            else:
                s.set_spinor_ptr(host_al.ctypes.data)
            E0, _ = s.norm()
            out_pg = s.get_spinor()
            out_al, k1 = pinned(prob.shape)
            out_off, k2 = pinned(prob.shape, 8)
            s.get_spinor_ptr(out_al.ctypes.data)
            s.get_spinor_ptr(out_off.ctypes.data)
            assert np.array_equal(out_pg, want), route
            assert np.array_equal(out_al, want), route
            assert np.array_equal(out_off, want), route
            states.append(E0)
            s.step(7)
            stepped.append(s.get_spinor())
        monkeypatch.delenv("DIRAC_HOST_COPY", raising=False)
    assert all(e == states[0] for e in states)
    for x in stepped[1:]:
        assert np.array_equal(x, stepped[0])
