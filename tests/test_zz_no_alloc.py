"""dirac_norm_noalloc, the entry point for callers that cannot allocate
device memory where they need the norm (their framework owns all device
memory through its own pool, or the call sits in a loop that cannot take
cudaMalloc's implicit synchronisation).  The test owns the device planes (a
test may allocate; the entry point may not) and checks the entry point
against dirac_norm on the same state, for two calls in a row that share the
library's fixed scratch array."""
import ctypes as C

import numpy as np
import pytest

from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac as D
    L = D.lib()
    L.dirac_norm_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double,
                                     C.c_double, C.c_void_p, C.c_int, C.POINTER(C.c_void_p),
                                     C.c_void_p, C.c_void_p]
    L.dirac_norm_noalloc.restype = C.c_int
    return torch, D, L


def device_planes(torch, prob, psi, precision, D):
    dtype = torch.complex128 if precision == D.FP64 else torch.complex64
    t = torch.from_numpy(np.ascontiguousarray(psi)).to(dtype).cuda()  # (P, Nz, Ny, Nx)
    ptrs = [t[k].data_ptr() for k in range(prob.n_planes)] + [None] * (8 - prob.n_planes)
    return t, (C.c_void_p * 8)(*ptrs)


def noalloc_norm(torch, L, D, prob, ptrs, t, precision, out=None):
    if out is None:
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
    N = (C.c_int * 3)(*[int(v) for v in (list(prob.N) + [1, 1, 1])[:3]])
    dx = (C.c_double * 3)(*[float(v) for v in (list(prob.dx) + [1.0] * 3)[:3]])
    stream = torch.cuda.current_stream()
    fs, _ = D._fields_struct(prob.fields)
    rc = L.dirac_norm_noalloc(prob.dims, N, dx, prob.dt, t, C.byref(fs), precision, ptrs, out.data_ptr(),
                              stream.cuda_stream)
    assert rc == D.OK
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dims,precision", [(3, "fp32"), (3, "fp64"), (2, "fp32")])
def test_noalloc_norm_matches_dirac_norm_twice(env, dims, precision):
    torch, D, L = env
    prec = D.FP32 if precision == "fp32" else D.FP64
    if dims == 3:
        prob = W.Problem(3, (21, 18, 15), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.7)
    else:
        prob = W.Problem(2, (70, 45, 1), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(2), 0.3)
    psi = W.random_state(prob, 31)
    with D.Sim(prob, prec) as s:
        s.set_spinor(psi)
        for _ in range(2):  # two calls in a row share the scratch array
            E_ref, naive_ref = s.norm()
            tstate, ptrs = device_planes(torch, prob, s.get_spinor(), prec, D)
            E, naive = noalloc_norm(torch, L, D, prob, ptrs, s.time, prec)
            del tstate
            # FP64: the same reduction on both sides; FP32: after steps dirac_norm
            # returns the functional accumulated by the last step's kernel (another
            # summation order), the tolerance of the fused-functional tests
            tol = 1e-13 if prec == D.FP64 else 2e-7
            assert abs(E - E_ref) <= tol * abs(E_ref)
            assert abs(naive - naive_ref) <= tol * naive_ref
            s.step(13)


@pytest.mark.parametrize("field", ["A_const", "plane_wave"])
def test_noalloc_norm_with_vector_potentials(env, field):
    """The constant-link and per-site plane-wave branches of the functional,
    against dirac_norm on the same state (FP64: the same reduction, 1e-13)."""
    torch, D, L = env
    prob = W.Problem(3, (20, 17, 22), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.6)
    if field == "A_const":
        prob = prob.with_fields(q=1.0, A_const=(0.21, -0.13, 0.08))
    else:  # a moving plane wave: the functional reads its link phases at t - dt/2
        k = 2 * np.pi / 22.0
        prob = prob.with_fields(q=1.0, Apw_amp=0.4, Apw_k=(0.0, 0.0, k), Apw_omega=k, Apw_phase=0.3,
                                Apw_pol=0)
    psi = W.random_state(prob, 37)
    with D.Sim(prob, D.FP64) as s:
        s.set_spinor(psi)
        s.step(7)  # t != 0: the link time matters for the plane wave
        for _ in range(2):
            E_ref, naive_ref = s.norm()
            tstate, ptrs = device_planes(torch, prob, s.get_spinor(), D.FP64, D)
            E, naive = noalloc_norm(torch, L, D, prob, ptrs, s.time, D.FP64)
            del tstate
            assert abs(E - E_ref) <= 1e-13 * abs(E_ref)
            assert abs(naive - naive_ref) <= 1e-13 * naive_ref
            s.step(5)


def test_noalloc_calls_allocate_nothing(env):
    """After one warm call, further calls leave the device's free memory and
    the caching allocator's reserved bytes unchanged."""
    torch, D, L = env
    prob = W.Problem(3, (24, 20, 18), (1.0, 1.0, 1.0), 0.9 * W.stability_limit(3), 0.5)
    psi = W.random_state(prob, 41)
    tstate, ptrs = device_planes(torch, prob, psi, D.FP32, D)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    first = noalloc_norm(torch, L, D, prob, ptrs, 0.0, D.FP32, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(5):
        again = noalloc_norm(torch, L, D, prob, ptrs, 0.0, D.FP32, out)
        assert np.array_equal(again, first)  # same state, same scratch, same order
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    del tstate


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, D, L = env
    N = (C.c_int * 3)(4096, 4096, 1)  # 128 x 512 reduction blocks > 8192
    dx = (C.c_double * 3)(1.0, 1.0, 1.0)
    dummy = (C.c_void_p * 8)(*([16] * 8))  # never dereferenced: rejected before any device work
    rc = L.dirac_norm_noalloc(2, N, dx, 0.5, 0.0, None, D.FP32, dummy, 16, None)
    assert rc == D.ERR_UNSUPPORTED
