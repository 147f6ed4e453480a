"""Batched stepping and the serving loop.

* dirac_batch_step packs simulations of different sizes, masses and fields
  into one persistent launch per time step; every simulation's result must
  equal, bit for bit, the result of stepping it alone, and the FP64 oracle
  within the FP32 (1e-5 rel L2) or FP64 (1e-12) tolerance.
* The serving loop admits requests as they arrive and HBM allows, batches
  the resident ones and retires them; each result keeps E to FP32 accuracy
  and its final state matches the oracle.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1309_3452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_3452_gb300 import dirac
    return dirac


def mix():
    r3 = 0.9 * W.stability_limit(3)
    r2 = 0.9 * W.stability_limit(2)
    return [
        (W.Problem(3, (40, 36, 30), (1.0, 1.0, 1.0), r3, 0.7), 0),
        (W.Problem(3, (17, 23, 11), (1.0, 1.0, 1.0), r3, 0.2), 0),
        (W.Problem(3, (64, 64, 64), (1.0, 1.0, 1.0), r3, 1.0,
                   W.Fields(step_axis=0, step_x0=32.25, step_V=1.3)), 0),
        (W.Problem(3, (33, 29, 21), (1.0, 1.0, 1.0), r3, 0.4,
                   W.Fields(step_axis=2, step_x0=8.25, step_V=-0.7)), 0),
        (W.Problem(2, (130, 97, 1), (1.0, 1.0, 1.0), r2, 0.3), 0),
        (W.Problem(2, (64, 64, 1), (1.0, 1.0, 1.0), r2, 0.0,
                   W.Fields(step_axis=0, step_x0=32.25, step_V=0.6)), 0),
        (W.Problem(2, (301, 45, 1), (1.0, 1.0, 1.0), r2, 0.9), 0),
        (W.Problem(3, (20, 20, 20), (1.0, 1.0, 1.0), r3, 0.5, W.Fields(q=1.0, A_const=(0.2, 0.1, 0.0))), 0),
        (W.Problem(3, (19, 18, 17), (1.0, 1.0, 1.0), r3, 0.5), 1),   # FP64: stepped alone
        (W.Problem(2, (40, 40, 1), (1.0, 1.0, 1.0), r2, 0.5,         # general field path: alone
                   W.Fields(sc_Z=1.0, sc_a=1.0, sc_center=(20.0, 20.0, 0.0))), 0),
    ]


def test_batch_equals_alone_bitwise(D):
    probs = mix()
    states = [W.random_state(p, 100 + i) for i, (p, _) in enumerate(probs)]
    alone = []
    for (p, prec), psi in zip(probs, states):
        with D.Sim(p, D.FP64 if prec else D.FP32) as s:
            s.set_spinor(psi)
            s.step(23)
            s.step(40)
            alone.append(s.get_spinor())
    sims = []
    try:
        for (p, prec), psi in zip(probs, states):
            s = D.Sim(p, D.FP64 if prec else D.FP32)
            s.set_spinor(psi)
            sims.append(s)
        D.batch_step(sims, 23)
        D.batch_step(sims[::-1], 40)  # another order, odd then even step counts
        for s, want in zip(sims, alone):
            assert abs(s.time - 63 * s.prob.dt) < 1e-12
            assert np.array_equal(s.get_spinor(), want)
    finally:
        for s in sims:
            s.close()
    # every member against the FP64 oracle on the same input
    for (p, prec), psi, got in zip(probs, states, alone):
        ref = O.step(p, psi, 63)
        assert rel(got, ref) < (FP64_TOL if prec else FP32_TOL), p


def test_batch_rejects_mixed_streams_and_duplicates(D):
    import torch
    p = W.Problem(2, (32, 32, 1), (1.0, 1.0, 1.0), 0.5, 0.1)
    st = torch.cuda.Stream()
    a = D.Sim(p, D.FP32)
    b = D.Sim(p, D.FP32, stream=st.cuda_stream)
    try:
        with pytest.raises(D.DiracError):
            D.batch_step([a, b], 3)
        with pytest.raises(D.DiracError):
            D.batch_step([a, a], 3)
    finally:
        a.close()
        b.close()


def test_serving_loop_small_stream(D):
    from paper_1309_3452_gb300 import serve
    reqs = serve.make_requests(12, seed=3, rate=20.0, max_side_3d=48, max_side_2d=256,
                               min_steps=20, max_steps=200)
    srv = serve.Server(hbm_budget=2 << 30, quantum=50)
    out = srv.run(reqs)
    assert out["requests"] == out["served"] == len(reqs)
    assert out["max_E_drift"] < 1e-6
    assert out["p99_s"] >= out["p50_s"] > 0.0
    for r in out["results"]:
        assert r.finished >= r.admitted >= r.arrival - 1e-9


def test_batch_graph_replay_and_membership_changes(D, monkeypatch):
    """Batched step loops are recorded as CUDA graphs and replayed while the
    group repeats (the serving loop's quanta); replays, odd and even step
    counts, a member leaving (destroyed) and one joining must all give the
    states of stepping alone, bit for bit, as with graphs switched off."""
    probs = [p for p, prec in mix() if prec == 0][:6]
    states = [W.random_state(p, 200 + i) for i, p in enumerate(probs)]
    plan = [(list(range(6)), 10), (list(range(6)), 10), (list(range(6)), 7), (list(range(6)), 10),
            ([0, 2, 3, 4, 5], 10), ([0, 2, 3, 4, 5], 10), ([0, 2, 3, 4, 5, 1], 6)]

    def run(graphs):
        if not graphs:
            monkeypatch.setenv("DIRAC_NO_GRAPHS", "1")
        sims = []
        for p, psi in zip(probs, states):
            s = D.Sim(p, D.FP32)
            s.set_spinor(psi)
            sims.append(s)
        out = {}
        try:
            for members, n in plan:
                if members == [0, 2, 3, 4, 5] and sims[1] is not None and 1 not in out:
                    out[1] = sims[1].get_spinor()  # member 1 leaves: destroyed, then re-created
                    sims[1].close()
                    sims[1] = None
                if 1 in members and sims[1] is None:
                    sims[1] = D.Sim(probs[1], D.FP32)
                    sims[1].set_spinor(out[1])
                D.batch_step([sims[i] for i in members], n)
            res = [s.get_spinor() for s in sims]
        finally:
            for s in sims:
                if s is not None:
                    s.close()
            monkeypatch.delenv("DIRAC_NO_GRAPHS", raising=False)
        return res

    with_graphs, without = run(True), run(False)
    for a, b in zip(with_graphs, without):
        assert np.array_equal(a, b)
    # and against stepping each simulation alone for the same number of steps
    total = [sum(n for members, n in plan if i in members) for i in range(6)]
    for i, (p, psi) in enumerate(zip(probs, states)):
        with D.Sim(p, D.FP32) as s:
            s.set_spinor(psi)
            s.step(total[i])
            assert np.array_equal(s.get_spinor(), with_graphs[i])


@pytest.mark.parametrize("policy", ["lockstep", "work"])
def test_serving_results_equal_stepping_alone(D, monkeypatch, policy):
    """Each request served in the mix (admitted and retired between rounds,
    batched with whatever else is resident, loops replayed as graphs, under
    either scheduling policy) ends in the same state as when stepped alone:
    its functional, from the same reduction, is identical to the last bit."""
    from paper_1309_3452_gb300 import serve
    monkeypatch.setenv("DIRAC_NO_FUSED_NORM", "1")  # both sides reduce the stored state
    reqs = serve.make_requests(24, seed=5, rate=40.0, max_side_3d=40, max_side_2d=192,
                               min_steps=30, max_steps=700)
    srv = serve.Server(hbm_budget=3 << 30, quantum=50, keep_states=True, policy=policy)
    out = srv.run(reqs)
    assert out["served"] == len(reqs)
    byid = {r.rid: r for r in reqs}
    import torch
    for res in out["results"]:
        req = byid[res.rid]
        psi = W.gaussian_packet_torch(req.prob, req.sigma, req.k0, req.center, "cuda")
        with D.Sim(req.prob, req.precision) as s:
            s.set_spinor_device(psi.data_ptr())
            E0, _ = s.norm()
            s.step(req.steps)
            E1, _ = s.norm()
        torch.cuda.synchronize()
        assert E0 == res.E0 and E1 == res.E1, res.rid
        # the served state against the FP64 oracle from the same initial packet
        ref = O.step(req.prob, psi.cpu().numpy(), req.steps)
        assert rel(res.state, ref) < FP32_TOL, res.rid


def test_allocation_refusal_is_reported_not_faulted(D):
    """A grid beyond the device's memory: dirac_create's cudaMalloc fails and
    the call returns DIRAC_ERR_OOM with nothing left allocated (no device
    fault; the context stays usable)."""
    import torch
    free0, _ = torch.cuda.mem_get_info()
    p = W.Problem(3, (2048, 2048, 2048), (1.0, 1.0, 1.0), 0.5, 0.5)  # 550 GB per FP32 state buffer
    with pytest.raises(D.DiracError) as e:
        D.Sim(p, D.FP32)
    assert e.value.status == D.ERR_OOM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    q = W.Problem(2, (64, 64, 1), (1.0, 1.0, 1.0), 0.5, 0.5)
    with D.Sim(q, D.FP32) as s:  # the device still works
        s.set_spinor(W.random_state(q, 1))
        s.step(3)
        assert np.isfinite(s.norm()[0])
