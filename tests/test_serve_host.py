"""The serving loop's scheduling, on the CPU (paper_1309_3452_gb300/serve.py).

The device work is replaced by fakes that only count steps, so what is
checked is the host logic: every request receives exactly its number of time
steps, is admitted only after it has arrived and while the resident states
fit the HBM budget, quanta never carry a request past its last step, and the
latency statistics are consistent.
"""
import pytest

from paper_1309_3452_gb300 import build as B

B.build()  # dirac_state_bytes is host code of the library

from paper_1309_3452_gb300 import dirac as D  # noqa: E402
from paper_1309_3452_gb300 import serve  # noqa: E402


class FakeStream:
    cuda_stream = None

    def synchronize(self):
        pass


class FakeSim:
    alive = []

    def __init__(self, req, need):
        self.req, self.need, self.steps, self.closed = req, need, 0, False
        self.launches = 0
        FakeSim.alive.append(self)

    def norm(self):
        return 1.0, 1.0

    def close(self):
        self.closed = True
        FakeSim.alive.remove(self)


def test_serving_schedule(monkeypatch):
    FakeSim.alive = []
    reqs = serve.make_requests(30, seed=1, rate=300.0, max_side_3d=64, max_side_2d=512,
                               min_steps=10, max_steps=400)
    needs = {r.rid: D.state_bytes(r.prob.dims, r.prob.N, r.precision) for r in reqs}
    budget = 3 * max(needs.values())  # a few requests at a time
    sims, calls = {}, []

    def admit(self, req):
        import time
        sims[req.rid] = FakeSim(req, needs[req.rid])
        sims[req.rid].admitted_wall = time.perf_counter()
        assert sum(s.need for s in FakeSim.alive) <= budget
        return sims[req.rid], 1.0

    def batch_step(group, n):
        calls.append((len(group), n))
        assert n >= 1
        for s in group:
            assert not s.closed
            s.steps += n
            s.launches += 1
            assert s.steps <= s.req.steps  # a quantum never runs past a request's last step

    monkeypatch.setattr(serve.Server, "_admit", admit)
    monkeypatch.setattr(serve.D, "batch_step", batch_step)
    srv = serve.Server(hbm_budget=budget, quantum=64, stream=FakeStream())
    out = srv.run(reqs)

    assert out["requests"] == len(reqs)
    assert all(sims[r.rid].steps == r.steps for r in reqs)
    assert all(s.closed for s in sims.values()) and not FakeSim.alive
    assert all(n <= 64 for _, n in calls)
    assert max(k for k, _ in calls) > 1  # requests were batched together
    for res in out["results"]:
        assert res.admitted >= res.arrival - 1e-9 and res.finished >= res.admitted
    assert out["p99_s"] >= out["p50_s"] > 0.0
    assert out["total_lups"] == sum(r.lups for r in reqs)


def test_request_stream_is_seeded_and_in_range():
    a = serve.make_requests(200, seed=7, rate=2.0)
    b = serve.make_requests(200, seed=7, rate=2.0)
    assert [(r.arrival, r.prob.N, r.steps, r.prob.m) for r in a] == \
           [(r.arrival, r.prob.N, r.steps, r.prob.m) for r in b]
    arrivals = [r.arrival for r in a]
    assert arrivals == sorted(arrivals) and arrivals[0] > 0.0
    for r in a:
        side = r.prob.N[0]
        if r.prob.dims == 2:
            assert 64 <= side <= 4096 and r.prob.N[2] == 1
        else:
            assert 32 <= side <= 384 and r.prob.N[0] == r.prob.N[1] == r.prob.N[2]
        assert 100 <= r.steps <= 5000 and 0.0 <= r.prob.m <= 1.0
        assert r.sigma == side / 8.0
    dims = [r.prob.dims for r in a]
    assert 0.3 < dims.count(2) / len(dims) < 0.7  # (2+1)D with probability 1/2


def test_percentile():
    assert serve.percentile([1.0, 2.0, 3.0, 4.0], 50) == pytest.approx(2.5)
    assert serve.percentile([5.0], 99) == 5.0
    assert serve.percentile([1.0, 2.0], 100) == 2.0
