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

    def check(self, tol):
        return True, {"E": 1.0, "E_ref": 1.0}

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
        return sims[req.rid]

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
    srv = serve.Server(hbm_budget=budget, quantum=64, stream=FakeStream(), policy="lockstep")
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


def fake_device(monkeypatch, needs, oom_at=(), steps_seen=None):
    """Patch the server's device work: admissions create FakeSims (raising
    DIRAC_ERR_OOM, as dirac_create does when cudaMalloc fails, on the
    admission attempts listed in oom_at), batch steps count steps."""
    sims, attempts = {}, []

    def admit(self, req):
        attempts.append(req.rid)
        if len(attempts) in oom_at:
            raise D.DiracError(D.ERR_OOM, "cudaMalloc(state): out of memory (injected)")
        sims[req.rid] = FakeSim(req, needs[req.rid])
        return sims[req.rid]

    def batch_step(group, n):
        for s in group:
            assert not s.closed
            s.steps += n
            s.launches += 1
            assert s.steps <= s.req.steps

    monkeypatch.setattr(serve.Server, "_admit", admit)
    monkeypatch.setattr(serve.D, "batch_step", batch_step)
    return sims, attempts


def test_oversize_request_is_rejected_not_raised(monkeypatch):
    FakeSim.alive = []
    reqs = serve.make_requests(8, seed=2, rate=500.0, max_side_3d=48, max_side_2d=256,
                               min_steps=10, max_steps=50)
    needs = {r.rid: D.state_bytes(r.prob.dims, r.prob.N, r.precision) for r in reqs}
    big = max(needs, key=needs.get)
    budget = max(v for k, v in needs.items() if k != big)  # everything fits but the largest
    sims, _ = fake_device(monkeypatch, needs)
    out = serve.Server(hbm_budget=budget, quantum=16, stream=FakeStream()).run(reqs)
    st = {r.rid: r.status for r in out["results"]}
    assert st[big] == "rejected" and big not in sims
    assert all(st[r.rid] == "ok" for r in reqs if r.rid != big)
    assert out["served"] == len(reqs) - 1 and not FakeSim.alive


def test_allocation_refusal_backs_off_until_a_request_retires(monkeypatch):
    """An injected DIRAC_ERR_OOM at admission: the request waits (no crash,
    no retry storm) until a resident request retires, then is admitted; an
    OOM with nothing resident rejects the request."""
    FakeSim.alive = []
    reqs = serve.make_requests(10, seed=4, rate=1000.0, max_side_3d=40, max_side_2d=128,
                               min_steps=20, max_steps=60)
    for r in reqs:
        r.arrival = 0.0  # all waiting at once: the first two are resident when the third fails
    needs = {r.rid: D.state_bytes(r.prob.dims, r.prob.N, r.precision) for r in reqs}
    sims, attempts = fake_device(monkeypatch, needs, oom_at=(3, 4))
    srv = serve.Server(hbm_budget=10 * sum(needs.values()), quantum=8, stream=FakeStream())
    out = srv.run(reqs)
    assert srv.oom_backoffs == 2
    # the third attempt failed; the same request came back only after a retirement
    refused = attempts[2]
    assert attempts[3] == refused  # retried: the 4th attempt is the same request (and failed again)
    assert attempts.count(refused) == 3
    assert all(r.status == "ok" for r in out["results"])
    assert all(sims[r.rid].steps == r.steps for r in reqs) and not FakeSim.alive
    # nothing resident: the OOM request cannot wait for memory to come back
    FakeSim.alive = []
    one = serve.make_requests(1, seed=4, rate=1000.0, max_side_3d=40, max_side_2d=128,
                              min_steps=20, max_steps=60)
    fake_device(monkeypatch, {one[0].rid: needs[one[0].rid]}, oom_at=(1,))
    out = serve.Server(hbm_budget=1 << 40, quantum=8, stream=FakeStream()).run(one)
    assert [r.status for r in out["results"]] == ["oom"]


def test_cancelled_and_timed_out_requests_free_their_slots(monkeypatch):
    FakeSim.alive = []
    reqs = serve.make_requests(12, seed=6, rate=2000.0, max_side_3d=40, max_side_2d=128,
                               min_steps=400, max_steps=500)
    needs = {r.rid: D.state_bytes(r.prob.dims, r.prob.N, r.precision) for r in reqs}
    reqs[0].cancel_after = 0.0   # cancelled as soon as it arrives
    reqs[1].timeout = 0.0        # times out before it can be admitted
    budget = needs[reqs[2].rid] + needs[reqs[3].rid]
    sims, _ = fake_device(monkeypatch, needs)
    # a client that cancels request 2 while it is resident
    real_batch = serve.D.batch_step
    quanta = []

    def batch_step(group, n):
        quanta.append([s.req.rid for s in group])
        if len(quanta) == 2:
            reqs[2].cancel_after = 0.0  # the client cancels now
        real_batch(group, n)

    monkeypatch.setattr(serve.D, "batch_step", batch_step)
    out = serve.Server(hbm_budget=max(budget, max(needs.values())), quantum=8, stream=FakeStream()).run(reqs)
    st = {r.rid: r for r in out["results"]}
    assert st[reqs[0].rid].status == "cancelled" and reqs[0].rid not in sims
    assert st[reqs[1].rid].status == "timeout" and reqs[1].rid not in sims
    assert st[reqs[2].rid].status == "cancelled" and sims[reqs[2].rid].closed
    assert 0 < st[reqs[2].rid].lups < reqs[2].lups  # it had run a few quanta
    assert all(st[r.rid].status == "ok" for r in reqs[3:])
    assert not FakeSim.alive
    assert out["served"] == len(reqs) - 3 and out["status_counts"]["cancelled"] == 2


def test_work_policy_shares_by_work(monkeypatch):
    """Under the "work" policy a resident with 2^k times fewer cells than the
    largest advances 2^k times as many steps per round (at most max_boost
    times the quantum, never past its last step); every request still gets
    exactly its steps, and a small request next to a large one finishes in
    fewer rounds than under "lockstep"."""
    import numpy as np
    from paper_1309_3452_gb300 import workloads as W

    def two_requests():
        big = W.Problem(3, (64, 64, 64), (1.0, 1.0, 1.0), 0.5, 0.5)
        small = W.Problem(3, (16, 16, 16), (1.0, 1.0, 1.0), 0.5, 0.5)  # 64 x fewer cells
        return [serve.Request(0, 0.0, big, 4.0, (0.0, 0.0, 0.0), (32.0, 32.0, 32.0), 1000),
                serve.Request(1, 0.0, small, 2.0, (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1000)]

    rounds = {}
    for policy in ("lockstep", "work"):
        FakeSim.alive = []
        reqs = two_requests()
        sims, calls = {}, []

        def admit(self, req):
            sims[req.rid] = FakeSim(req, 1)
            return sims[req.rid]

        def batch_step(group, n):
            calls.append((sorted(s.req.rid for s in group), n))
            for s in group:
                s.steps += n
                s.launches += 1
                assert s.steps <= s.req.steps

        monkeypatch.setattr(serve.Server, "_admit", admit)
        monkeypatch.setattr(serve.D, "batch_step", batch_step)
        srv = serve.Server(hbm_budget=1 << 40, quantum=50, stream=FakeStream(), policy=policy, max_boost=8)
        out = srv.run(reqs)
        assert all(sims[r.rid].steps == r.steps for r in reqs)
        assert out["served"] == 2
        # the round in which the small request received its last steps
        rounds[policy] = next(i for i, (ids, _) in enumerate(calls)
                              if 1 in ids and sum(n for j, n in calls[:i + 1] if 1 in j) == 1000)
        if policy == "work":
            first = dict((tuple(ids), n) for ids, n in calls[:2])
            assert first[(0,)] == 50 and first[(1,)] == 400  # boost capped at 8 (64 x fewer cells)
    assert rounds["work"] < rounds["lockstep"]
    with pytest.raises(ValueError):
        serve.Server(hbm_budget=1, stream=FakeStream(), policy="fifo")
    del np
