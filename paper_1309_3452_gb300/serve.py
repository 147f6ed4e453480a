"""Serving loop: continuous batching of many simulations on one GPU.

Requests (a grid, a mass, an optional Klein step, an initial packet and a
number of time steps) arrive over time.  The server admits a request as soon
as it has arrived and its device state fits the HBM budget next to the
simulations already resident, keeps every admitted state resident until its
steps are done, and advances all resident simulations together with
dirac_batch_step in rounds: under the "lockstep" policy every resident
advances by at most `quantum` steps per round (shortened so the request that
finishes first finishes exactly); under "work" a resident with 2^k times fewer
cells than the largest advances 2^k times as many steps (capped, never past
its last step), so the residents share the device by work.  Between rounds finished
requests leave (their conserved functional is read and checked against the
value reduced when their state was set) and waiting ones join.  Latency =
finish - arrival on the wall clock.

Admission never waits for the device: the initial packet is built and set on
the server's stream, and the functional of the initial state, reduced there
by dirac_set_spinor, is read only when the request retires.  A request that
can never fit the budget is rejected; one whose creation fails with
DIRAC_ERR_OOM (the device has less free memory than the budget assumed) waits
until a resident request has retired and is then tried again (rejected if
nothing else is resident); a request may be cancelled by its client or time
out, before or after admission, and then leaves between rounds, freeing its
memory.

The stepping, the norms and the state set-up all run in libdirac; this
module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import statistics
import time
from typing import List, Optional

import numpy as np

from . import dirac as D
from . import workloads as W


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the stream
    prob: W.Problem
    sigma: float
    k0: tuple
    center: tuple
    steps: int
    precision: int = D.FP32
    cancel_after: Optional[float] = None  # the client cancels this long after arrival (s)
    timeout: Optional[float] = None       # dropped once its latency would exceed this (s)

    @property
    def lups(self) -> float:
        return float(self.prob.cells) * self.steps


def make_requests(n: int, seed: int = 0, rate: float = 1.0, max_side_3d: int = 384,
                  max_side_2d: int = 4096, min_steps: int = 100, max_steps: int = 5000) -> List[Request]:
    """Seeded request stream: Poisson arrivals with the given rate (1/s); each
    request is (2+1)D with probability 1/2 (side ~ U{64..max_side_2d}) else
    (3+1)D (side ~ U{32..max_side_3d}); m ~ U[0,1]; a Klein step along x
    with probability 1/2; steps ~ U{min_steps..max_steps}; packet sigma =
    side/8 at a quarter of the box (Klein) or the centre, k0 as the (3+1)D
    workload (u*d, d uniform on the sphere, u ~ U[0,1])."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        dims = 2 if rng.random() < 0.5 else 3
        side = int(rng.integers(64, max_side_2d + 1)) if dims == 2 else int(rng.integers(32, max_side_3d + 1))
        m = float(rng.random())
        klein = rng.random() < 0.5
        steps = int(rng.integers(min_steps, max_steps + 1))
        d = rng.standard_normal(3)
        k0 = tuple(float(v) for v in rng.random() * d / np.linalg.norm(d))
        N = (side, side, side) if dims == 3 else (side, side, 1)
        fields = W.Fields()
        if klein:
            E = math.sqrt(m * m + k0[0] ** 2)
            fields = W.Fields(step_axis=0, step_x0=side / 2.0 + 0.25, step_V=2.0 * E + m)
        prob = W.Problem(dims, N, (1.0, 1.0, 1.0), 0.9 * W.stability_limit(dims), m, fields)
        c = side / 4.0 if klein else side / 2.0
        center = (c, side / 2.0, side / 2.0)
        out.append(Request(i, t, prob, side / 8.0, k0[:dims], center[:dims], steps))
    return out


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float          # nan if never admitted
    finished: float          # when it retired, was rejected, cancelled or timed out
    lups: float              # site updates done for it
    E0: float
    E1: float
    status: str = "ok"       # ok | rejected | oom | cancelled | timeout
    state: Optional[np.ndarray] = None  # the final state (Server(keep_states=True))

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    def __init__(self, hbm_budget: int, quantum: int = 100, stream=None, device="cuda",
                 keep_states: bool = False, drift_tol: float = 1e-6, policy: str = "work",
                 max_boost: int = 64):
        import torch
        if policy not in ("lockstep", "work"):
            raise ValueError(f"unknown policy {policy}")
        self.torch = torch
        self.budget = int(hbm_budget)
        self.quantum = int(quantum)
        self.policy = policy
        self.max_boost = int(max_boost)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.device = device
        self.keep_states = keep_states
        self.drift_tol = drift_tol

    def _admit(self, req: Request):
        """Create the request's simulation and enqueue its initial state on the
        server's stream; nothing here waits for the device.  The packet tensor
        belongs to the stream (caching allocator), so releasing it right away
        is safe: its memory is reused only by later work on that stream."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            psi = W.gaussian_packet_torch(req.prob, req.sigma, req.k0, req.center, self.device)
        sim = D.Sim(req.prob, req.precision, stream=self.stream.cuda_stream)
        try:
            sim.set_spinor_device(psi.data_ptr())
        except Exception:
            sim.close()
            raise
        del psi
        return sim

    def _retire(self, sim):
        """(E0, E1, state): the functional of the initial state (reduced when it
        was set) and of the final one (dirac_check, which also tests the
        paper's bounds); synchronises the stream."""
        _, r = sim.check(self.drift_tol)
        state = sim.get_spinor() if self.keep_states else None
        return r["E_ref"], r["E"], state

    def _round(self, resident):
        """[(steps, members)]: the batch_step calls of one round.  "lockstep":
        every resident advances the same number of steps, at most `quantum`
        and no more than the nearest finish needs, so a request's latency
        follows its number of steps.  "work": a resident with 2^k times fewer
        cells than the largest one advances 2^k times further (k at most
        log2(max_boost), never past its last step), so the residents receive
        about equal work per round and a request's latency follows its own
        work (cells x steps)."""
        if self.policy == "lockstep":
            return [(min(self.quantum, min(r[2] for r in resident)), list(resident))]
        cmax = max(r[0].prob.cells for r in resident)
        groups = collections.OrderedDict()
        for r in resident:
            boost = 1
            while boost < self.max_boost and r[0].prob.cells * boost * 2 <= cmax:
                boost *= 2
            groups.setdefault(min(self.quantum * boost, r[2]), []).append(r)
        return list(groups.items())

    def run(self, requests: List[Request], log=None) -> dict:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        resident = []  # [req, sim, remaining, admitted, bytes]
        used = 0
        results: List[Result] = []
        launches = 0
        self.oom_backoffs = 0
        hold = False  # an admission failed with DIRAC_ERR_OOM: wait for a retirement
        nan = float("nan")
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0

        def gone(req, t):
            """the client's cancel time or the timeout has passed at time t"""
            if req.cancel_after is not None and t >= req.arrival + req.cancel_after:
                return "cancelled"
            if req.timeout is not None and t >= req.arrival + req.timeout:
                return "timeout"
            return None

        while pending or resident:
            # drop waiting requests that were cancelled or timed out
            for req in [r for r in pending if r.arrival <= now() and gone(r, now())]:
                pending.remove(req)
                results.append(Result(req.rid, req.arrival, nan, now(), 0.0, nan, nan, gone(req, now())))
            # admit every arrived request that fits
            while pending and pending[0].arrival <= now() and not hold:
                req = pending[0]
                need = D.state_bytes(req.prob.dims, req.prob.N, req.precision)
                if need > self.budget:  # can never fit
                    pending.popleft()
                    results.append(Result(req.rid, req.arrival, nan, now(), 0.0, nan, nan, "rejected"))
                    continue
                if used + need > self.budget:
                    break
                try:
                    sim = self._admit(req)
                except D.DiracError as e:
                    if e.status != D.ERR_OOM:
                        raise
                    self.oom_backoffs += 1
                    if not resident:  # nothing will free memory for it
                        pending.popleft()
                        results.append(Result(req.rid, req.arrival, nan, now(), 0.0, nan, nan, "oom"))
                        continue
                    hold = True
                    break
                pending.popleft()
                resident.append([req, sim, req.steps, now(), need])
                used += need
            if not resident:
                if pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival - now())))
                continue
            for n, members in self._round(resident):
                sims = [r[1] for r in members]
                before = sum(s.launches for s in sims)
                D.batch_step(sims, n)
                launches += sum(s.launches for s in sims) - before
                for r in members:
                    r[2] -= n
            leaving = [r for r in resident if r[2] == 0 or gone(r[0], now())]
            if leaving:
                for r in leaving:
                    req, sim, left, adm, need = r
                    status = "ok" if left == 0 else gone(req, now())
                    if status == "ok":
                        E0, E1, state = self._retire(sim)
                    else:
                        E0, E1, state = nan, nan, None
                    results.append(Result(req.rid, req.arrival, adm, now(), req.prob.cells * (req.steps - left),
                                          E0, E1, status, state))
                    sim.close()
                    used -= need
                    if log:
                        log(f"{status} {req.rid}: {req.prob.dims}D N={req.prob.N[0]} steps={req.steps} "
                            f"latency {results[-1].latency:.2f}s")
                resident = [r for r in resident if not any(r is x for x in leaving)]
                hold = False
            else:
                self.stream.synchronize()
        makespan = now()
        ok = [r for r in results if r.status == "ok"]
        lat = sorted(r.latency for r in ok)
        total = sum(r.lups for r in results)
        drift = max((abs(r.E1 - r.E0) / abs(r.E0) for r in ok), default=nan)
        counts = collections.Counter(r.status for r in results)
        return {"requests": len(results), "served": len(ok), "status_counts": dict(counts),
                "makespan_s": makespan, "glups": total / makespan / 1e9,
                "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
                "mean_s": statistics.mean(lat) if lat else nan,
                "max_E_drift": drift, "gpu_launches": launches, "total_lups": total,
                "oom_backoffs": self.oom_backoffs, "results": results}


def percentile(sorted_vals, p):
    if not sorted_vals:
        return float("nan")
    k = (len(sorted_vals) - 1) * p / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return sorted_vals[lo] + (sorted_vals[hi] - sorted_vals[lo]) * (k - lo)


def plain_fp64_glups(requests: List[Request], device="cuda") -> float:
    """The plain path: each request alone, FP64, one simulation per launch
    sequence (no batching), back to back; site updates per second."""
    import torch
    total, t = 0.0, 0.0
    stream = torch.cuda.Stream()
    for req in requests:
        with torch.cuda.stream(stream):
            psi = W.gaussian_packet_torch(req.prob, req.sigma, req.k0, req.center, device)
        with D.Sim(req.prob, D.FP64, stream=stream.cuda_stream) as sim:
            sim.set_spinor_device(psi.data_ptr())
            sim.norm()
            del psi
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(req.steps)
            sim.norm()
            b.record(stream)
            b.synchronize()
            t += a.elapsed_time(b) / 1e3
            total += req.lups
    return total / t / 1e9
