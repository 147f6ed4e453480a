#!/usr/bin/env python
"""Throughput benchmark of the staggered leap-frog Dirac stepper on GB300.

One benchmark step = one pass of the whole hot path over one workload: with
the state resident in HBM, advance it by the workload's number of time steps
(both half-steps each) and evaluate the conserved functional E (FP64).

Default workload (the largest single-GPU configuration): (3+1)D 512^3
periodic grid, m = 1, soft-core potential -1/sqrt(|x-c|^2+1) at the centre
plus a moving plane-wave vector potential A_x = 0.5 cos(2 pi z/64 - omega t),
seeded Gaussian packet (sigma = 24), 2000 time steps, FP32 stencil with FP64
reductions.  Others: --workload 3d128 (1000 steps, no fields), 2d4096 (Klein
step, 5000 steps), 3d512, 2d4096k37, 3d256laser, 3d128links, 2d2048links,
2d64, serve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: one independent replica per GPU (the method is
advanced per simulation; replicas need no data exchange), timing is the max
over ranks, value = total site updates / time.

Prints ONE JSON line (rank 0).  GLUPS = cells x time steps / s / 1e9 (one
site update = one unit cell advanced one full time step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spinor site-updates/s (GLUPS) & % HBM roofline; served p50/p99 latency"
L2_BYTES = 129 * 1024 * 1024


# host states larger than this are built in place (separable generator) and
# the oracle's CPU sample takes a window of the grid instead of all of it
BIG_STATE_BYTES = 2 << 30


def workload(name):
    """(prob, state, n, desc): state is a canonical complex128 array, or
    ("packet", sigma, k0, center) for grids whose host state is built in place."""
    from paper_1309_3452_gb300 import workloads as W
    if name == "3d512laser":
        prob, _, n = W.workload_laser(N=512, steps=2000, packet=False)
        state = ("packet", 24.0, tuple(W.random_k0(1)), (256.0, 256.0, 256.0))
        desc = ("(3+1)D 512^3 periodic, m=1, soft core -1/sqrt(|x-c|^2+1) at the centre + A_x = 0.5 "
                "cos(2 pi z/64 - omega t), omega = 2 pi/64, Gaussian packet sigma=24 at the centre, seeded k0 "
                "(|k0|<=1), dt=0.9/sqrt(3), 2000 time steps + E per step")
    elif name == "3d128":
        prob, state, n = W.workload_3d(N=128, steps=1000)
        desc = ("(3+1)D 128^3 periodic, m=1, no fields, Gaussian packet sigma=10 at the centre, "
                "seeded k0 (|k0|<=1), dt=0.9/sqrt(3), 1000 time steps + E per step")
    elif name == "3d512":
        prob, _, n = W.workload_3d(N=512, steps=200, sigma=24.0, packet=False)
        state = ("packet", 24.0, tuple(W.random_k0(0)), (256.0, 256.0, 256.0))
        desc = "(3+1)D 512^3 periodic, m=1, no fields, packet sigma=24, 200 time steps + E per step"
    elif name == "3d256laser":  # the laser fields on a 256^3 grid (profiling size)
        prob, _, _ = W.workload_laser(N=256, steps=2000, packet=False)
        n = 50
        state = ("packet", 24.0, tuple(W.random_k0(1)), (128.0, 128.0, 128.0))
        desc = ("(3+1)D 256^3, m=1, soft core -1/sqrt(|x-c|^2+1) at the centre + A_x = 0.5 cos(2 pi z/64 - "
                "omega t), packet sigma=24 seeded k0; 50 time steps + E per step")
    elif name == "2d4096":
        prob, state, n = W.workload_klein(N=4096, steps=5000)
        desc = ("(2+1)D 4096^2 Klein step (V0 = 2E+m at x0 = N/2+1/4), m=0.2, packet sigma=40, "
                "5000 time steps + E per step")
    elif name == "2d4096k37":
        prob, state, n = W.workload_klein_oblique(N=4096)
        desc = ("(2+1)D 4096^2 Klein refraction (Sect. 5): m=0, step V=2E at x0=N/2+1/4, packet sigma=64, "
                f"|k0|=0.25 at 37 deg to the step; {n} time steps + E per step")
    elif name == "3d128links":
        prob, state, n = W.workload_links(3, 128, 200)
        desc = ("(3+1)D 128^3 periodic, m=1, static vector potential given by seeded random link "
                "integrals in [-0.3, 0.3] (q=1), packet as 3d128; 200 time steps + E per step")
    elif name == "2d2048links":
        prob, state, n = W.workload_links(2, 2048, 200)
        desc = ("(2+1)D 2048^2 periodic, m=1, static vector potential given by seeded random link "
                "integrals in [-0.3, 0.3] (q=1), packet sigma=10; 200 time steps + E per step")
    elif name == "2d64":
        prob, state, n = W.workload_2d64(0.5)
        desc = "(2+1)D 64^2, m=0.5, packet sigma=6, 200 time steps + E per step"
    else:
        raise SystemExit(f"unknown workload {name}")
    return prob, state, n, desc


def host_state(prob, state, pinned):
    """The canonical complex128 host state: (numpy view, torch buffer or None).
    Packets are written in place into the (page-locked) buffer."""
    import numpy as np
    from paper_1309_3452_gb300 import workloads as W
    buf = None
    if pinned:
        import torch
        buf = torch.empty(tuple(prob.shape) + (2,), dtype=torch.float64, pin_memory=True)
        arr = buf.numpy().view(np.complex128).reshape(prob.shape)
    else:
        arr = np.empty(prob.shape, np.complex128)
    if isinstance(state, tuple):
        _, sigma, k0, center = state
        W.gaussian_packet_separable(prob, sigma, k0, center, out=arr)
    else:
        arr[...] = state
    return arr, buf


def cpu_sample(prob, state):
    """The oracle's bounded CPU sample of a workload: the grid itself, or for
    states above BIG_STATE_BYTES a window of half the extent per axis around
    the packet, with the fields at their true positions (the oracle's origin)
    and the packet sampled there.  Returns (prob, psi, origin, what)."""
    import numpy as np
    from paper_1309_3452_gb300 import workloads as W
    nbytes = int(np.prod(prob.shape)) * 16
    if nbytes <= BIG_STATE_BYTES:
        psi, _ = host_state(prob, state, pinned=False)
        return prob, psi, (0, 0, 0), "the full grid"
    _, sigma, k0, center = state
    Nw = [max(2, n // 2) if a < prob.dims else 1 for a, n in enumerate(prob.N)]
    origin = [int(center[a] - Nw[a] / 2) if a < prob.dims else 0 for a in range(3)]
    wp = W.Problem(prob.dims, tuple(Nw), prob.dx, prob.dt, prob.m, prob.fields)
    psi = W.gaussian_packet_separable(wp, sigma, k0, center, origin=origin, box=prob.N)
    what = (f"a {'x'.join(map(str, Nw[:prob.dims]))} window of the grid at cell {origin[:prob.dims]} "
            f"(same fields at their true positions, the packet sampled there)")
    return wp, psi, tuple(origin), what


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.f:
            return None
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.f.name)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


KERNEL_SOURCES = {  # the files that determine each timed kernel's code
    "step_fp32": ["step_fused.cu", "common.cuh", "kernels.cuh"],
    "step_fp64": ["step_split.cu", "common.cuh", "kernels.cuh"],
}


def max_over_ranks(value, dist, device=None):
    """The maximum of a per-rank float over all ranks (the slowest rank's
    time); returns the local value when not distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(lups_per_rank, world, seconds):
    """Replicas: every rank advances its own simulation, so the job's
    throughput is world x the per-rank site updates over the slowest rank's time."""
    return world * lups_per_rank / seconds / 1e9


def kernel_source_hash(kernel):
    """The first 12 hex digits of the SHA-1 of the kernel's source files with
    comments and white space removed: an edited comment keeps a capture's
    counters valid, any change of the code does not."""
    h = hashlib.sha1()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1309_3452_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, workload_name):
    """DRAM bytes per launch from a committed ncu summary, valid only while
    the kernel sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(f"{kernel}@{workload_name}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def oracle_rate(prob, psi, origin, budget_s):
    """Time steps of the oracle on (prob, psi) that take about budget_s
    seconds, from a one-step and a three-step probe."""
    from oracle import oracle as O
    t = time.perf_counter()
    st = O.step(prob, psi, 1, origin=origin)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    st = O.step(prob, st, 3, origin=origin)
    t3 = time.perf_counter() - t
    per_step = max((t3 - t1) / 2.0, 1e-4)
    return st, max(1, min(2000, int(budget_s / per_step)))


def cpu_baseline(prob, state, budget_s=15.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload:
    as many time steps of the same grid (or of a window of it) as fit in
    about budget_s seconds."""
    from oracle import oracle as O
    O.build()
    sp, psi, origin, what = cpu_sample(prob, state)
    st, k = oracle_rate(sp, psi, origin, budget_s)
    t = time.perf_counter()
    O.step(sp, st, k, origin=origin)
    dt = time.perf_counter() - t
    return {"value": sp.cells * k / dt / 1e9, "unit": "GLUPS", "cores": O.threads(), "kind": "oracle",
            "sample": f"{k} time steps of {what} (FP64, {dt:.1f} s incl. layout conversion)"}


def run_reference(args, prob, state, n, desc, rank, world):
    from oracle import oracle as O
    if rank != 0:
        return
    O.build()
    sp, psi, origin, what = cpu_sample(prob, state)
    st, per_step = oracle_rate(sp, psi, origin, 8.0)  # each bench step: ~8 s of CPU work
    per_step = min(per_step, 20)
    for _ in range(args.warmup):
        st = O.step(sp, st, per_step, origin=origin)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        st = O.step(sp, st, per_step, origin=origin)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = sp.cells * per_step * args.steps / total / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": desc, "grid": list(prob.N[:prob.dims]), "sample": what,
                      "time_steps_per_step": per_step, "precision": "fp64 (CPU oracle)",
                      "parallelism": "oracle, rank 0 only"},
           "cpu_baseline": {"kind": "oracle", "cores": O.threads(), "value": value, "unit": "GLUPS",
                            "sample": f"{per_step} time steps per step of {what} of the {desc} workload"},
           "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serve(args, rank, world):
    """Serving stream: seeded Poisson requests of mixed (2+1)D / (3+1)D sizes,
    masses, Klein steps and step counts, FP32, admitted by free HBM and
    continuously batched (paper_1309_3452_gb300/serve.py).

    Arrival rate: --rate, else 0.8 x the sustainable rate, found by a sweep:
    the capacity C (requests/s) is measured on a burst of the stream's first
    requests (all arriving at once), then prefixes of the stream run at
    0.5 C, 0.7 C, 0.85 C and 1.0 C; the sustainable rate is the highest at
    which p99 latency stays within 3x its value at 0.5 C (the queue does not
    grow without bound)."""
    import torch
    from paper_1309_3452_gb300 import serve
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    srv = serve.Server(budget, quantum=args.quantum, policy=args.serve_policy)
    stream = serve.make_requests(args.requests, seed=args.seed, rate=1.0)
    mean_lups = sum(r.lups for r in stream) / len(stream)
    sweep = []
    if args.rate > 0:
        rate = args.rate
        rule = "given (--rate)"
        glups_sat = None
    else:
        m = args.sweep_requests
        burst = serve.make_requests(m, seed=args.seed, rate=1e9)
        srv.run(burst[:8])  # the process's first launches, allocations and module loads, untimed
        c = srv.run(burst)
        glups_sat = c["glups"]
        cap = glups_sat * 1e9 / (sum(r.lups for r in burst) / len(burst))
        base = None
        sustainable = 0.5 * cap
        for f in (0.5, 0.7, 0.85, 1.0):
            o = srv.run(serve.make_requests(m, seed=args.seed, rate=f * cap))
            sweep.append({"rate_per_s": f * cap, "p50_s": o["p50_s"], "p99_s": o["p99_s"],
                          "glups": o["glups"]})
            base = o["p99_s"] if base is None else base
            if o["p99_s"] <= 3.0 * base:
                sustainable = f * cap
        rate = 0.8 * sustainable
        rule = ("0.8 x the sustainable rate of a sweep over prefixes of the stream "
                f"({m} requests each; burst capacity {cap:.3f}/s)")
    reqs = serve.make_requests(args.requests, seed=args.seed, rate=rate)
    log = None
    if args.progress:
        def log(msg):
            print(msg, file=sys.stderr, flush=True)
        log(f"rate {rate:.4f}/s ({rule}); sweep {sweep}")
    with Clocks(local) as clk:
        out = srv.run(reqs, log=log)
    # the plain FP64 path (one simulation per launch sequence) on a subsample
    sub = []
    for r in reqs[:8]:
        r2 = serve.Request(r.rid, 0.0, r.prob, r.sigma, r.k0, r.center, min(r.steps, 200))
        sub.append(r2)
    fp64 = serve.plain_fp64_glups(sub)
    served_bytes = sum(r.lups * (128.0 if r.prob.dims == 3 else 64.0) for r in reqs)
    peak = None
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except Exception:
        pass
    achieved = served_bytes / out["makespan_s"] / 1e9
    # latency by request size (thirds of the served requests by site updates):
    # the spread of p99 over p50 mostly reflects the spread of the sizes
    by_size = None
    okr = sorted((r for r in out["results"] if r.status == "ok"), key=lambda r: r.lups)
    if len(okr) >= 3:
        by_size = []
        for part in (okr[:len(okr) // 3], okr[len(okr) // 3:2 * len(okr) // 3], okr[2 * len(okr) // 3:]):
            lat = sorted(r.latency for r in part)
            by_size.append({"requests": len(part), "site_updates_max": part[-1].lups,
                            "p50_s": serve.percentile(lat, 50), "p99_s": serve.percentile(lat, 99)})
    res = {"metric": METRIC, "value": out["glups"], "unit": "GLUPS", "n_gpus": world,
           "steps": out["requests"], "warmup": 8, "ms_per_step": 1000.0 * out["makespan_s"] / out["requests"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "serving stream: seeded Poisson arrivals; each request (2+1)D side "
                                  "U{64..4096} or (3+1)D side U{32..384} (p = 1/2), m ~ U[0,1], Klein step "
                                  "p = 1/2, 100..5000 steps, FP32; admitted by free HBM, continuously "
                                  "batched in quanta",
                      "requests": out["requests"], "seed": args.seed, "rate_per_s": rate, "rate_rule": rule,
                      "rate_sweep": sweep, "burst_glups": glups_sat, "quantum_steps": args.quantum, "policy": args.serve_policy,
                      "hbm_budget_bytes": budget, "parallelism": f"replicas x{world}"},
           "serving": {"p50_latency_s": out["p50_s"], "p99_latency_s": out["p99_s"],
                       "mean_latency_s": out["mean_s"], "makespan_s": out["makespan_s"],
                       "max_E_rel_drift": out["max_E_drift"], "total_site_updates": out["total_lups"],
                       "status_counts": out["status_counts"], "oom_backoffs": out["oom_backoffs"],
                       "latency_by_size": by_size},
           "fp64_plain": {"value": fp64, "unit": "GLUPS",
                          "sample": "the stream's first 8 requests, min(steps, 200) each, one FP64 "
                                    "simulation at a time"},
           "ratio_served_fp32_vs_plain_fp64": out["glups"] / fp64,
           "gpu_launches": out["gpu_launches"], "clocks": clk.summary(),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak if peak else None, "traffic": None,
                        "note": "served site updates x algorithmic bytes (128 B (3+1)D, 64 B (2+1)D) over "
                                "the wall-clock makespan"},
           "cpu_baseline": None,
           "e2e": None, "e2e_note": "requests carry parameters; packets are built on the device (no host "
                                    "state to copy); value is already wall clock, arrival to retirement"}
    if rank == 0:
        print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d512laser",
                    choices=["3d512laser", "3d128", "3d512", "3d256laser", "2d4096", "2d4096k37", "3d128links",
                             "2d2048links", "2d64", "serve"])
    ap.add_argument("--time-steps", type=int, default=0,
                    help="time steps per bench step instead of the workload's own (profiling runs only; "
                         "the JSON line then names the count)")
    ap.add_argument("--requests", type=int, default=40, help="serve: requests in the stream")
    ap.add_argument("--quantum", type=int, default=100, help="serve: steps per batching quantum")
    ap.add_argument("--serve-policy", default="work", choices=["lockstep", "work"],
                    help="serve: every resident the same steps per round, or the same work")
    ap.add_argument("--seed", type=int, default=0, help="serve: request stream seed")
    ap.add_argument("--sweep-requests", type=int, default=40, help="serve: requests per rate-sweep point")
    ap.add_argument("--progress", action="store_true", help="serve: log every retired request to stderr")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serve: arrival rate in requests/s (0: 0.8 x the sustainable rate, measured first)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end line (profiling runs)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison line")
    ap.add_argument("--plan", default="autotune",
                    help="launch plan: 'autotune' (timed by dirac_autotune before the warm-up), 'rule' "
                         "(the built-in rule), or a fixed 'CHUNK' / 'CHUNK:CHUNK2' (levels per work "
                         "item of the one-step / (2+1)D two-step kernel), e.g. to profile the plan "
                         "the autotuner picked")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "serve":
        return run_serve(args, rank, world)
    prob, state, n, desc = workload(args.workload)
    if args.time_steps > 0:
        n = args.time_steps
        desc += f" [profiling run: {n} time steps per bench step]"

    if args.impl == "reference":
        return run_reference(args, prob, state, n, desc, rank, world)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1309_3452_gb300 import dirac as D

    stream = torch.cuda.Stream()
    prec = D.FP32 if args.precision == "fp32" else D.FP64
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    # the canonical complex128 state in page-locked host memory (built in place for big grids)
    psi, hbuf = host_state(prob, state, pinned=True)
    nbytes = int(np.prod(prob.shape)) * 16

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        sim = D.Sim(prob, prec, stream=stream.cuda_stream)
        sim.set_spinor_ptr(hbuf.data_ptr())
    E_start, _ = sim.norm()
    # launch plan (chunk lengths, one or two steps per pass): measured on this state, untimed
    if args.plan == "autotune":
        plan = dict(sim.autotune(), source="autotune")
    elif args.plan == "rule":
        plan = dict(sim.plan, source="rule")
    else:
        c = [int(v) for v in args.plan.split(":")]
        sim.set_plan(chunk=c[0], two_step=int(prob.dims == 2 and len(c) > 1), chunk2=c[1] if len(c) > 1 else 0)
        plan = dict(sim.plan, source="fixed")

    for _ in range(args.warmup):
        sim.step(n)
        sim.norm()
    launches0 = sim.launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    norm_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    barrier()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))  # evict the state from L2 between timed steps
            torch.cuda.synchronize()
            ev[i][0].record(stream)
            sim.step(n)
            norm_ev[i][0].record(stream)
            E_end, _ = sim.norm()
            norm_ev[i][1].record(stream)
            ev[i][1].record(stream)
        barrier()
    launches = sim.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    norm_ms = [a.elapsed_time(b) for a, b in norm_ev]
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    lups = prob.cells * n
    value = whole_job_glups(lups, world, ms_per_step / 1e3)

    # dominant kernel: the time-step kernel, one launch per time step ((2+1)D: per
    # two-step pass); its time = the timed region minus the norm read, per time step.
    # Algorithmic bytes per site update: every value read once and written once
    # (16 values x 8 B in (3+1)D FP32); analytic fields add nothing.  The bytes the
    # library's path moves with its per-site tables (if any) are reported beside.
    stencil_ms = (sum(step_ms) - sum(norm_ms)) / args.steps / n
    elem = 8 if args.precision == "fp32" else 16
    bpl = 2.0 * prob.n_planes * elem
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak else "fallback"
    peak = peak or 6800.0
    achieved = bpl * prob.cells / (stencil_ms / 1e3) / 1e9
    kname = "step_fp32" if args.precision == "fp32" else "step_fp64"
    traffic = ncu_traffic(kname, args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src, "kernel": "one full time step (all launches of a step)",
                "algorithmic_bytes_per_lup": bpl, "time_step_us": stencil_ms * 1e3,
                "path_bytes_per_lup": sim.algorithmic_bytes,
                "path_bytes_note": "state plus the per-site tables the library's path reads (not the roofline)"}

    # end to end through the C ABI with the page-locked host buffer: set, step, norm, get
    e2e = None
    if not args.no_e2e:
        e2e_ms = []
        for i in range(max(1, min(3, args.steps))):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.set_spinor_ptr(hbuf.data_ptr())
            sim.step(n)
            sim.norm()
            sim.get_spinor_ptr(hbuf.data_ptr())
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_ms_step = max_over_ranks(statistics.median(e2e_ms), dist, "cuda")
        e2e = {"value": whole_job_glups(lups, world, e2e_ms_step / 1e3), "unit": "GLUPS", "ms_each": e2e_ms,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8 * 5,
               "ms_per_step": e2e_ms_step, "host_buffer": "page-locked, canonical complex128"}

    # the plain FP64 one-simulation-per-launch path on the same workload (a few time steps)
    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        with D.Sim(prob, D.FP64, stream=stream.cuda_stream) as s64:
            s64.set_spinor_ptr(hbuf.data_ptr())
            s64.step(1)
            s64.norm()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64.step(2)
            b.record(stream)
            b.synchronize()
            n64 = max(1, min(max(1, n // 10), int(3000.0 / max(a.elapsed_time(b) / 2.0, 1e-3))))
            a.record(stream)
            s64.step(n64)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            fp64 = {"value": prob.cells * n64 / (ms / 1e3) / 1e9, "unit": "GLUPS",
                    "time_steps": n64, "ms": ms}
    E_drift = abs(E_end - E_start) / abs(E_start)
    sim.close()
    del hbuf, psi

    clocks = clk.summary()
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(prob, state)
    out = {"metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
           "config": {"workload": desc, "grid": list(prob.N[:prob.dims]), "time_steps_per_step": n,
                      "precision": args.precision + (" stencil, fp64 reductions"
                                                     if args.precision == "fp32" else ""),
                      "l2": f"flushed between timed steps (write of {2 * L2_BYTES >> 20} MiB); "
                            f"state {D.state_bytes(prob.dims, prob.N, prec) >> 20} MiB",
                      "parallelism": f"replicas x{world}", "plan": plan},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": launches, "clocks": clocks, "fp64_plain": fp64,
           "E_rel_drift": E_drift}
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
