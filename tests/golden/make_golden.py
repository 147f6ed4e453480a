"""Write sampled expected values of the full-size (3+1)D 128^3 workload
(1000 time steps from the seeded Gaussian packet) computed by the FP64 CPU
oracle only.  The GPU tests compare the CUDA path with these samples.

    python tests/golden/make_golden.py        (about 3-10 min on 8-16 cores)

Output: tests/golden/workload_3d128_1000.json with the sampled sites (plane,
z, y, x), their complex values, E and the naive norm after 1000 steps.
Samples: the 256 largest-amplitude values and 256 uniformly drawn sites
(seed 0)."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1309_3452_gb300 import workloads as W  # noqa: E402


def main():
    prob, psi, n = W.workload_3d(N=128, steps=1000)
    out = O.step(prob, psi, n)
    ob = O.observables(prob, out, n * prob.dt)
    flat = np.abs(out).reshape(-1)
    top = np.argsort(flat)[-256:]
    rng = np.random.default_rng(0)
    uni = rng.choice(flat.size, 256, replace=False)
    idx = np.unique(np.concatenate([top, uni]))
    sites = [list(map(int, np.unravel_index(i, out.shape))) for i in idx]
    vals = [[float(out.reshape(-1)[i].real), float(out.reshape(-1)[i].imag)] for i in idx]
    rec = {"workload": "3d128", "steps": int(n), "dt": prob.dt, "E": ob["E"], "naive": ob["naive"],
           "E0": O.observables(prob, psi, 0.0)["E"], "rms": float(np.sqrt(np.mean(np.abs(out) ** 2))),
           "sites": sites, "values": vals,
           "source": "oracle/dirac_oracle.c via tests/golden/make_golden.py"}
    with open(os.path.join(HERE, "workload_3d128_1000.json"), "w") as f:
        json.dump(rec, f)


if __name__ == "__main__":
    main()
