"""Measured ceilings of this GPU for the roofline of the FP64 path.

The FP32 stencil is held against the HBM copy bandwidth; the FP64 path
(per-site FP64 arithmetic, GB300's FP64 rate is a small fraction of its FP32
rate) is held against the FP64 arithmetic rate.  This module measures that
rate with the library's FP64 FMA-chain kernel (dirac_fp64_fma_rate), and for
reference a large FP64 matrix product (cuBLAS DGEMM: 2 n^3 flops, best of
several runs, CUDA events) and the copy bandwidth, and prints one JSON line.

  python -m paper_1309_3452_gb300.peaks [--n 8192] [--reps 5]
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    n = args.n
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = torch.empty_like(a)
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    fp64_tflops = 2.0 * n ** 3 / best / 1e12
    del a, b, c
    x = torch.empty(1 << 28, dtype=torch.float64, device=dev)  # 2 GiB
    y = torch.empty_like(x)
    y.copy_(x)
    torch.cuda.synchronize()
    cbest = float("inf")
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        y.copy_(x)
        e1.record()
        e1.synchronize()
        cbest = min(cbest, e0.elapsed_time(e1) / 1e3)
    copy_gbs = 2.0 * x.numel() * 8 / cbest / 1e9
    from . import dirac as D
    fma = D.fp64_fma_rate()
    print(json.dumps({"fp64_fma_tflops": fma, "how_fp64_fma": "dirac_fp64_fma_rate: independent FP64 FMA "
                      "chains, 8 per thread, 2 flops per FMA, best of 3",
                      "fp64_dgemm_tflops": fp64_tflops, "how_fp64": f"torch.matmul float64 {n}^3, 2 n^3 flops, "
                      f"best of {args.reps}", "copy_gbs": copy_gbs,
                      "how_copy": "copy of 2 GiB float64 (read + write bytes), best of "
                                  f"{args.reps}", "gpu": torch.cuda.get_device_name(dev)}), flush=True)


if __name__ == "__main__":
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
