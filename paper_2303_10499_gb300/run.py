"""Command-line runner: advance one of the named workloads on the GPU and
print the solver statistics, the time per step and, with --eager, the
per-kernel times of each step.

    python -m paper_2303_10499_gb300.run --workload bubble640x320 --steps 10
        [--mixed] [--graph] [--eager]

--eager advances every step with gea_profile_step: the kernels of the CUDA
graph launched one by one from the host, each bracketed by CUDA events (the
form a kernel profiler can attach to; kernels inside a graph with conditional
nodes cannot be profiled individually).
"""
import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="bubble640x320")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--mixed", action="store_true", help="mixed-precision step")
    ap.add_argument("--graph", action="store_true", help="CUDA-graph driver")
    ap.add_argument("--eager", action="store_true", help="per-kernel launches (profiled step)")
    args = ap.parse_args(argv)

    import torch
    from . import build as B
    from . import gea
    from . import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    B.build()
    wl = W.get(args.workload)
    s = gea.Solver(wl.grid, wl.const, graph=args.graph, mixed=args.mixed)
    s.set_conservative(wl.fields)
    per_kernel = {}
    t0 = time.perf_counter()
    for _ in range(args.steps):
        if args.eager:
            for k, v in s.profile_step().items():
                a = per_kernel.setdefault(k, {"launches": 0, "cells": 0, "ms": 0.0})
                for f in a:
                    a[f] += v[f]
        else:
            s.step(1)
    dt = time.perf_counter() - t0
    out = {"workload": wl.name, "steps": args.steps, "host_ms_per_step": dt * 1e3 / max(args.steps, 1),
           "stats": s.stats()}
    if per_kernel:
        out["per_kernel"] = per_kernel
    print(json.dumps(out))
    s.close()


if __name__ == "__main__":
    main()
