"""Command-line runner: advance one of the named workloads on the GPU and
print the solver statistics, the time per step and, with --eager, the
per-kernel times of each step.

    python -m paper_2303_10499_gb300.run --workload bubble640x320 --steps 10
        [--mixed] [--graph] [--eager]
    python -m paper_2303_10499_gb300.run --ensemble 12 --steps 2
    python -m paper_2303_10499_gb300.run --conv 16,16,0 --h 2048 --w 4096 --steps 5
    python -m paper_2303_10499_gb300.run --workload bubble3d_192x192x96 --steps 3 [--eager]

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
    ap.add_argument("--ensemble", type=int, default=0,
                    help="step this many LES bubbles of the ensemble workload in one launch per step")
    ap.add_argument("--conv", default="", help="cin,cout,mode: time gea_conv3x3 on an h x w image")
    ap.add_argument("--h", type=int, default=2048)
    ap.add_argument("--w", type=int, default=4096)
    args = ap.parse_args(argv)

    import torch
    from . import build as B
    from . import gea
    from . import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    B.build()
    if args.conv:
        return run_conv(args)
    if args.ensemble:
        return run_ensemble(args)
    wl = W.get(args.workload)
    if isinstance(wl.grid, W.Grid3):
        s = gea.Solver3D(wl.grid, wl.const)
    else:
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


def run_conv(args):
    """Time the tensor-core convolution on zero data (the time does not
    depend on the values)."""
    import torch
    from . import gea
    cin, cout, mode = (int(v) for v in args.conv.split(","))
    h, w = args.h, args.w
    sh, sw = (2 * h, 2 * w) if mode == gea.CONV_POOL else (h, w)
    x0 = torch.zeros(sh * sw * cin, dtype=torch.int16, device="cuda")
    x1 = torch.zeros((h // 2) * (w // 2) * cin, dtype=torch.int16, device="cuda") if mode == gea.CONV_UPADD else None
    wt = torch.zeros(cout * 9 * cin, dtype=torch.int16, device="cuda")
    b = torch.zeros(cout, dtype=torch.float32, device="cuda")
    y = torch.zeros(h * w * cout, dtype=torch.int16, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gea.conv3x3(x0, wt, y, 1, h, w, cin, cout, mode=mode, flags=gea.CONV_RELU, x1=x1, bias=b)
    e0.record()
    for _ in range(args.steps):
        gea.conv3x3(x0, wt, y, 1, h, w, cin, cout, mode=mode, flags=gea.CONV_RELU, x1=x1, bias=b)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    byts = (sh * sw * cin + (h // 2) * (w // 2) * cin * (mode == gea.CONV_UPADD) + h * w * cout) * 2
    print(json.dumps({"conv": [cin, cout, mode], "h": h, "w": w, "ms": ms, "GB/s": byts / ms / 1e6,
                      "TFLOP/s": 2 * 9 * cin * cout * h * w / ms / 1e9}))


def run_ensemble(args):
    import torch
    from . import gea
    from . import workloads as W
    wls = W.les_ensemble(args.ensemble, seed=0)
    ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
    for sv, wl in zip(ss, wls):
        sv.set_conservative(wl.fields)
    E = gea.Ensemble(ss, stream=torch.cuda.current_stream())
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E.step(1)
    dt = time.perf_counter() - t0
    print(json.dumps({"members": len(ss), "cells": sum(wl.grid.cells for wl in wls), "steps": args.steps,
                      "host_ms_per_step": dt * 1e3 / max(args.steps, 1), "blocks": E.blocks(),
                      "stats0": ss[0].stats()}))
    E.close()


if __name__ == "__main__":
    main()
