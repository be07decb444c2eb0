"""Command-line runner: advance one of the named workloads on the GPU and
print the solver statistics, the time per step and, with --eager, the
per-kernel times of each step.

    python -m paper_2303_10499_gb300.run --workload bubble640x320 --steps 10
        [--mixed] [--graph] [--eager]
    python -m paper_2303_10499_gb300.run --ensemble 12 --steps 2
    python -m paper_2303_10499_gb300.run --conv 16,16,0 --h 2048 --w 4096 --steps 5
    python -m paper_2303_10499_gb300.run --workload bubble3d_192x192x96 --steps 3 [--eager]
    python -m paper_2303_10499_gb300.run --workload bubble640x320 --steps 5 --trace

--eager advances every step with gea_profile_step: the kernels of the CUDA
graph launched one by one from the host, each bracketed by CUDA events (the
form a kernel profiler can attach to; kernels inside a graph with conditional
nodes cannot be profiled individually).

--trace advances --steps steps, then traces one more step of the persistent
driver (gea_set_trace) and prints one line per phase: the grid barrier that
ends it, the mean and largest time a block spent in the phase (from its
release from the previous barrier, or its entry, to its arrival), and the
time from the last arrival to the releases.
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
    ap.add_argument("--trace", action="store_true", help="phase trace of one persistent step")
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
    if args.trace:
        return run_trace(args, s, wl)
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


def phase_labels(st, n_corr, les):
    """Names of the phases of one FP64 persistent step with a one-level
    preconditioner, in the order of their grid barriers (the structure of
    the step kernel), from the step's sweep and iteration counts."""
    lab = ["LES eddy viscosity"] if les else []
    lab.append("Step 1: predictor set-up + momentum sweep 1")
    lab += [f"momentum sweep {j}" for j in range(2, st["jac_u"] + 1)]
    lab.append("Step 2: enthalpy right-hand side + sweep 1")
    lab += [f"enthalpy sweep {j}" for j in range(2, st["jac_h"] + 1)]
    lab.append("EOS update + H(u)")
    for c in range(n_corr):
        if c > 0:
            lab.append("H(u)")
        lab.append(f"corrector {c + 1}: pressure right-hand side")
        its = st["cg_iters"][c]
        if its > 0:
            lab.append(f"corrector {c + 1}: first preconditioning")
        for i in range(1, its + 1):
            lab += [f"corrector {c + 1}: CG {i} p, A p", f"corrector {c + 1}: CG {i} update + preconditioning"]
        if c + 1 < n_corr:
            lab.append(f"corrector {c + 1}: correction")
    lab.append(f"corrector {n_corr}: correction + step end")
    return lab


def run_trace(args, s, wl):
    import numpy as np
    for _ in range(args.steps):
        s.step(1)
    tr = s.trace_step()
    st = s.stats()
    a, r = tr["arrive"], tr["release"]
    prev = np.vstack([tr["entry"][None, :], r[:-1]])
    work = (a - prev) / 1e3
    lab = None
    if st["driver"] == "persistent" and st["mg_levels"] == 1:
        lab = phase_labels(st, wl.const.n_corr, wl.const.cs > 0)
        if len(lab) != tr["barriers"]:
            lab = None
    for k in range(tr["barriers"]):
        print(json.dumps({"barrier": k + 1, "phase": lab[k] if lab else None,
                          "block_us_mean": round(float(work[k].mean()), 2),
                          "block_us_max": round(float(work[k].max()), 2),
                          "release_after_last_arrival_us": round(float((r[k] - a[k].max()).mean() / 1e3), 2)}))
    step_us = float(r[-1].max()) / 1e3
    print(json.dumps({"workload": wl.name, "driver": st["driver"], "blocks": tr["blocks"],
                      "barriers": tr["barriers"], "step_us": round(step_us, 1),
                      "sum_block_us_max": round(float(work.max(axis=1).sum()), 1),
                      "sum_block_us_mean": round(float(work.mean(axis=1).sum()), 1),
                      "sum_release_us": round(float(sum((r[k] - a[k].max()).mean() for k in range(tr["barriers"])) / 1e3), 1),
                      "stats": st}))
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
