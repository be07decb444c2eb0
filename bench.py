#!/usr/bin/env python
"""Throughput of one time step of the GEA pressure-based Euler solver
(Girfoglio, Quaini & Rozza, arXiv 2303.10499, Section 3) on GB300.

A step is one pass of the whole hot path: continuity predictor, implicit
momentum and enthalpy predictors, EOS update and the PISO correctors with
their multigrid-preconditioned CG pressure solves, on the smooth rising
bubble (640 x 320 cells, dt = 0.05 s, FP64) unless --workload says otherwise.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. value = cell-steps/s summed over ranks (each rank runs
an independent replica: the solver runs on one GPU), timed with CUDA events
on the solver's stream, L2 flushed (256 MB write) between timed steps.
--impl reference times the FP64 CPU oracle on this machine's host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-steps/sec and pressure-solve ms/step vs plain FP64 GPU at matched error"
UNIT = "cell-steps/s"

# Algorithmic traffic and arithmetic per cell of one launch: 8-byte words read
# once plus written once (an FP32 value is half a word), and operations (add,
# mul, div, sqrt each 1; an FMA counts 2) in the precision named last.
# Coarse-level multigrid kernels are per cell of the level they run on.
# Derivations are in the design notes. The mx_ kernels are the
# mixed-precision step.
KERNEL_MODEL = {
    "pred_setup": (22, 66, "f64"),
    "mom_jacobi": (16, 44, "f64"),
    "enth_rhs": (13, 41, "f64"),
    "enth_jacobi": (13, 22, "f64"),
    "eos_coef": (16, 33, "f64"),
    "mg_coarsen": (17, 18, "f64"),
    "H": (17, 44, "f64"),
    "helm_rhs": (15, 51, "f64"),
    "mg_down": (5.25, 11.5, "f64"),
    "mg_coarse": (7, 6.5, "f64"),
    "mg_up": (7.25, 15, "f64"),
    "mg_single": (6, 15, "f64"),
    "cg_pspmv": (7, 13.5, "f64"),
    "cg_update_single": (11, 22, "f64"),
    "cg_update_down": (10.25, 18, "f64"),
    "correct": (16, 38, "f64"),
    "mx_pred": (23.5, 104, "f64"),
    "mx_mom": (8, 46, "f32"),
    "mx_enth_rhs": (23.5, 70, "f64"),
    "mx_enth": (6.5, 31, "f32"),
    "mx_eos": (18, 33, "f64"),
    "mx_coarsen": (8.5, 18, "f32"),
    "mx_helm_rhs": (14.5, 51, "f64"),
    "mx_mg_down": (2.625, 11.5, "f32"),
    "mx_mg_coarse": (3.5, 6.5, "f32"),
    "mx_mg_up": (3.625, 15, "f32"),
    "mx_mg_single": (3, 15, "f32"),
    "mx_pspmv": (3.5, 13.5, "f32"),
    "mx_update_single": (5.5, 22, "f32"),
    "mx_update_down": (5.125, 18, "f32"),
    "mx_p_apply": (2.5, 1, "f64"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bubble640x320")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-w3", action="store_true",
                    help="skip the nested 4096 x 2048 FP64 record (w3) of the default line")
    ap.add_argument("--graph", action="store_true",
                    help="always step through the CUDA graph of per-phase kernels (default: the "
                         "library picks the persistent kernel on small grids)")
    ap.add_argument("--tune-tiles", action="store_true",
                    help="graph driver: run the tile-column autotuner (tiles a block walks in the "
                         "per-phase reduction kernels) before timing, from the same initial state")
    ap.add_argument("--mixed", action="store_true",
                    help="time the mixed-precision step (FP32 inner solves) on the main line; by "
                         "default it is timed beside the FP64 step under 'mixed_precision'")
    ap.add_argument("--learned", action="store_true",
                    help="the learned-preconditioner configuration: smooth bubble 4096 x 2048, pressure "
                         "solves to 1e-8 relative residual, plain MG-CG against the network's initial "
                         "guess (trained first on the solver's own pressure systems)")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="the batched LES configuration: this many non-smooth bubbles (grids 100^2, 200^2, "
                         "400^2, Smagorinsky cs = 0.17) advanced by one launch per step, against the same "
                         "members stepped one after another")
    ap.add_argument("--three-d", default=None, metavar="WORKLOAD",
                    help="the three-dimensional step on a 3D workload (bubble3d_512x512x256: the "
                         "10 km cube bubble, 67M cells)")
    ap.add_argument("--sweep", action="store_true",
                    help="the size sweep of the smooth bubble, 256 x 128 to 8192 x 4096 cells (FP64, "
                         "pressure solves to 1e-8 of ||b||): ms per step, cell-steps/s and the whole "
                         "step against the FP64 and HBM ceilings per size")
    ap.add_argument("--full-run", action="store_true",
                    help="the 640 x 320 bubble run to t = 1020 s (20,400 steps at dt = 0.05 s), FP64 "
                         "and mixed precision, with the per-field error of the mixed run at the end")
    ap.add_argument("--mixed-tolerance", action="store_true",
                    help="the mixed-precision step at several inner tolerances on the 640 x 320 bubble: "
                         "ms per step against max |theta'| from the FP64 step after 100 steps and at "
                         "t = 1020 s")
    ap.add_argument("--oracle-table", action="store_true",
                    help="the FP64 CPU oracle, single-threaded, on W0 (160 x 80, 100 steps), W1 "
                         "(640 x 320, 100 steps) and W3 (4096 x 2048, 3 steps) from t = 0, beside the "
                         "FP64 GPU step on the same steps")
    ap.add_argument("--dts", type=lambda t: [float(x) for x in t.split(",")], default=[0.05, 0.2, 0.5],
                    help="--learned: time steps of the 4096 x 2048 runs (comma separated)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


def peaks(measure=False):
    """Roofline denominators. HBM: the measured copy bandwidth of the peaks
    file. FP64 and FP32: with measure=True the FMA-chain probe of the library
    (gea_probe_fma) on this GPU, in this run; otherwise the nominal rates,
    152 SMs x (2 FP64 | 128 FP32) FMA lanes x 2 flops x 2.07 GHz."""
    p = {"hbm_gbs": 6800.0, "fp64_tflops": 1.25, "fp32_tflops": 80.5, "src": "fallback",
         "fp64_src": "nominal", "fp32_src": "nominal"}
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p["hbm_gbs"] = float(m["hbm_gbs"])
        p["src"] = "measured"
    except Exception:
        pass
    if measure:
        from paper_2303_10499_gb300 import gea
        f64 = gea.probe_fma(64, iters=16384)
        f32 = gea.probe_fma(32, iters=16384 * 32)
        p["fp64_tflops"], p["fp32_tflops"] = f64["tflops"], f32["tflops"]
        p["fp64_src"] = (f"measured in this run: gea_probe_fma FP64, {f64['blocks']} x 256 threads x 8 "
                         f"FMA chains x {f64['iters']} steps, best of 5 CUDA-event timed launches "
                         f"({f64['ms']:.2f} ms)")
        p["fp32_src"] = (f"measured in this run: gea_probe_fma FP32, {f32['blocks']} x 256 threads x 8 "
                         f"FMA chains x {f32['iters']} steps ({f32['ms']:.2f} ms)")
    return p


def job_rate(local_seconds, units_per_rank, world, device="cuda"):
    """Whole-job throughput of `world` independent replicas: every rank
    processed `units_per_rank` units in its own `local_seconds`; the job took
    the slowest rank's time (max over ranks with an all-reduce on `device`,
    "cuda" for NCCL, "cpu" for gloo), so the rate is world x units / max."""
    t = float(local_seconds)
    if world > 1:
        import torch
        x = torch.tensor([t], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" in r[5 + j]
                          and "Not" not in r[5 + j]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# the CUDA sources each kernel with a recorded DRAM traffic figure is built
# from (profiles/traffic.json keys every figure by the hash of its kernel's
# sources; a change to any of them invalidates that figure alone)
KERNEL_SOURCES = {
    "k_persistent": ("gea_internal.cuh", "gea_tiles_body.cuh", "gea_persistent_body.cuh"),
    "mg_up": ("gea_internal.cuh", "gea_tiles_body.cuh", "gea_tiles.cuh", "gea_kernels.cu"),
    "mom_jacobi": ("gea_internal.cuh", "gea_tiles_body.cuh", "gea_tiles.cuh", "gea_kernels.cu"),
    "g3_": ("gea_internal.cuh", "gea3d.cu"),
}


def kernel_sources(kernel):
    for k, v in KERNEL_SOURCES.items():
        if kernel == k or (k.endswith("_") and kernel.startswith(k)):
            return v
    return None


def kernels_sha256(sources):
    """Hash of a kernel's CUDA sources (any change invalidates the recorded
    counters)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2303_10499_gb300", "csrc")
    for f in sources:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def traffic_for(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/traffic.json), if it was taken on the kernel's current
    CUDA sources (else None)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t.get("per_launch", {}).get(workload, {}).get(kernel)
        src = kernel_sources(kernel)
        if not e or src is None or e.get("sources_sha256") != kernels_sha256(src):
            return None
        return e.get("bytes")
    except Exception:
        return None


def step_model(prof):
    """Algorithmic FP64 words and operations of one step: the per-cell model
    of each phase times the cells its launches covered in the profiled step
    (the same iteration counts as a timed step, up to the state's drift)."""
    words = sum(KERNEL_MODEL.get(k, (0, 0, ""))[0] * v["cells"] for k, v in prof.items())
    flops = sum(KERNEL_MODEL.get(k, (0, 0, ""))[1] * v["cells"] for k, v in prof.items())
    return words * 8.0, flops


def roofline(prof, pk, ms_per_step, persistent, workload):
    total = sum(v["ms"] for v in prof.values())
    share = {k: round(v["ms"] / total, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    step_bytes, step_flops = step_model(prof)
    prec = "f64"
    if persistent:
        # the timed region runs one kernel, the persistent step kernel, once
        # per step: its duration is the event-timed step
        name, launches, per_launch_ms = "k_persistent (whole step)", 1, ms_per_step
        bytes_l, flops_l = step_bytes, step_flops
    else:
        name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
        words, flops, prec = KERNEL_MODEL.get(name, (0, 0, "f64"))
        launches = d["launches"]
        per_launch_ms = d["ms"] / d["launches"]
        cells = d["cells"] / d["launches"]
        bytes_l, flops_l = words * 8 * cells, flops * cells
    t = per_launch_ms * 1e-3
    gbs = bytes_l / t / 1e9
    tfl = flops_l / t / 1e12
    alu = pk["fp64_tflops"] if prec == "f64" else pk["fp32_tflops"]
    if flops_l / (alu * 1e12) >= bytes_l / (pk["hbm_gbs"] * 1e9):
        src = pk["fp64_src"] if prec == "f64" else pk["fp32_src"]
        if src == "nominal":
            src = ("FP64 nominal 1.25 TFLOP/s of GB300 (152 SMs x 2 FP64 FMA lanes x 2 flops x 2.07 GHz)"
                   if prec == "f64" else
                   "FP32 nominal 80.5 TFLOP/s (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)")
        out = {"bound": "alu", "achieved": tfl, "peak": alu, "unit": "TFLOP/s",
               "frac": tfl / alu,
               "peak_source": src + " (the measured peaks file has no entry for this precision)"}
    else:
        out = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": gbs / pk["hbm_gbs"], "peak_source": f"{pk['src']} hbm_gbs"}
    out.update({"kernel": name, "launches_per_step": launches, "avg_launch_ms": per_launch_ms,
                "algorithmic_bytes_per_launch": bytes_l, "algorithmic_flops_per_launch": flops_l,
                "hbm_gbs_achieved": gbs, "fp64_tflops_achieved": tfl,
                "traffic": traffic_for(name.split()[0], workload),
                "phase_share_of_eager_step": share,
                "timing": ("CUDA events around each timed step on the solver stream"
                           if persistent else
                           "CUDA events around each launch of one eager step on the solver stream")})
    return out


def timed_steps(s, stream, flush, steps, warmup, world, local):
    """warmup untimed steps, then `steps` steps each bracketed by CUDA events
    on the solver stream, L2 flushed before each. Returns per-step ms, the
    launches counted by the library and the sampled clocks."""
    import torch
    for _ in range(warmup):
        s.step_async(1)
    s.sync()
    l0 = s.stats()["launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    clk = ClockSampler(local)
    clk.start()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        s.step_async(1)
        e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    s.sync()
    launches = s.stats()["launches"] - l0
    return [e0.elapsed_time(e1) for e0, e1 in evs], launches, clocks


def whole_step(prof, pk, ms_per_step):
    """The whole step against both ceilings: the model's FP64 operations and
    algorithmic bytes of one step (per-phase model x cells of the eager
    profiled step's launches) over the event-timed step."""
    step_bytes, step_flops = step_model(prof)
    t = ms_per_step * 1e-3
    tfl, gbs = step_flops / t / 1e12, step_bytes / t / 1e9
    t_alu = step_flops / (pk["fp64_tflops"] * 1e12)
    t_hbm = step_bytes / (pk["hbm_gbs"] * 1e9)
    return {"flops_per_step": step_flops, "bytes_per_step": step_bytes,
            "fp64_tflops": tfl, "frac_fp64": tfl / pk["fp64_tflops"],
            "hbm_gbs": gbs, "frac_hbm": gbs / pk["hbm_gbs"],
            "bound": "alu" if t_alu >= t_hbm else "hbm",
            "frac_binding": max(t_alu, t_hbm) / t,
            "ms_at_binding_roofline": max(t_alu, t_hbm) * 1e3}


def per_kernel_account(prof, pk):
    """Every kernel of one eager profiled step against its binding roofline:
    model flops (FP64 or FP32) and algorithmic bytes of its launches over
    their summed CUDA-event time, with its share of the step."""
    total = sum(v["ms"] for v in prof.values())
    out = {}
    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        if k not in KERNEL_MODEL or v["ms"] <= 0:
            continue
        words, flops, prec = KERNEL_MODEL[k]
        t = v["ms"] * 1e-3
        tfl = flops * v["cells"] / t / 1e12
        gbs = words * 8 * v["cells"] / t / 1e9
        alu = pk["fp64_tflops"] if prec == "f64" else pk["fp32_tflops"]
        out[k] = {"share": round(v["ms"] / total, 4), "launches": v["launches"],
                  "ms": round(v["ms"], 4), "tflops": round(tfl, 4), "frac_alu": round(tfl / alu, 3),
                  "gbs": round(gbs, 1), "frac_hbm": round(gbs / pk["hbm_gbs"], 3),
                  "avg_cells_per_launch": v["cells"] // max(1, v["launches"])}
    return out


def w3_record(gea, W, stream, flush, pk, local, steps=10, warmup=3):
    """The 4096 x 2048 smooth bubble (larger than L2: the HBM/FP64-roofline
    workload), FP64, CUDA-graph driver: pressure solves to 1e-8 of ||b|| (the
    timing tolerance) and to the parity tolerance 1e-17, each timed like the
    main line, with the whole step's roofline fractions and the dominant
    kernel's."""
    import copy
    import torch
    wl = W.get("bubble4096x2048")
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()}
    out = {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.nz], "cells": wl.grid.cells,
           "dt": wl.const.dt, "driver": None, "runs": {}}
    for rtol in (1e-8, wl.const.cg_rtol):
        const = copy.copy(wl.const)
        const.cg_rtol = rtol
        s = gea.Solver(wl.grid, const, stream=stream)
        s.set_conservative(dev)
        ms, launches, clocks = timed_steps(s, stream, flush, steps, warmup, 1, local)
        st = s.stats()
        prof = s.profile_step()
        mean = statistics.mean(ms)
        out["driver"] = st["driver"]
        out["mg_levels"] = st["mg_levels"]
        out["runs"][f"{rtol:g}"] = {
            "cg_rtol": rtol, "value": wl.grid.cells * steps / (sum(ms) / 1e3), "unit": UNIT,
            "steps": steps, "warmup": warmup, "ms_per_step": mean, "ms_per_step_min": min(ms),
            "pressure_solve_ms_per_step": pressure_ms(s),
            "cg_iters_last_step": st["cg_iters"], "jacobi_sweeps_last_step": [st["jac_u"], st["jac_h"]],
            "gpu_launches": int(launches), "clocks": clocks,
            "whole_step": whole_step(prof, pk, mean),
            "dominant_kernel": roofline(prof, pk, mean, False, wl.name),
            "per_kernel": per_kernel_account(prof, pk),
        }
        s.close()
    del dev
    return out


def pressure_ms(s):
    """Pressure-solve time per step (events around the solves inside the step)."""
    pms = []
    for _ in range(5):
        s.step(1)
        pms.append(s.pressure_ms())
    return statistics.mean(pms)


def matched_error(gea, wl, steps):
    """The mixed-precision step against the FP64 step, both on this GPU from
    the initial state: max |theta'| difference (K) and relative L2 of the
    conservative fields (momenta against the momentum vector) after `steps`
    steps."""
    import numpy as np
    out = []
    for mixed in (False, True):
        s = gea.Solver(wl.grid, wl.const, mixed=mixed)
        s.set_conservative(wl.fields)
        s.step(steps)
        th, _, _ = s.diagnostics(wl.theta_bar)
        out.append((s.get_conservative(), th))
        s.close()
    (c64, th64), (c32, th32) = out
    m = np.hypot(np.linalg.norm(c64["rhou"]), np.linalg.norm(c64["rhow"]))
    rel = {k: float(np.linalg.norm(c32[k] - c64[k]) / np.linalg.norm(c64[k])) for k in ("rho", "rhoe")}
    rel.update({k: float(np.linalg.norm(c32[k] - c64[k]) / m) for k in ("rhou", "rhow")})
    return {"steps": steps, "max_abs_dtheta_K": float(np.abs(th32 - th64).max()),
            "rel_l2": rel, "against": "FP64 GPU step (equal to the FP64 oracle to <= 1e-10 rel. L2)"}


def learned_training_set(W, learned, steps=8, every=2):
    """Pressure systems (the first corrector's r0 and operator, every `every`
    steps of `steps`) of the configurations the learned stage is trained on:
    the 160 x 80 and 640 x 320 bubbles and LES members on 100^2, 200^2 and
    400^2 cells -- none of them the 4096 x 2048 grid it is evaluated on."""
    wls = [W.get("bubble160x80"), W.get("bubble640x320")] + [W.les_member(n) for n in (100, 200, 400)]
    samples = []
    for wl in wls:
        samples += learned.collect(wl, steps, every=every, const=wl.const)
    return samples, [wl.name for wl in wls]


def run_learned(args):
    """The learned pressure stage on the 4096 x 2048 bubble, pressure solves to
    1e-8 of ||b||, for each time step in --dts (the configuration leaves dt
    open; the Helmholtz operator's Laplacian part grows with dt^2, which is
    what gives a learned start something to do). Per dt, timed like the main
    line: plain FP64 MG-CG, the learned initial guess, flexible CG with the
    network stage, the mixed-precision step alone and with the learned
    guess. Two networks: one trained on held-out configurations (the smaller
    bubbles and the LES members, none on this grid) and one trained on the
    first steps of this run itself (in distribution), for reference."""
    import copy
    import numpy as np
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea, learned
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    base = W.get("bubble4096x2048")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def train_net(samples, crop, batch, iters):
        net = gea.Net(8, 1024, 1024, relu=False)
        net.set_params(learned.initial_params(1) * 0.5)
        tr = learned.train(net, samples, iters, n=batch, h=crop, w=crop, lr=2e-3)
        return net, {"samples": len(samples), "iterations": iters, "batch": f"{batch} x {crop} x {crop} crops",
                     "seconds": tr["seconds"], "loss_first": tr["losses"][0],
                     "loss_last20": float(np.mean(tr["losses"][-20:]))}

    t0 = time.perf_counter()
    held_samples, held_names = learned_training_set(W, learned)
    t_collect = time.perf_counter() - t0
    net_held, tr_held = train_net(held_samples, 64, 8, 400)
    tr_held.update({"collect_s": t_collect, "workloads": held_names})
    del held_samples

    def arm(const, mixed, net, mode):
        s = gea.Solver(base.grid, const, stream=stream, graph=True, mixed=mixed)
        s.set_conservative(base.fields)
        if net is not None:
            s.attach_net(net, mode)
        ms, launches, clocks = timed_steps(s, stream, flush, args.steps, args.warmup, world, local)
        its = []
        for _ in range(3):
            s.step(1)
            its.append(s.stats()["cg_iters"])
        pms = pressure_ms(s)
        th, _, _ = s.diagnostics(base.theta_bar)
        n_steps = args.warmup + args.steps + 3 + 5
        s.close()
        return {"value": base.grid.cells * args.steps / (sum(ms) / 1e3), "unit": UNIT,
                "ms_per_step": statistics.mean(ms), "pressure_solve_ms_per_step": pms,
                "cg_iters_per_step": its, "gpu_launches": int(launches), "clocks": clocks,
                "steps_before_theta": n_steps, "_theta": th}

    per_dt = {}
    for dt in args.dts:
        const = copy.copy(base.const)
        const.dt = dt
        const.cg_rtol = 1e-8
        # the in-distribution reference network: trained on this run's own
        # first steps (FP64 solver, parity tolerance) at this dt
        own_const = copy.copy(base.const)
        own_const.dt = dt
        own_const.cg_rtol = 1e-10   # the first corrector's r0 hardly depends on it
        own = learned.collect(base, 8, every=2, const=own_const)
        net_own, tr_own = train_net(own, 256, 8, 400)
        del own
        arms = {
            "plain_fp64": arm(const, False, None, 0),
            "learned_guess_fp64": arm(const, False, net_held, 1),
            "network_fcg_fp64": arm(const, False, net_held, 2),
            "mixed": arm(const, True, None, 0),
            "mixed_learned_guess": arm(const, True, net_held, 1),
            "learned_guess_fp64_own_net": arm(const, False, net_own, 1),
            "mixed_learned_guess_own_net": arm(const, True, net_own, 1),
        }
        net_own.close()
        th0 = arms["plain_fp64"]["_theta"]
        v0 = arms["plain_fp64"]["value"]
        for k, a in arms.items():
            a["max_abs_dtheta_K_vs_plain_fp64"] = float(np.abs(a["_theta"] - th0).max())
            a["speedup_vs_plain_fp64"] = a["value"] / v0
        for a in arms.values():
            a.pop("_theta")
        ratio = 2 * dt * dt * base.const.R * 300.0 * (1 / base.grid.dx ** 2 + 1 / base.grid.dz ** 2)
        per_dt[f"{dt:g}"] = {"dt": dt, "laplacian_to_diagonal_ratio": ratio, "arms": arms,
                             "own_net_training": tr_own}
    best = max(((d, k, a) for d, v in per_dt.items() for k, a in v["arms"].items()
                if "learned" in k or "fcg" in k), key=lambda t: t[2]["speedup_vs_plain_fp64"])
    first = per_dt[f"{args.dts[0]:g}"]["arms"]
    res = {
        "metric": METRIC, "value": first["mixed_learned_guess"]["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": first["mixed_learned_guess"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16",
        "data": "synthetic",
        "config": {"workload": base.name + " learned pressure stage", "grid": [base.grid.nx, base.grid.nz],
                   "dts": list(args.dts), "cg_rtol": 1e-8, "value_arm": f"mixed_learned_guess at dt {args.dts[0]:g}",
                   "network": "4-level U-Net, 16 base channels, linear, "
                   f"{gea.net_param_count()} parameters, bfloat16 tensor-core layers",
                   "l2": "flushed between timed steps (256 MB write, untimed)"},
        "per_dt": per_dt,
        "held_out_training": tr_held,
        "best_learned_arm": {"dt": best[0], "arm": best[1], "speedup_vs_plain_fp64": best[2]["speedup_vs_plain_fp64"],
                             "max_abs_dtheta_K_vs_plain_fp64": best[2]["max_abs_dtheta_K_vs_plain_fp64"]},
    }
    net_held.close()
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_ensemble(args):
    """The LES ensemble: one cooperative launch per step for all members
    against one launch per member per step, same states, same step counts;
    then the same members in mixed precision, in one launch."""
    import numpy as np
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import ensemble as ensemble_tuner
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    wls = W.les_ensemble(args.ensemble, seed=0)
    cells = sum(wl.grid.cells for wl in wls)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(step_all, reset):
        reset()
        for _ in range(args.warmup):
            step_all()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        clk = ClockSampler(local)
        clk.start()
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            step_all()
            e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        return [e0.elapsed_time(e1) for e0, e1 in evs], clocks

    solvers = [gea.Solver(wl.grid, wl.const, stream=stream) for wl in wls]

    def reset():
        for sv, wl in zip(solvers, wls):
            sv.set_conservative(wl.fields)

    # one launch per member per step (each member's own driver)
    ms_seq, _ = timed(lambda: [sv.step_async(1) for sv in solvers], reset)
    for sv in solvers:
        sv.sync()
    # block partition: tiles only, then the autotuner's choice
    E0 = gea.Ensemble(solvers, stream=stream)
    ms_tiles, _ = timed(lambda: E0.step_async(1), reset)
    E0.sync()
    E0.close()
    reset()
    E, tune = ensemble_tuner.autotune(solvers, stream=stream)
    ms_ens, clocks = timed(lambda: E.step_async(1), reset)
    E.sync()
    iters = [sv.stats()["cg_iters"] for sv in solvers[:3]]
    nb = E.blocks()
    E.close()
    # the mixed-precision members (FP64 state, FP32 inner solves) in one
    # launch, with the tuned shape, against the FP64 ensemble: time per step
    # and max |theta'| difference after the same steps from the same states
    shape = [k for k, v in gea.TILE_SHAPES.items() if v == tune["tile_shape"]][0]
    mixed = [gea.Solver(wl.grid, wl.const, stream=stream, mixed=True) for wl in wls]
    for sv in mixed:
        sv.set_tile_shape(shape)

    def reset_mixed():
        for sv, wl in zip(mixed, wls):
            sv.set_conservative(wl.fields)

    # the tuned partition's work weights, from the FP64 members' iterations
    tiles_m, its_m = ensemble_tuner.member_work(solvers, shape)
    w_mix = tiles_m * (1.0 + its_m) ** float(tune["beta"])
    EM = gea.Ensemble(mixed, stream=stream, weights=w_mix)
    ms_mix, clocks_mix = timed(lambda: EM.step_async(1), reset_mixed)
    EM.sync()
    EM.close()
    n_check = 20
    reset()
    reset_mixed()
    E1 = gea.Ensemble(solvers, stream=stream)
    E1.step(n_check)
    E1.close()
    EM = gea.Ensemble(mixed, stream=stream, weights=w_mix)
    EM.step(n_check)
    EM.close()
    dth = max(float(np.abs(m.diagnostics(wl.theta_bar)[0] - f.diagnostics(wl.theta_bar)[0]).max())
              for m, f, wl in zip(mixed, solvers, wls))
    value = cells * args.steps / (sum(ms_ens) / 1e3)
    seq = cells * args.steps / (sum(ms_seq) / 1e3)
    sizes = sorted({wl.grid.nx for wl in wls})
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms_ens), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"LES ensemble of {len(wls)} non-smooth bubbles", "grids": sizes,
                   "cells_per_step": cells, "cs": wls[0].const.cs, "mu": wls[0].const.mu,
                   "dt": wls[0].const.dt, "l2": "flushed between timed steps (256 MB write, untimed)",
                   "blocks_per_member": {str(n): sorted({b for b, wl in zip(nb, wls) if wl.grid.nx == n})
                                         for n in sizes}},
        "one_launch_per_member": {"value": seq, "unit": UNIT, "ms_per_step": statistics.mean(ms_seq)},
        "ensemble_blocks_by_tiles": {"value": cells * args.steps / (sum(ms_tiles) / 1e3), "unit": UNIT,
                                     "ms_per_step": statistics.mean(ms_tiles)},
        "autotune": tune if not isinstance(tune, dict) else {k: v for k, v in tune.items() if k != "blocks"},
        "tile_shape": {"chosen": tune["tile_shape"],
                       "note": "one block shape per cooperative launch, so one shape for all members",
                       "best_ms_32x8": min(tune["ms_per_step_by_shape_and_beta"]["32x8"].values()),
                       "best_ms_chosen": min(tune["ms_per_step_by_shape_and_beta"][tune["tile_shape"]].values()),
                       "gain_vs_32x8": min(tune["ms_per_step_by_shape_and_beta"]["32x8"].values()) /
                       min(tune["ms_per_step_by_shape_and_beta"][tune["tile_shape"]].values())},
        "speedup_vs_one_launch_per_member": value / seq,
        "mixed_precision_ensemble": {
            "value": cells * args.steps / (sum(ms_mix) / 1e3), "unit": UNIT,
            "ms_per_step": statistics.mean(ms_mix), "speedup_vs_fp64_ensemble": statistics.mean(ms_ens) /
            statistics.mean(ms_mix), "tile_shape": tune["tile_shape"], "clocks": clocks_mix,
            "max_abs_dtheta_K_vs_fp64_ensemble": dth, "steps_compared": n_check},
        "cg_iters_last_step_first_members": iters,
        "gpu_launches": 1, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(res), flush=True)


# Per-cell model of the three-dimensional kernels (same conventions as
# KERNEL_MODEL; coarsening and restriction per coarse cell).
KERNEL_MODEL_3D = {
    "g3_les": (5, 60, "f64"),
    "g3_mx_r0mom": (31.5, 87, "f64"),
    "g3_mx_mom": (11.5, 93, "f32"),
    "g3_mx_u1": (7.5, 3, "f64"),
    "g3_mx_r0h": (16.5, 31, "f64"),
    "g3_mx_enth": (8.5, 31, "f32"),
    "g3_mx_h1": (2.5, 1, "f64"),
    "g3_mx_pupd": (1.5, 2, "f32"),
    "g3_mx_spmv": (3, 15, "f32"),
    "g3_mx_update": (3, 6, "f32"),
    "g3_mx_papply": (2.5, 1, "f64"),
    "g3_pred": (31, 102, "f64"),
    "g3_mom": (23, 93, "f64"),
    "g3_kin": (4, 6, "f64"),
    "g3_enth_rhs": (15, 45, "f64"),
    "g3_enth": (17, 31, "f64"),
    "g3_eos": (9, 7, "f64"),
    "g3_faces": (8, 15, "f64"),
    "g3_diag": (6, 7, "f64"),
    "g3_coarsen": (38, 32, "f64"),
    "g3_H": (24, 87, "f64"),
    "g3_helm_rhs": (18, 70, "f64"),
    "g3_mg_down": (49, 137, "f64"),
    "g3_mg_coarse": (7, 17, "f64"),
    "g3_mg_up": (7.125, 20, "f64"),
    "g3_mg_single": (6, 20, "f64"),
    "g3_pupd": (3, 2, "f64"),
    "g3_spmv": (6, 15, "f64"),
    "g3_update": (6, 6, "f64"),
    "g3_correct": (20, 61, "f64"),
}


def run_3d(args):
    """The three-dimensional step (include/gea3d.h) on a 3D workload, timed
    like the main line; roofline of its dominant kernel from one eager
    step; end to end through the C ABI with pinned host buffers."""
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    wl = W.get(args.three_d)
    g = wl.grid
    cells = g.cells
    stream = torch.cuda.current_stream()
    s = gea.Solver3D(g, wl.const, stream=stream)
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()}
    s.set_conservative(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ms, launches, clocks = timed_steps(s, stream, flush, args.steps, args.warmup, world, local)
    st = s.stats()
    value, _ = job_rate(sum(ms) / 1e3, cells * args.steps, world)
    prof = s.profile_step()
    KERNEL_MODEL.update(KERNEL_MODEL_3D)
    roof = roofline(prof, peaks(measure=True), statistics.mean(ms), False, wl.name)

    host = s.get_state()
    pin_in = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in wl.fields.items()}
    out = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory().numpy() for k, v in host.items()}
    bi = sum(v.nbytes for v in pin_in.values())
    bo = sum(v.nbytes for v in out.values())
    ne = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ne):
        s.set_conservative(pin_in)
        s.step(1)
        s.get_state(out)
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * cells * ne / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": bo,
           "path": "gea3d_set_conservative(host) + gea3d_step(1) + gea3d_get_state(host)"}
    s.close()
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "grid": [g.nx, g.ny, g.nz], "cells": cells,
                   "domain_m": [g.lx, g.ly, g.lz], "dt": wl.const.dt, "n_corr": wl.const.n_corr,
                   "jac_rtol": wl.const.jac_rtol, "cg_rtol": wl.const.cg_rtol, "cs": wl.const.cs,
                   "mg_levels": st["mg_levels"],
                   "l2": "inputs larger than L2 (each field 0.5 GB) and 256 MB flush between steps",
                   "driver": "graph", "parallelism": f"replicas x{world}"},
        "cg_iters_last_step": st["cg_iters"], "jacobi_sweeps_last_step": [st["jac_u"], st["jac_h"]],
        "ms_per_step_min": min(ms), "ms_per_step_median": statistics.median(ms),
        "gpu_launches": int(launches) * world, "clocks": clocks, "e2e": e2e, "roofline": roof,
    }
    # the mixed-precision 3D step timed the same way, and its difference from
    # the FP64 GPU step (equal to the 3D oracle to <= 1e-10) after 20 steps
    sm = gea.Solver3D(g, wl.const, stream=stream, mixed=True)
    sm.set_conservative(dev)
    ms_m, launches_m, clocks_m = timed_steps(sm, stream, flush, args.steps, args.warmup, world, local)
    st_m = sm.stats()
    value_m, _ = job_rate(sum(ms_m) / 1e3, cells * args.steps, world)
    res["mixed_precision"] = {
        "value": value_m, "unit": UNIT, "ms_per_step": statistics.mean(ms_m), "speedup_vs_fp64": value_m / value,
        "cg_iters_last_step": st_m["cg_iters"], "jacobi_sweeps_last_step": [st_m["jac_u"], st_m["jac_h"]],
        "gpu_launches": int(launches_m) * world, "clocks": clocks_m, "driver": st_m["driver"],
        "error_vs_fp64": matched_error3(gea, wl, dev, stream, 20) if rank == 0 else None,
    }
    sm.close()
    if rank == 0 and world == 1:
        # at matched error: inner tolerance 1e-3, against the FP64 step over
        # the configuration's 200 steps (bar: max |theta'| <= 1e-3 K)
        rt = 1e-3
        sq = gea.Solver3D(g, wl.const, stream=stream, mixed=True, mp_rtol=rt)
        sq.set_conservative(dev)
        ms_q, _, clocks_q = timed_steps(sq, stream, flush, args.steps, args.warmup, world, local)
        its_q = sq.stats()["cg_iters"]
        sq.close()
        err_q = matched_error3(gea, wl, dev, stream, wl.steps, mp_rtol=rt)
        res["mixed_precision_matched_error"] = {
            "mp_rtol": rt, "ms_per_step": statistics.mean(ms_q),
            "speedup_vs_fp64": statistics.mean(ms) / statistics.mean(ms_q), "cg_iters_last_step": its_q,
            "clocks": clocks_q, "error_vs_fp64": err_q, "bar_K": 1e-3,
            "within_bar": bool(err_q["max_abs_dtheta_K"] <= 1e-3)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline3(args.cpu_seconds)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


def matched_error3(gea, wl, dev, stream, steps, mp_rtol=0.0):
    """The mixed 3D step (inner tolerance mp_rtol; 0: the library default)
    against the FP64 3D step, both on this GPU from the initial state: max
    |theta'| difference (K) and relative L2 per field (velocities against
    the velocity vector's norm) after `steps` steps."""
    import numpy as np
    out = []
    for mixed in (False, True):
        s = gea.Solver3D(wl.grid, wl.const, stream=stream, mixed=mixed, mp_rtol=mp_rtol if mixed else 0.0)
        s.set_conservative(dev)
        s.step(steps)
        out.append((s.get_state(), s.diagnostics(wl.theta_bar)[0]))
        s.close()
    (a, tha), (b, thb) = out
    vel = np.sqrt(sum(np.linalg.norm(a[k]) ** 2 for k in ("u", "v", "w")))
    rel = {k: float(np.linalg.norm(b[k] - a[k]) / np.linalg.norm(a[k])) for k in ("rho", "T", "p", "pp")}
    rel.update({k: float(np.linalg.norm(b[k] - a[k]) / vel) for k in ("u", "v", "w")})
    return {"steps": steps, "max_abs_dtheta_K": float(np.abs(thb - tha).max()), "rel_l2": rel,
            "against": "FP64 GPU 3D step (equal to the 3D oracle to <= 1e-10 rel. L2)"}


def cpu_baseline3(seconds):
    """The FP64 3D CPU oracle as it stands, single-threaded, on a bounded
    sample: the same bubble on a 64x64x32 grid, consecutive steps from t = 0
    (per cell-step the work is that of the full grid's step up to the
    solvers' iteration counts)."""
    from paper_2303_10499_gb300 import workloads as W
    from oracle import oracle3d
    wl = W.get("bubble3d_64x64x32")
    q = oracle3d.Oracle3D(wl.grid, wl.const)
    st = q.derive(wl.fields)
    t0 = time.perf_counter()
    q.step(st, 1)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(seconds / max(t1, 1e-6)) - 1))
    t0 = time.perf_counter()
    q.step(st, n)
    dt = time.perf_counter() - t0
    return {"value": wl.grid.cells * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"steps 2..{n + 1} of {wl.name} from t=0 ({n} steps, {dt:.1f} s)"}


def run_ours(args):
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        torch.distributed.barrier()
    wl = W.get(args.workload)
    cells = wl.grid.cells
    stream = torch.cuda.current_stream()
    s = gea.Solver(wl.grid, wl.const, stream=stream, graph=args.graph, mixed=args.mixed)
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()}
    s.set_conservative(dev)
    tuned = None
    if args.tune_tiles and s.stats()["driver"] != "persistent":
        tuned = s.tune_tiles()
        s.set_conservative(dev)   # time from the initial state again
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ms, launches, clocks = timed_steps(s, stream, flush, args.steps, args.warmup, world, local)
    st = s.stats()
    value, _ = job_rate(sum(ms) / 1e3, cells * args.steps, world)

    pms = pressure_ms(s)
    prof = s.profile_step()
    pk = peaks(measure=True)
    roof = roofline(prof, pk, statistics.mean(ms), st["driver"] == "persistent", wl.name)
    roof["whole_step"] = whole_step(prof, pk, statistics.mean(ms))

    # end to end through the C ABI with host buffers: H2D of the full state,
    # one step, D2H of the full state, every step
    nx, nz = wl.grid.nx, wl.grid.nz
    host = s.get_full()
    pin = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    out = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory().numpy() for k, v in host.items()}
    nbytes = sum(v.nbytes for v in pin.values())
    ne = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ne):
        s.set_full(pin)
        s.step(1)
        s.get_full(out)
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * cells * ne / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes,
           "path": "gea_set_state(FULL, host) + gea_step(1) + gea_get_state(FULL, host)"}
    s.close()

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.mixed else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": [nx, nz], "cells": cells,
                   "domain_m": [wl.grid.lx, wl.grid.lz], "dt": wl.const.dt,
                   "n_corr": wl.const.n_corr, "jac_rtol": wl.const.jac_rtol,
                   "cg_rtol": wl.const.cg_rtol, "mg_levels": st["mg_levels"],
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "driver": st["driver"],
                   "tiles_per_block": tuned if tuned else "size rule (4 on grids of >= 16384 tiles, else 1)",
                   "parallelism": f"replicas x{world}"},
        "pressure_solve_ms_per_step": pms,
        "cg_iters_last_step": st["cg_iters"], "jacobi_sweeps_last_step": [st["jac_u"], st["jac_h"]],
        "ms_per_step_min": min(ms), "ms_per_step_median": statistics.median(ms),
        "gpu_launches": int(launches) * world, "clocks": clocks, "e2e": e2e, "roofline": roof,
    }
    if not args.mixed:
        # the mixed-precision step timed the same way, with its error against
        # the FP64 step at 100 steps
        sm = gea.Solver(wl.grid, wl.const, stream=stream, mixed=True)
        sm.set_conservative(dev)
        ms_m, launches_m, clocks_m = timed_steps(sm, stream, flush, args.steps, args.warmup, world,
                                                 local)
        st_m = sm.stats()
        value_m, _ = job_rate(sum(ms_m) / 1e3, cells * args.steps, world)
        pms_m = pressure_ms(sm)
        sm.close()
        res["mixed_precision"] = {
            "value": value_m, "unit": UNIT, "ms_per_step": statistics.mean(ms_m),
            "pressure_solve_ms_per_step": pms_m, "speedup_vs_fp64": value_m / value,
            "pressure_speedup_vs_fp64": pms / pms_m if pms_m > 0 else None,
            "cg_iters_last_step": st_m["cg_iters"],
            "jacobi_sweeps_last_step": [st_m["jac_u"], st_m["jac_h"]],
            "gpu_launches": int(launches_m) * world, "clocks": clocks_m, "driver": st_m["driver"],
            "error_vs_fp64": matched_error(gea, wl, 100) if rank == 0 else None,
        }
    if rank == 0 and world == 1 and not args.mixed and wl.name == "smooth_bubble_640x320":
        # the mixed step at matched error: inner tolerance 1e-3, timed the same
        # way, with its max |theta'| distance from the FP64 run over the
        # configuration's whole horizon (t = 1020 s); the bar is 1e-3 K
        import numpy as np
        rt = 1e-3
        sq = gea.Solver(wl.grid, wl.const, stream=stream, mixed=True, mp_rtol=rt)
        sq.set_conservative(dev)
        ms_q, _, clocks_q = timed_steps(sq, stream, flush, args.steps, args.warmup, world, local)
        its_q = sq.stats()["cg_iters"]
        sq.close()
        nfull = int(round(1020.0 / wl.const.dt))
        th64, _ = theta_after(gea, wl, stream, False, 0.0, nfull)
        thq, stq = theta_after(gea, wl, stream, True, rt, nfull)
        err = float(np.abs(thq - th64).max())
        res["mixed_precision_matched_error"] = {
            "mp_rtol": rt, "value": cells * args.steps / (sum(ms_q) / 1e3), "unit": UNIT,
            "ms_per_step": statistics.mean(ms_q), "speedup_vs_fp64": statistics.mean(ms) / statistics.mean(ms_q),
            "cg_iters_last_step": its_q, "clocks": clocks_q,
            "max_abs_dtheta_K_vs_fp64_t1020": err, "bar_K": 1e-3, "within_bar": bool(err <= 1e-3 and stq == 0),
            "steps_compared": nfull}
    if rank == 0 and not args.no_w3 and wl.name != "bubble4096x2048":
        res["w3"] = w3_record(gea, W, stream, flush, pk, local)
    res["peaks"] = {k: v for k, v in pk.items()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds, args.workload)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


SWEEP_SIZES = [(256, 128), (512, 256), (640, 320), (1024, 512), (2048, 1024), (4096, 2048), (8192, 4096)]


def run_sweep(args):
    """Throughput against grid size: the smooth bubble (20 km x 10 km,
    dt = 0.05 s) from 256 x 128 to 8192 x 4096 cells, FP64, pressure solves
    to 1e-8 of ||b||, the library's own choice of driver (the persistent
    kernel while a grid's tiles fit the co-resident blocks a few times, the
    CUDA graph above). Each size is timed like the main line (L2 flushed
    before every timed step) and its whole step is set against the FP64 and
    HBM ceilings on the flop and byte model of one profiled step. The
    working set moves from L2 (129 MB) into HBM between 640 x 320 and
    2048 x 1024."""
    import copy
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    pk = peaks(measure=True)
    rows = []
    for nx, nz in SWEEP_SIZES:
        wl = W.smooth_bubble_20km(nx, nz, dt=0.05)
        const = copy.copy(wl.const)
        const.cg_rtol = 1e-8
        s = gea.Solver(wl.grid, const, stream=stream)
        s.set_conservative({k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()})
        ms, launches, clocks = timed_steps(s, stream, flush, args.steps, args.warmup, 1, local)
        st = s.stats()
        prof = s.profile_step()
        mean = statistics.mean(ms)
        ws = whole_step(prof, pk, mean)
        rows.append({"grid": [nx, nz], "cells": wl.grid.cells, "driver": st["driver"],
                     "mg_levels": st["mg_levels"], "ms_per_step": mean, "ms_per_step_min": min(ms),
                     "value": wl.grid.cells * args.steps / (sum(ms) / 1e3), "unit": UNIT,
                     "cg_iters_last_step": st["cg_iters"],
                     "jacobi_sweeps_last_step": [st["jac_u"], st["jac_h"]],
                     "gpu_launches": int(launches), "clocks": clocks,
                     "bytes_per_step": ws["bytes_per_step"], "hbm_gbs": ws["hbm_gbs"],
                     "frac_hbm": ws["frac_hbm"], "fp64_tflops": ws["fp64_tflops"],
                     "frac_fp64": ws["frac_fp64"], "bound": ws["bound"],
                     "frac_binding": ws["frac_binding"]})
        s.close()
        torch.cuda.empty_cache()
    top = rows[-1]
    res = {"metric": METRIC, "value": top["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": top["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "smooth_bubble size sweep", "dt": 0.05, "cg_rtol": 1e-8,
                      "value_at": f"{top['grid'][0]}x{top['grid'][1]}",
                      "l2": "flushed between timed steps (256 MB write, untimed)"},
           "sweep": rows, "peaks": pk}
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_full(args):
    """The 640 x 320 smooth bubble run to t = 1020 s (20,400 steps of
    0.05 s) by the FP64 step and by the mixed-precision step, each from the
    initial state, timed over the whole run (CUDA events around chunks of
    steps, no L2 flush: this is a production run); then the mixed run's
    per-field error against the FP64 run at t = 1020 s: max |theta'|
    difference (K), relative L2 of rho and rho e, of rho u and rho w
    against the momentum vector. The FP64 step itself equals the FP64 oracle
    to <= 1e-10 relative L2 over the first 100 steps (the parity tests); a
    20,400-step oracle run would take about 50 minutes of one host core."""
    import numpy as np
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    wl = W.get("bubble640x320")
    t_end, chunk = 1020.0, 1000
    nsteps = int(round(t_end / wl.const.dt))
    stream = torch.cuda.current_stream()
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()}
    arms = {}
    for mixed in (False, True):
        s = gea.Solver(wl.grid, wl.const, stream=stream, mixed=mixed)
        s.set_conservative(dev)
        clk = ClockSampler(local)
        clk.start()
        ms, done, iters = 0.0, 0, []
        while done < nsteps:
            n = min(chunk, nsteps - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step_async(n)
            e1.record(stream)
            s.sync()
            ms += e0.elapsed_time(e1)
            done += n
            iters.append(s.stats()["cg_iters"])
        clocks = clk.stop()
        st = s.stats()
        th, _, _ = s.diagnostics(wl.theta_bar)
        arms["mixed" if mixed else "fp64"] = {
            "steps": done, "t_end_s": done * wl.const.dt, "seconds": ms / 1e3,
            "ms_per_step": ms / done, "value": wl.grid.cells * done / (ms / 1e3), "unit": UNIT,
            "driver": st["driver"], "status": st["status"], "cg_iters_every_1000_steps": iters,
            "theta_prime_K": {"min": float(th.min()), "max": float(th.max())}, "clocks": clocks,
            "_cons": s.get_conservative(), "_theta": th}
        s.close()
    a64, a32 = arms["fp64"], arms["mixed"]
    c64, c32 = a64.pop("_cons"), a32.pop("_cons")
    th64, th32 = a64.pop("_theta"), a32.pop("_theta")
    m = np.hypot(np.linalg.norm(c64["rhou"]), np.linalg.norm(c64["rhow"]))
    rel = {k: float(np.linalg.norm(c32[k] - c64[k]) / np.linalg.norm(c64[k])) for k in ("rho", "rhoe")}
    rel.update({k: float(np.linalg.norm(c32[k] - c64[k]) / m) for k in ("rhou", "rhow")})
    res = {"metric": METRIC, "value": a32["value"], "unit": UNIT, "n_gpus": 1, "steps": nsteps,
           "warmup": 0, "ms_per_step": a32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": wl.name + " to t = 1020 s", "grid": [wl.grid.nx, wl.grid.nz],
                      "dt": wl.const.dt, "cg_rtol": wl.const.cg_rtol, "value_arm": "mixed",
                      "l2": "not flushed (whole-run timing, steps in chunks of 1000)"},
           "fp64": a64, "mixed": a32, "speedup_vs_fp64": a32["value"] / a64["value"],
           "error_vs_fp64_at_t_end": {"max_abs_dtheta_K": float(np.abs(th32 - th64).max()),
                                      "rel_l2": rel}}
    if rank == 0:
        print(json.dumps(res), flush=True)


def theta_after(gea, wl, stream, mixed, rtol, n):
    """theta' (device diagnostics) and status after n steps of the FP64 or
    mixed step (inner tolerance rtol; 0: the library default) from the
    workload's initial state."""
    s = gea.Solver(wl.grid, wl.const, stream=stream, mixed=mixed, mp_rtol=rtol)
    s.set_conservative(wl.fields)
    done = 0
    while done < n:
        k = min(2000, n - done)
        s.step(k)
        done += k
    st = s.stats()["status"]
    th, _, _ = s.diagnostics(wl.theta_bar)
    s.close()
    return th, st


def run_mixed_tolerance(args):
    """Speed against accuracy of the mixed-precision step on the 640 x 320
    bubble: for each inner tolerance mp_rtol of its FP32 solves, the step
    timed like the main line (L2 flushed between timed steps) and its
    max |theta'| distance from the FP64 step after 100 steps and at
    t = 1020 s (20,400 steps, both runs from the initial state). The FP64
    step is timed the same way; speedup = FP64 ms / mixed ms."""
    import numpy as np
    import torch
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    B.build()
    wl = W.get("bubble640x320")
    nfull = int(round(1020.0 / wl.const.dt))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(mixed, rtol):
        s = gea.Solver(wl.grid, wl.const, stream=stream, mixed=mixed, mp_rtol=rtol)
        s.set_conservative(wl.fields)
        ms, _, clocks = timed_steps(s, stream, flush, args.steps, args.warmup, 1, local)
        its = s.stats()["cg_iters"]
        s.close()
        return statistics.mean(ms), its, clocks

    ref100, _ = theta_after(gea, wl, stream, False, 0.0, 100)
    reffull, _ = theta_after(gea, wl, stream, False, 0.0, nfull)
    ms64, its64, _ = timed(False, 0.0)
    rows = []
    for rtol in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2):
        ms, its, clocks = timed(True, rtol)
        t100, st100 = theta_after(gea, wl, stream, True, rtol, 100)
        tfull, stfull = theta_after(gea, wl, stream, True, rtol, nfull)
        rows.append({"mp_rtol": rtol, "ms_per_step": ms, "speedup_vs_fp64": ms64 / ms,
                     "cg_iters_last_step": its, "clocks": clocks,
                     "max_abs_dtheta_K_100_steps": float(np.abs(t100 - ref100).max()),
                     "max_abs_dtheta_K_t1020": float(np.abs(tfull - reffull).max()),
                     "status": [st100, stfull]})
    ok = [r for r in rows if r["max_abs_dtheta_K_t1020"] <= 1e-3 and r["status"] == [0, 0]]
    best = max(ok, key=lambda r: r["speedup_vs_fp64"]) if ok else None
    res = {"metric": METRIC, "value": wl.grid.cells / (best["ms_per_step"] / 1e3) if best else None,
           "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": best["ms_per_step"] if best else None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": wl.name + " mixed-precision inner tolerance sweep",
                      "value_arm": "fastest mp_rtol with max |dtheta'| <= 1e-3 K at t = 1020 s",
                      "l2": "flushed between timed steps (256 MB write, untimed)"},
           "fp64": {"ms_per_step": ms64, "cg_iters_last_step": its64}, "sweep": rows,
           "best": best}
    print(json.dumps(res), flush=True)


def run_oracle_table(args):
    """The oracle timings of the measurement plan: the FP64 CPU oracle as it
    stands, single-threaded, on W0 (the 160 x 80 bubble, 100 steps), W1 (640
    x 320, 100 steps) and W3 (4096 x 2048, 3 steps), every run from t = 0,
    and the FP64 GPU step on the same steps from the same state (CUDA events
    around the whole run on the solver stream, no L2 flush), with the
    largest relative L2 difference of the state fields between the two at
    the end."""
    import numpy as np
    import torch
    import oracle
    from paper_2303_10499_gb300 import build as B
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W

    world, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    B.build()
    oracle.build_oracle()
    stream = torch.cuda.current_stream()
    rows = []
    for name, n in (("bubble160x80", 100), ("bubble640x320", 100), ("bubble4096x2048", 3)):
        wl = W.get(name)
        o = oracle.Oracle(wl.grid, wl.const)
        so = o.derive(wl.fields)
        t0 = time.perf_counter()
        o.step(so, n)
        t_cpu = time.perf_counter() - t0
        s = gea.Solver(wl.grid, wl.const, stream=stream)
        s.set_conservative(wl.fields)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step_async(n)
        e1.record(stream)
        s.sync()
        t_gpu = e0.elapsed_time(e1) / 1e3
        g = s.get_full()
        st = s.stats()
        s.close()
        diff = max(float(np.linalg.norm(g[k] - so[k]) / np.linalg.norm(so[k])) for k in ("rho", "T", "pp"))
        rows.append({"workload": name, "grid": [wl.grid.nx, wl.grid.nz], "steps": n,
                     "oracle": {"seconds": t_cpu, "value": wl.grid.cells * n / t_cpu, "unit": UNIT,
                                "cores": 1, "kind": "oracle"},
                     "gpu_fp64": {"seconds": t_gpu, "value": wl.grid.cells * n / t_gpu, "unit": UNIT,
                                  "driver": st["driver"]},
                     "gpu_over_oracle": t_cpu / t_gpu,
                     "max_rel_l2_rho_T_pp_gpu_vs_oracle": diff})
    w1 = rows[1]
    res = {"metric": METRIC, "value": w1["gpu_fp64"]["value"], "unit": UNIT, "n_gpus": 1,
           "steps": w1["steps"], "warmup": 0, "ms_per_step": w1["gpu_fp64"]["seconds"] * 1e3 / w1["steps"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "oracle table W0, W1, W3 from t = 0", "value_at": "bubble640x320",
                      "l2": "not flushed (whole-run timing)"},
           "oracle_table": rows}
    print(json.dumps(res), flush=True)


def _oracle_replica(job):
    """One host process of the all-cores baseline: `n` oracle steps of the
    named workload after one untimed step; returns (cell-steps, seconds)."""
    name, n = job
    import oracle
    from paper_2303_10499_gb300 import workloads as W
    wl = W.get(name)
    o = oracle.Oracle(wl.grid, wl.const)
    st = o.derive(wl.fields)
    o.step(st, 1)
    t0 = time.perf_counter()
    o.step(st, n)
    return wl.grid.cells * n, time.perf_counter() - t0


def cpu_baseline(wl, seconds, name=None):
    """The FP64 CPU oracle as it stands, single-threaded, on a bounded sample
    of the same workload (consecutive steps from t = 0); with `name` (the
    workload's key) also on every host core at once: one independent oracle
    process per core (spawned: this process holds a CUDA context), each on
    the same sample, aggregate cell-steps over the slowest process's time."""
    import oracle
    o = oracle.Oracle(wl.grid, wl.const)
    st = o.derive(wl.fields)
    t0 = time.perf_counter()
    o.step(st, 1)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(seconds / max(t1, 1e-6)) - 1))
    t0 = time.perf_counter()
    o.step(st, n)
    dt = time.perf_counter() - t0
    out = {"value": wl.grid.cells * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"steps 2..{n + 1} of {wl.name} from t=0 ({n} steps, {dt:.1f} s)"}
    if name is not None:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        cores = os.cpu_count() or 1
        nr = max(1, int(n * 0.7))
        try:
            with ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
                res = list(ex.map(_oracle_replica, [(name, nr)] * cores, timeout=600))
            work = sum(r[0] for r in res)
            slowest = max(r[1] for r in res)
            out["all_cores"] = {"value": work / slowest, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{cores} processes, each steps 2..{nr + 1} of {wl.name} from t=0 "
                                          f"(slowest {slowest:.1f} s)"}
        except Exception as e:   # the single-core figure stands on its own
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2303_10499_gb300 import workloads as W
    import oracle
    wl = W.get(args.workload)
    o = oracle.Oracle(wl.grid, wl.const)
    st = o.derive(wl.fields)
    for _ in range(args.warmup):
        o.step(st, 1)
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.step(st, 1)
        ms.append((time.perf_counter() - t0) * 1e3)
    value = wl.grid.cells * args.steps / (sum(ms) / 1e3)
    res = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.nz], "cells": wl.grid.cells,
                   "dt": wl.const.dt, "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} consecutive steps of {wl.name} after "
                                   f"{args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.learned:
        run_learned(args)
    elif args.ensemble:
        run_ensemble(args)
    elif args.three_d:
        run_3d(args)
    elif args.sweep:
        run_sweep(args)
    elif args.full_run:
        run_full(args)
    elif args.oracle_table:
        run_oracle_table(args)
    elif args.mixed_tolerance:
        run_mixed_tolerance(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
