"""Write the round-off floor of one oracle step on the 4096 x 2048 bubble.

The oracle advances the smooth bubble on 4096 x 2048 cells by one step
three times: as it stands; with its reductions (residual norms, CG dot
products) in reverse index order; and from the initial conservative fields
with every value moved by one unit in the last place, up or down at random
(seed 0), which stands for an evaluation that rounds each cell's values
differently -- as any other correct FP64 program does, through fused
multiply-adds and another order of operations. The near-hydrostatic state
amplifies such rounding (p' ~ 1e5 Pa, velocities ~3e-3 m/s after one step).
The difference of each variant from the plain run per field -- relative L2,
with momenta and face fluxes measured against the norm of their vector, as
the GPU parity test does -- is written to roundoff_floor_bubble4096x2048.txt.
The GPU parity test of this workload takes its bar from this file.

Calls only oracle/ (and the seeded input generator). Run from the repository
root: python tests/golden/make_roundoff_floor.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2303_10499_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "roundoff_floor_bubble4096x2048.txt")


def run(wl, reverse, fields=None):
    oracle.set_reverse_sums(reverse)
    try:
        o = oracle.Oracle(wl.grid, wl.const)
        s = o.derive(fields if fields is not None else wl.fields)
        o.step(s, 1)
    finally:
        oracle.set_reverse_sums(False)
    return s


def ulp_noise(fields, seed=0):
    """Every value moved to its upper or lower FP64 neighbour at random."""
    rng = np.random.default_rng(seed)
    out = {}
    for k in ("rho", "rhou", "rhow", "rhoe"):
        v = np.ascontiguousarray(fields[k], dtype=np.float64)
        up = rng.integers(0, 2, size=v.shape).astype(bool)
        out[k] = np.where(up, np.nextafter(v, np.inf), np.nextafter(v, -np.inf))
    return out


def field_errors(a, b, wl):
    cv = wl.const.cp - wl.const.R
    ca = a.conservative(wl.const.g, cv, wl.grid.dz)
    cb = b.conservative(wl.const.g, cv, wl.grid.dz)
    m = np.hypot(np.linalg.norm(cb["rhou"]), np.linalg.norm(cb["rhow"]))
    f = np.hypot(np.linalg.norm(b["phix"]), np.linalg.norm(b["phiz"]))
    out = {}
    for k in ("rho", "rhoe"):
        out[k] = np.linalg.norm(ca[k] - cb[k]) / np.linalg.norm(cb[k])
    for k in ("rhou", "rhow"):
        out[k] = np.linalg.norm(ca[k] - cb[k]) / m
    for k in ("T", "h", "p", "pp", "pold"):
        out[k] = np.linalg.norm(a[k] - b[k]) / np.linalg.norm(b[k])
    for k in ("phix", "phiz"):
        out[k] = np.linalg.norm(a[k] - b[k]) / f
    return out


def main():
    wl = W.get("bubble4096x2048")
    fwd = run(wl, False)
    rev = field_errors(run(wl, True), fwd, wl)
    ulp = field_errors(run(wl, False, ulp_noise(wl.fields)), fwd, wl)
    with open(OUT, "w") as fh:
        fh.write("# Round-off floor of one oracle step, smooth bubble 4096 x 2048 (dt 0.05 s,\n"
                 "# cg_rtol 1e-17): relative L2 difference from the plain oracle run of (a) the\n"
                 "# oracle with its reductions in reverse index order and (b) the oracle from\n"
                 "# inputs moved by one ulp up or down at random (seed 0). Momenta and face\n"
                 "# fluxes against the norm of their vector. Written by make_roundoff_floor.py.\n"
                 "# field reverse_sums ulp_inputs\n")
        for k in rev:
            fh.write(f"{k} {rev[k]:.6e} {ulp[k]:.6e}\n")
    print(rev)
    print(ulp)


if __name__ == "__main__":
    main()
