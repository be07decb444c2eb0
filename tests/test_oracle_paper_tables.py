"""The oracle against numbers the paper prints for its own solver: the
non-smooth rising thermal bubble of Section 4.2 at 10 m resolution, whose
theta' extrema at t = 420 s Table 3 gives (tests/golden/paper_tables.txt).

The oracle and the paper's OpenFOAM solver share the scheme of Section 3 but
not its unstated details (interpolation, boundary and solver settings), so
agreement is expected within a band, the one the GPU test of the same
set-up uses: theta'_max within 3 %, the small undershoot theta'_min of the
printed sign and within a factor 2. The linear solves stop at 1e-10 of
their right-hand side here (the parity runs use 1e-17): far below what moves
an extremum by a fraction of the band, and it keeps the 4200 steps of this
run to about a minute of one host core.
"""
import dataclasses
import os

import numpy as np

import oracle
from paper_2303_10499_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def table3(res, t):
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        case, r, tt, q, v = line.split()
        if case == "nonsmooth" and int(r) == res and int(tt) == t:
            rows[q] = float(v)
    return rows


def test_nonsmooth_bubble_10m_table3_at_420s():
    wl = W.paper_nonsmooth_bubble(10.0)
    const = dataclasses.replace(wl.const, cg_rtol=1e-10, jac_rtol=1e-10)
    o = oracle.Oracle(wl.grid, const)
    s = o.derive(wl.fields)
    steps = int(round(420.0 / const.dt))
    o.step(s, steps)
    th, _, _ = o.diagnostics(s, wl.theta_bar)
    want = table3(10, 420)
    print("theta' extrema", float(th.min()), float(th.max()), "Table 3", want)
    assert np.isfinite(th).all()
    assert abs(th.max() - want["th_max"]) <= 0.03 * want["th_max"], (th.max(), want["th_max"])
    assert 2.0 * want["th_min"] <= th.min() <= 0.5 * want["th_min"], (th.min(), want["th_min"])
