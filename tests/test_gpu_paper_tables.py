"""The paper's benchmark extrema (tests/golden/paper_tables.txt: Section 4.1
Table 1 and Section 4.2 Table 3, the values it prints for its own solver)
against this step on the same set-ups, run on the GPU (the FP64 step equals
the oracle to 1e-10 per field over 100 steps, tests/test_gpu_parity.py).

The two solvers share the scheme of Section 3 but not its unstated
details (OpenFOAM's interpolation, boundary and solver settings against
the readings here), so only agreement within a stated band is expected.
Measured: u and w extrema within 0.9 % of Table 1 (u +-1.916, w -1.697 and
2.482 m/s); theta'_max within 1.7 % of Table 3 (0.516, 0.529 at 5 m; 0.587,
0.569 at 10 m); the small undershoots theta'_min have the printed sign and
magnitude within a factor 2 (-0.014, -0.017 at 5 m; -0.042, -0.104 at
10 m), being sensitive to the dispersive fourth-order face values. Bands:
3 %, 3 % and a factor 2.
"""
import os

import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def table():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        case, res, t, q, v = line.split()
        rows[(case, int(res), int(t), q)] = float(v)
    return rows


@pytest.fixture(scope="module")
def gea():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea as G
    return G


def extrema(G, wl, times):
    """u, w and theta' extrema at the given times (s), stepping dt."""
    s = G.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    out, done = {}, 0
    for t in times:
        n = int(round(t / wl.const.dt)) - done
        s.step(n)
        done += n
        assert s.stats()["status"] == 0
        f = s.get_full()
        th, _, _ = s.diagnostics(wl.theta_bar)
        out[t] = {"u_min": f["u"].min(), "u_max": f["u"].max(), "w_min": f["w"].min(),
                  "w_max": f["w"].max(), "th_min": th.min(), "th_max": th.max()}
    s.close()
    return out


def test_smooth_bubble_table1(gea):
    ref = table()
    got = extrema(gea, W.paper_smooth_bubble(5.0), [600])[600]
    print({k: round(float(v), 4) for k, v in got.items()})
    for q in ("u_min", "u_max", "w_min", "w_max"):
        want = ref[("smooth", 5, 600, q)]
        assert abs(got[q] - want) <= 0.03 * abs(want), (q, got[q], want)
    # the printed u extrema are mirror images; so are ours (symmetric bubble)
    assert abs(got["u_min"] + got["u_max"]) <= 1e-9 * got["u_max"]


@pytest.mark.parametrize("res", [5, 10])
def test_nonsmooth_bubble_table3(gea, res):
    ref = table()
    got = extrema(gea, W.paper_nonsmooth_bubble(float(res)), [420, 600])
    print(res, {t: {k: round(float(v), 4) for k, v in d.items() if k.startswith("th")} for t, d in got.items()})
    for t in (420, 600):
        want = ref[("nonsmooth", res, t, "th_max")]
        assert abs(got[t]["th_max"] - want) <= 0.03 * want, (res, t, got[t]["th_max"], want)
        lo = ref[("nonsmooth", res, t, "th_min")]
        assert 2.0 * lo <= got[t]["th_min"] <= 0.5 * lo, (res, t, got[t]["th_min"], lo)
