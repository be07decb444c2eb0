"""Tile columns of the graph driver's per-phase reduction kernels
(gea_set_tiles_per_block) and the tile-column autotuner (Solver.tune_tiles).

A block walking n tiles of a column changes only which tiles share a block
partial, so the step's results agree across n to the order of the
reduction sums. The grid is ragged in both directions (1000 x 516 cells:
the last tile column 8 cells wide, the last tile row 4 cells high), and
n = 16 leaves the last block of each column with one tile.
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea
    return gea


def run(G, wl, n, steps, mixed=False):
    s = G.Solver(wl.grid, wl.const, graph=True, mixed=mixed)
    s.set_conservative(wl.fields)
    s.set_tiles_per_block(n)
    s.step(steps)
    st = s.stats()
    out = s.get_full()
    s.close()
    assert st["status"] == 0, st
    return out, st


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_results_do_not_depend_on_the_tile_column(G, mixed):
    wl = W.smooth_bubble_20km(1000, 516, dt=0.1, steps=4)
    ref, st0 = run(G, wl, 1, 4, mixed)
    for n in (0, 3, 4, 16):
        got, st = run(G, wl, n, 4, mixed)
        for k in ("rho", "T", "pp", "u", "w"):
            d = np.linalg.norm(got[k] - ref[k])
            scale = np.linalg.norm(ref[k]) if k not in ("u", "w") else \
                np.hypot(np.linalg.norm(ref["u"]), np.linalg.norm(ref["w"]))
            # FP64: the order of the sums; mixed: the FP32 inner solves'
            # iterates move by their rounding (bound well inside the mixed
            # step's own distance to the FP64 step)
            assert d <= (1e-8 if mixed else 1e-11) * scale, (n, k, d / scale)


def test_tuner_picks_a_candidate_and_keeps_stepping(G):
    wl = W.smooth_bubble_20km(1024, 512, dt=0.1, steps=20)
    s = G.Solver(wl.grid, wl.const, graph=True)
    s.set_conservative(wl.fields)
    res = s.tune_tiles(candidates=(1, 4), steps=2)
    assert res["tiles_per_block"] in (1, 4)
    assert set(res["ms_per_step"]) == {1, 4} and all(v > 0 for v in res["ms_per_step"].values())
    s.step(2)
    st = s.stats()
    assert st["status"] == 0 and st["steps_done"] == 2 + 2 * 3, st
    with pytest.raises(G.GeaError) as ei:
        s.set_tiles_per_block(17)
    assert ei.value.code == G.GEA_ERR_INVAL
    s.close()
