"""Tile shapes of the persistent step kernels (gea_set_tile_shape) and the
tile-shape autotuners (Solver.tune_tile_shape, ensemble.autotune).

The persistent kernels exist for 32 x 8, 16 x 16 and 64 x 4 tiles (one
thread per cell, 256 threads a block). The shape decides which cells share a
block and so only the order of the reduction sums: every shape meets the
oracle parity bar (1e-10 relative L2 per field after 20 steps) on a grid
that is ragged against all three shapes (100 x 70 cells: 4 x 9, 7 x 5 and
2 x 18 tiles, each with partial tiles), for the FP64 step, the
mixed-precision step (its bar against the oracle) and an ensemble launch.
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [0, 1, 2]


@pytest.fixture(scope="module")
def gea():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea as G
    return G


def rel_l2(a, b):
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def ragged():
    grid = W.Grid(100, 70, 40.0 * 100, 30.0 * 70)
    c = W.Constants(dt=0.2, n_corr=2, mu=1.5)
    return W.random_flow(grid, c, seed=10070, uamp=3.0, thamp=2.0)


_REF = {}


def oracle_ref(oracle_mod, wl, steps):
    if steps not in _REF:
        o = oracle_mod.Oracle(wl.grid, wl.const)
        so = o.derive(wl.fields)
        o.step(so, steps)
        _REF[steps] = so
    return _REF[steps]


def errors(s, so, wl):
    cv = wl.const.cp - wl.const.R
    co = so.conservative(wl.const.g, cv, wl.grid.dz)
    gc = s.get_conservative()
    g = s.get_full()
    e = {k: rel_l2(gc[k], co[k]) for k in ("rho", "rhou", "rhow", "rhoe")}
    e.update({k: rel_l2(g[k], so[k]) for k in ("T", "pp", "phix", "phiz")})
    return e


@pytest.mark.parametrize("shape", SHAPES, ids=["32x8", "16x16", "64x4"])
def test_shape_parity_fp64(gea, oracle_mod, shape):
    wl = ragged()
    so = oracle_ref(oracle_mod, wl, 20)
    s = gea.Solver(wl.grid, wl.const)
    s.set_tile_shape(shape)
    s.set_conservative(wl.fields)
    s.step(20)
    st = s.stats()
    assert st["driver"] == "persistent" and st["status"] == 0, st
    e = errors(s, so, wl)
    assert max(e.values()) <= 1e-10, e


@pytest.mark.parametrize("shape", SHAPES, ids=["32x8", "16x16", "64x4"])
def test_shape_parity_mixed(gea, oracle_mod, shape):
    """The mixed-precision step (FP32 inner solves to 1e-5 of their initial
    residual) against the FP64 oracle: the bars of its ragged-size tests
    (scalars 5e-9, momenta 5e-7 relative L2)."""
    wl = ragged()
    so = oracle_ref(oracle_mod, wl, 20)
    s = gea.Solver(wl.grid, wl.const, mixed=True)
    s.set_tile_shape(shape)
    s.set_conservative(wl.fields)
    s.step(20)
    assert s.stats()["driver"] == "mixed_persistent"
    e = errors(s, so, wl)
    assert e["rho"] <= 5e-9 and e["rhoe"] <= 5e-9 and e["T"] <= 5e-9 and e["pp"] <= 5e-9, e
    assert e["rhou"] <= 5e-7 and e["rhow"] <= 5e-7, e


def test_shapes_agree_to_reduction_order(gea):
    """The three shapes give the same state up to the order of the sums."""
    wl = W.get("bubble160x80")
    out = []
    for shape in SHAPES:
        s = gea.Solver(wl.grid, wl.const)
        s.set_tile_shape(shape)
        s.set_conservative(wl.fields)
        s.step(20)
        out.append(s.get_full())
    for o in out[1:]:
        for k in ("rho", "T", "pp"):
            assert np.abs(o[k] - out[0][k]).max() <= 1e-13 * np.abs(out[0][k]).max(), k
        for k in ("u", "w"):
            assert np.abs(o[k] - out[0][k]).max() <= 1e-10 * np.abs(out[0]["w"]).max(), k


def test_ensemble_shape_matches_member_runs(gea):
    """An ensemble launch with 16 x 16 tiles gives each member its own
    persistent run's result (same shape) up to the order of the sums."""
    wls = [W.random_flow(W.Grid(nx, nz, 40.0 * nx, 30.0 * nz), W.Constants(dt=0.2, mu=1.5),
                         seed=nx + nz, uamp=2.0) for nx, nz in ((64, 48), (100, 70), (40, 24))]
    solvers = []
    for wl in wls:
        s = gea.Solver(wl.grid, wl.const)
        s.set_tile_shape(1)
        s.set_conservative(wl.fields)
        solvers.append(s)
    E = gea.Ensemble(solvers)
    E.step(10)
    E.close()
    for s, wl in zip(solvers, wls):
        ref = gea.Solver(wl.grid, wl.const)
        ref.set_tile_shape(1)
        ref.set_conservative(wl.fields)
        ref.step(10)
        a, b = s.get_full(), ref.get_full()
        for k in ("rho", "T", "pp"):
            assert np.abs(a[k] - b[k]).max() <= 1e-13 * np.abs(b[k]).max(), k
        for k in ("u", "w"):
            vmax = max(np.abs(b["u"]).max(), np.abs(b["w"]).max())
            assert np.abs(a[k] - b[k]).max() <= 1e-10 * vmax, k


def test_mixed_shapes_rejected_in_one_ensemble(gea):
    wl = W.get("bubble160x80")
    a = gea.Solver(wl.grid, wl.const)
    b = gea.Solver(wl.grid, wl.const)
    b.set_tile_shape(2)
    with pytest.raises(gea.GeaError) as ei:
        gea.Ensemble([a, b])
    assert ei.value.code == gea.GEA_ERR_INVAL


def test_tile_shape_autotuners(gea):
    """The single-context tuner keeps the fastest shape and the state goes on
    stepping correctly; the ensemble tuner reports every shape it timed."""
    import torch
    from paper_2303_10499_gb300 import ensemble
    wl = W.get("bubble640x320")
    s = gea.Solver(wl.grid, wl.const, stream=torch.cuda.current_stream())
    s.set_conservative(wl.fields)
    rep = s.tune_tile_shape(steps=2)
    assert set(rep["ms_per_step"]) == {"32x8", "16x16", "64x4"}
    assert rep["tile_shape"] == min(rep["ms_per_step"], key=rep["ms_per_step"].get)
    s.step(2)
    assert s.stats()["status"] == 0
    sols = [gea.Solver(w.grid, w.const) for w in W.les_ensemble(6, seed=0)]
    for sv, w in zip(sols, W.les_ensemble(6, seed=0)):
        sv.set_conservative(w.fields)
    E, rep = ensemble.autotune(sols, betas=(0.0, 1.0), trial_steps=1)
    assert set(rep["ms_per_step_by_shape_and_beta"]) == {"32x8", "16x16", "64x4"}
    E.step(1)
    E.close()
    for sv in sols:
        assert sv.stats()["status"] == 0
