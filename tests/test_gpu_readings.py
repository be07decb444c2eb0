"""Reading flags (gea_constants.reading_flags): the literal K^{n-1} of eq.
step3_sd (GEA_READING_K_LAGGED) against the oracle with the same reading.

The reading changes one term of the enthalpy right-hand side, rho^n K^n ->
rho^n K^{n-1}, and makes K^{n-1} part of the state. The oracle's pin
(tests/test_oracle_pins.py) fixes that term's sign and factor; here the CUDA
path matches that oracle to the parity bar (1e-10 relative L2 per field
after 100 steps) on both drivers, the FULL checkpoint carries K^{n-1} bit
for bit, and the reading does change the flow.
"""
import dataclasses

import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def lagged(wl, gea):
    wl = dataclasses.replace(wl)
    wl.const = dataclasses.replace(wl.const, reading_flags=gea.READING_K_LAGGED)
    return wl


_REF = {}


def oracle_run(oracle_mod, key, wl, steps):
    if key not in _REF:
        o = oracle_mod.Oracle(wl.grid, wl.const)
        so = o.derive(wl.fields)
        o.step(so, steps)
        _REF[key] = so
    return _REF[key]


def errs(s, so, wl):
    cv = wl.const.cp - wl.const.R
    co = so.conservative(wl.const.g, cv, wl.grid.dz)
    gc, g = s.get_conservative(), s.get_full()
    e = {k: rel_l2(gc[k], co[k]) for k in ("rho", "rhou", "rhow", "rhoe")}
    e.update({k: rel_l2(g[k], so[k]) for k in ("T", "h", "p", "pp", "pold", "phix", "phiz", "Kold")})
    return e


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_lagged_k_parity_100_steps(gea, oracle_mod, graph):
    wl = lagged(W.get("bubble160x80"), gea)
    so = oracle_run(oracle_mod, "bubble", wl, 100)
    s = gea.Solver(wl.grid, wl.const, graph=graph)
    s.set_conservative(wl.fields)
    s.step(100)
    e = errs(s, so, wl)
    assert max(e.values()) <= 1e-10, e


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_lagged_k_parity_moving_ragged(gea, oracle_mod, graph):
    """A moving stratified state on a ragged grid (K^{n-1} and K^n differ
    everywhere from the second step on)."""
    grid = W.Grid(66, 42, 40.0 * 66, 30.0 * 42)
    wl = lagged(W.random_flow(grid, W.Constants(dt=0.2, mu=1.5), seed=6642, uamp=4.0, thamp=2.0), gea)
    so = oracle_run(oracle_mod, "ragged", wl, 20)
    s = gea.Solver(grid, wl.const, graph=graph)
    s.set_conservative(wl.fields)
    s.step(20)
    e = errs(s, so, wl)
    assert max(e.values()) <= 1e-10, e
    # the reading matters: the default reading's flow differs
    d = gea.Solver(grid, dataclasses.replace(wl.const, reading_flags=0), graph=graph)
    d.set_conservative(wl.fields)
    d.step(20)
    assert rel_l2(d.get_full()["h"], s.get_full()["h"]) > 1e-9


def test_lagged_k_mixed_against_oracle(gea, oracle_mod):
    """The mixed-precision step with the same reading (its ragged-size bars)."""
    grid = W.Grid(66, 42, 40.0 * 66, 30.0 * 42)
    wl = lagged(W.random_flow(grid, W.Constants(dt=0.2, mu=1.5), seed=6642, uamp=4.0, thamp=2.0), gea)
    so = oracle_run(oracle_mod, "ragged", wl, 20)
    s = gea.Solver(grid, wl.const, mixed=True)
    s.set_conservative(wl.fields)
    s.step(20)
    e = errs(s, so, wl)
    assert e["rho"] <= 5e-9 and e["rhoe"] <= 5e-9 and e["T"] <= 5e-9, e
    assert e["rhou"] <= 5e-7 and e["rhow"] <= 5e-7, e


def test_lagged_k_checkpoint_bitwise(gea):
    wl = lagged(W.get("bubble160x80"), gea)
    a = gea.Solver(wl.grid, wl.const)
    a.set_conservative(wl.fields)
    a.step(4)
    ck = a.get_full()
    a.step(3)
    ref = a.get_full()
    b = gea.Solver(wl.grid, wl.const)
    b.set_full(ck)
    b.step(3)
    got = b.get_full()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    # without K^{n-1} the state of this reading is incomplete
    del ck["Kold"]
    with pytest.raises(gea.GeaError) as ei:
        b.set_full(ck)
    assert ei.value.code == gea.GEA_ERR_INVAL


def test_reading_flags_validated(gea):
    wl = W.get("bubble160x80")
    with pytest.raises(gea.GeaError):
        gea.Solver(wl.grid, dataclasses.replace(wl.const, reading_flags=2))
    g3 = W.Grid3(8, 8, 8, 800.0, 800.0, 800.0)
    with pytest.raises(gea.GeaError):
        gea.Solver3D(g3, dataclasses.replace(wl.const, reading_flags=1))
