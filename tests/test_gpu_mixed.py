"""The mixed-precision step (GEA_FLAG_MIXED) against the FP64 oracle.

The mixed step solves the same discrete equations (Section 3) with each
linear solve done as one defect correction: FP64 residual, FP32 solve of the
increment to ||r|| <= mp_rtol ||r0||, FP64 update. Its results therefore
differ from the FP64 solution by the inexact solves, not by round-off: a
solve leaves an error of about mp_rtol times the increment it computes, and
these errors accumulate over the run. The bar for this path is the accuracy
the application needs: max |theta'| error <= 1e-3 K after 100 steps of the
rising-bubble workloads, with the relative L2 errors of rho, rho u, rho w
and rho e reported and bounded. Measured, the path is far inside that bar
(about 1e-9 K and 5e-10 in the momenta), because each solve only computes
the step's increment of an FP64 field; the bounds below are regression
bounds a factor ~10 above the measured errors.
"""
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


def field_errors(gs, so, const, grid):
    """Relative L2 errors of the conservative fields (momenta against the
    norm of the momentum vector) and the primitive ones."""
    cv = const.cp - const.R
    co = so.conservative(const.g, cv, grid.dz)
    z = (np.arange(grid.nz) + 0.5)[:, None] * grid.dz
    cg = {"rho": gs["rho"], "rhou": gs["rho"] * gs["u"], "rhow": gs["rho"] * gs["w"],
          "rhoe": gs["rho"] * (cv * gs["T"] + 0.5 * (gs["u"] ** 2 + gs["w"] ** 2) + const.g * z)}
    m = np.hypot(np.linalg.norm(co["rhou"]), np.linalg.norm(co["rhow"]))
    out = {}
    for k in ("rho", "rhoe"):
        out[k] = np.linalg.norm(cg[k] - co[k]) / np.linalg.norm(co[k])
    for k in ("rhou", "rhow"):
        out[k] = np.linalg.norm(cg[k] - co[k]) / m
    for k in ("T", "p", "pp"):
        out[k] = np.linalg.norm(gs[k] - so[k]) / np.linalg.norm(so[k])
    return out


_ORACLE_100 = {}


def oracle_100(oracle_mod, name):
    """The oracle's state after 100 steps of a named workload (computed once)."""
    if name not in _ORACLE_100:
        wl = W.get(name)
        o = oracle_mod.Oracle(wl.grid, wl.const)
        so = o.derive(wl.fields)
        o.step(so, 100)
        _ORACLE_100[name] = (o, so)
    return _ORACLE_100[name]


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("name", ["bubble160x80", "bubble640x320"])
def test_mixed_100_steps_against_oracle(gea, oracle_mod, name, graph):
    wl = W.get(name)
    o, so = oracle_100(oracle_mod, name)
    s = gea.Solver(wl.grid, wl.const, mixed=True, graph=graph)
    s.set_conservative(wl.fields)
    s.step(100)
    st = s.stats()
    assert st["driver"] == ("mixed" if graph else "mixed_persistent")
    assert st["status"] == 0 and st["steps_done"] == 100
    errs = field_errors(s.get_full(), so, wl.const, wl.grid)
    th_g, m_g, _ = s.diagnostics(wl.theta_bar)
    th_o, m_o, _ = o.diagnostics(so, wl.theta_bar)
    dth = np.abs(th_g - th_o).max()
    print(name, "max|dtheta'|", dth, errs, st)
    assert dth <= 1e-3
    # measured (default mp_rtol 1e-5): dtheta' 1.3e-9 K, rho u 4.7e-10, rho w
    # 4.1e-10, rho 4.5e-13, rho e 1.4e-13; the bounds leave a factor ~10
    assert dth <= 1e-7
    assert errs["rho"] <= 1e-11 and errs["rhoe"] <= 1e-11 and errs["T"] <= 1e-11
    assert errs["p"] <= 1e-11 and errs["pp"] <= 1e-11
    assert errs["rhou"] <= 5e-9 and errs["rhow"] <= 5e-9
    # the FP32 solves change mass only by the FP64 flux update (conservative)
    assert abs(m_g - m_o) / m_o < 1e-11


@pytest.mark.parametrize("nx,nz,ncorr", [(37, 23, 2), (66, 130, 3), (4, 4, 1), (128, 96, 2)])
def test_mixed_ragged_sizes(gea, oracle_mod, nx, nz, ncorr):
    """Sizes off the 32 x 8 tile, odd sizes (one multigrid level), the
    smallest grid, several corrector counts, on a moving stratified state."""
    grid = W.Grid(nx, nz, 40.0 * nx, 30.0 * nz)
    c = W.Constants(dt=0.2, n_corr=ncorr, mu=1.5)
    wl = W.random_flow(grid, c, seed=nx * 1000 + nz, uamp=3.0, thamp=2.0)
    o = oracle_mod.Oracle(grid, c)
    so = o.derive(wl.fields)
    o.step(so, 20)
    s = gea.Solver(grid, c, mixed=True)
    s.set_conservative(wl.fields)
    s.step(20)
    errs = field_errors(s.get_full(), so, c, grid)
    print((nx, nz), errs, s.stats())
    # measured: up to 3.3e-10 (rho, rho e) and 3.2e-8 (momenta, 4 x 4 grid)
    assert errs["rho"] <= 5e-9 and errs["rhoe"] <= 5e-9
    assert errs["rhou"] <= 5e-7 and errs["rhow"] <= 5e-7


def test_mixed_rest_atmosphere(gea):
    """A hydrostatic rest state: every r0 is round-off, so the FP32 solves
    add round-off-sized increments and the atmosphere stays at rest."""
    wl = W.rest_atmosphere(W.Grid(160, 80, 20000.0, 10000.0), W.Constants(dt=0.1))
    s = gea.Solver(wl.grid, wl.const, mixed=True)
    s.set_conservative(wl.fields)
    s.step(100)
    st = s.get_full()
    assert np.abs(st["u"]).max() < 1e-9 and np.abs(st["w"]).max() < 1e-9
    th, _, _ = s.diagnostics(wl.theta_bar)
    assert np.abs(th).max() < 1e-9


def test_mixed_profiled_step_equals_graph_step(gea):
    """The per-kernel profiled step launches the same kernels in the same
    order as the graph: identical results, bit for bit."""
    wl = W.get("bubble640x320")
    a = gea.Solver(wl.grid, wl.const, mixed=True, graph=True)
    a.set_conservative(wl.fields)
    a.step(3)
    b = gea.Solver(wl.grid, wl.const, mixed=True, graph=True)
    b.set_conservative(wl.fields)
    b.step(2)
    prof = b.profile_step()
    assert any(k.startswith("mx_") for k in prof)
    ra, rb = a.get_full(), b.get_full()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


def test_mixed_deterministic_and_checkpoint(gea):
    wl = W.get("bubble160x80")
    out = []
    for _ in range(2):
        s = gea.Solver(wl.grid, wl.const, mixed=True)
        s.set_conservative(wl.fields)
        s.step(10)
        out.append(s.get_full())
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
    b = gea.Solver(wl.grid, wl.const, mixed=True)
    b.set_full(out[0])
    b.step(4)
    a = gea.Solver(wl.grid, wl.const, mixed=True)
    a.set_conservative(wl.fields)
    a.step(14)
    ra, rb = a.get_full(), b.get_full()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


def test_mixed_noconv_keeps_last_state(gea):
    wl = W.get("bubble160x80")
    wl.const.cg_maxit = 1
    s = gea.Solver(wl.grid, wl.const, mixed=True, mp_rtol=1e-7)
    s.set_conservative(wl.fields)
    before = s.get_full()
    with pytest.raises(gea.GeaError) as ei:
        s.step(3)
    assert ei.value.code == gea.GEA_ERR_NOCONV
    after = s.get_full()
    for k in before:
        assert np.array_equal(before[k], after[k]), k


def test_mixed_tolerance_controls_error(gea, oracle_mod):
    """A tighter inner tolerance gives a smaller error against the oracle."""
    wl = W.get("bubble160x80")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, 30)
    e = {}
    for rt in (1e-3, 1e-6):
        s = gea.Solver(wl.grid, wl.const, mixed=True, mp_rtol=rt)
        s.set_conservative(wl.fields)
        s.step(30)
        e[rt] = field_errors(s.get_full(), so, wl.const, wl.grid)
    print(e)
    assert e[1e-6]["rhow"] < e[1e-3]["rhow"]


def test_mixed_persistent_and_graph_agree(gea):
    """The two drivers of the mixed step run the same tile functions; the
    FP32 reductions are grouped differently (a persistent block sums several
    tiles), so the inner solves differ at FP32 rounding and the FP64 fields
    agree to far below the step's own error against the FP64 solution."""
    wl = W.get("bubble640x320")
    out = []
    for graph in (False, True):
        s = gea.Solver(wl.grid, wl.const, mixed=True, graph=graph)
        s.set_conservative(wl.fields)
        s.step(20)
        assert s.stats()["status"] == 0
        out.append(s.get_full())
    for k in ("rho", "T", "pp"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-11 * np.abs(out[1][k]).max(), k
    vmax = max(np.abs(out[1]["u"]).max(), np.abs(out[1]["w"]).max())
    for k in ("u", "w"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-8 * vmax, k


def test_mixed_persistent_multi_step_launch(gea):
    """n steps in one persistent launch equal n launches of one step, bit
    for bit, and the persistent driver is deterministic."""
    wl = W.get("bubble160x80")
    a = gea.Solver(wl.grid, wl.const, mixed=True)
    a.set_conservative(wl.fields)
    a.step(6)
    assert a.stats()["driver"] == "mixed_persistent"
    b = gea.Solver(wl.grid, wl.const, mixed=True)
    b.set_conservative(wl.fields)
    for _ in range(6):
        b.step(1)
    ra, rb = a.get_full(), b.get_full()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
