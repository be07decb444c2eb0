"""The multigrid preconditioner of the pressure solve (Section 3, Step 3:
eq. p_prime_sd in its Helmholtz form, solved by CG with one V(1,1)-cycle of a
Galerkin hierarchy as the preconditioner).

The default hierarchy of the 160 x 80 and 640 x 320 bubbles has one level
(their Helmholtz operator is strongly diagonally dominant), so these tests
force deep hierarchies with mg_min_cells:

* CG needs a linear, symmetric, positive definite preconditioner. The
  V-cycle is applied through gea_apply_precond to seeded random vectors:
  x.My = y.Mx and M(x + 2y) = Mx + 2My to round-off, x.Mx > 0.
* The converged pressure does not depend on the preconditioner, so the
  100-step oracle parity bar of 1e-10 relative L2 per field holds with four
  levels on both drivers, and on a grid whose levels are all ragged against
  the 32 x 8 tile.
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


def rel_l2(a, b):
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


_ORACLE = {}


def oracle_state(oracle_mod, name, wl, steps):
    """The oracle's state after `steps` steps (cached: the same run serves both
    drivers)."""
    key = (name, steps)
    if key not in _ORACLE:
        o = oracle_mod.Oracle(wl.grid, wl.const)
        so = o.derive(wl.fields)
        o.step(so, steps)
        _ORACLE[key] = so
    return _ORACLE[key]


def check_state(gs, so, wl, tol):
    cv = wl.const.cp - wl.const.R
    co = so.conservative(wl.const.g, cv, wl.grid.dz)
    gc = gs.get_conservative()
    g = gs.get_full()
    errs = {k: rel_l2(gc[k], co[k]) for k in ("rho", "rhou", "rhow", "rhoe")}
    errs.update({k: rel_l2(g[k], so[k]) for k in ("T", "h", "p", "pp", "pold", "phix", "phiz")})
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    return errs


# (workload, mg_min_cells, levels): 160x80 -> 20x10 and 640x320 -> 80x40
DEEP = [("bubble160x80", 200, 4), ("bubble640x320", 3200, 4)]


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("name,mgmin,levels", DEEP)
def test_parity_100_steps_multilevel(gea, oracle_mod, name, mgmin, levels, graph):
    wl = W.get(name)
    so = oracle_state(oracle_mod, name, wl, 100)
    s = gea.Solver(wl.grid, wl.const, mg_min_cells=mgmin, graph=graph)
    s.set_conservative(wl.fields)
    s.step(100)
    st = s.stats()
    assert st["mg_levels"] == levels and st["status"] == 0, st
    assert st["driver"] == ("graph" if graph else "persistent"), st
    errs = check_state(s, so, wl, 1e-10)
    print(name, levels, errs, st)


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_parity_multilevel_ragged_even(gea, oracle_mod, graph):
    """96 x 64 down to 12 x 8: every level is ragged against the tile (3 x 8,
    1.5 x 4, 0.75 x 2 and 0.375 x 1 tiles), on a moving stratified state."""
    grid = W.Grid(96, 64, 40.0 * 96, 30.0 * 64)
    c = W.Constants(dt=0.2, n_corr=2, mu=1.5)
    wl = W.random_flow(grid, c, seed=9664, uamp=3.0, thamp=2.0)
    o = oracle_mod.Oracle(grid, c)
    so = o.derive(wl.fields)
    o.step(so, 20)
    s = gea.Solver(grid, c, mg_min_cells=100, graph=graph)
    s.set_conservative(wl.fields)
    s.step(20)
    assert s.stats()["mg_levels"] == 4
    check_state(s, so, wl, 1e-10)


@pytest.mark.parametrize("name,nx,nz,mgmin,levels", [
    ("bubble160x80", 160, 80, 200, 4),
    ("bubble640x320", 640, 320, 3200, 4),
    ("ragged96x64", 96, 64, 100, 4),
    ("single160x80", 160, 80, 0, 1),
])
def test_vcycle_linear_symmetric_positive(gea, name, nx, nz, mgmin, levels):
    """M = one V(1,1)-cycle (damped Jacobi pre-smoothing from zero, averaging
    restriction, Galerkin coarse operators, piecewise-constant prolongation,
    the same damped Jacobi post-smoothing; two sweeps on the coarsest level)
    is a symmetric positive definite linear operator, as the preconditioned
    CG of the pressure solve requires; an asymmetric or non-linear V-cycle
    would only slow CG down, which a parity test would not see."""
    if name.startswith("ragged"):
        grid = W.Grid(nx, nz, 40.0 * nx, 30.0 * nz)
        c = W.Constants(dt=0.2, n_corr=2, mu=1.5)
        wl = W.random_flow(grid, c, seed=7, uamp=3.0, thamp=2.0)
    else:
        wl = W.get(name.replace("single", "bubble"))
    s = gea.Solver(wl.grid, wl.const, mg_min_cells=mgmin)
    s.set_conservative(wl.fields)
    s.step(2)
    assert s.stats()["mg_levels"] == levels
    rng = np.random.default_rng(2303)
    for trial in range(3):
        x = rng.standard_normal((nz, nx))
        y = rng.standard_normal((nz, nx))
        if trial == 2:   # smooth vectors reach the coarse levels
            x = np.cumsum(np.cumsum(x, 0), 1)
            y = np.cumsum(np.cumsum(y, 0), 1)
        mx, my = s.apply_precond(x), s.apply_precond(y)
        sym = abs(np.vdot(x, my) - np.vdot(y, mx))
        assert sym <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(my), (trial, sym)
        assert np.vdot(x, mx) > 0 and np.vdot(y, my) > 0
        lin = s.apply_precond(x + 2.0 * y) - (mx + 2.0 * my)
        assert np.abs(lin).max() <= 1e-12 * (np.abs(mx).max() + 2.0 * np.abs(my).max()), trial
    # applying M leaves the solver state and its next step untouched
    ref = gea.Solver(wl.grid, wl.const, mg_min_cells=mgmin)
    ref.set_conservative(wl.fields)
    ref.step(3)
    s.step(1)
    a, b = s.get_full(), ref.get_full()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_smoother_weight_changes_iterations_not_the_solution(gea):
    """gea_set_smoother_weight: the weight of the preconditioner's Jacobi
    sweeps changes how fast CG converges, not what it converges to (the
    pressure solve runs to the same relative residual), on a one-level and a
    three-level hierarchy; weights outside (0, 2) are refused."""
    for name, mgmin in (("bubble160x80", 0), ("bubble160x80", 400)):
        wl = W.get(name)
        out = []
        for om in (None, 0.7, 0.95):
            s = gea.Solver(wl.grid, wl.const, mg_min_cells=mgmin)
            s.set_conservative(wl.fields)
            if om is not None:
                s.set_smoother_weight(om)
            s.step(5)
            assert s.stats()["status"] == 0
            out.append(s.get_full())
            s.close()
        ref = out[0]
        vel = np.hypot(np.linalg.norm(ref["u"]), np.linalg.norm(ref["w"]))
        for g in out[1:]:
            for f in ("rho", "T", "pp"):
                assert np.linalg.norm(g[f] - ref[f]) / np.linalg.norm(ref[f]) < 1e-12, (name, mgmin, f)
            for f in ("u", "w"):
                assert np.linalg.norm(g[f] - ref[f]) / vel < 1e-9, (name, mgmin, f)
    s = gea.Solver(wl.grid, wl.const)
    for bad in (0.0, -0.5, 2.0):
        with pytest.raises(gea.GeaError):
            s.set_smoother_weight(bad)
    s.close()
