"""Parity of the three-dimensional CUDA step (include/gea3d.h) with the FP64
three-dimensional oracle, and properties that hold at any size.

Tolerances as in the two-dimensional parity tests: every solve is driven to
round-off, so the two sides differ by summation order only; 1e-10 relative
L2 per field, velocity components against the norm of the velocity vector.
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "u", "v", "w", "T", "p", "pp")


@pytest.fixture(scope="module")
def gea():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea as G
    return G


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3d
    return oracle3d


def compare(g, so, tol):
    vel = np.sqrt(sum(np.linalg.norm(so[k]) ** 2 for k in ("u", "v", "w")))
    out = {}
    for k in FIELDS:
        ref = vel if k in ("u", "v", "w") else np.linalg.norm(so[k])
        out[k] = np.linalg.norm(g[k] - so[k]) / max(ref, 1e-300)
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, (bad, out)
    return out


def run_both(gea, o3, wl, steps, **kw):
    q = o3.Oracle3D(wl.grid, wl.const)
    so = q.derive(wl.fields)
    sto = q.step(so, steps)
    s = gea.Solver3D(wl.grid, wl.const, **kw)
    s.set_conservative(wl.fields)
    s.step(steps)
    return so, sto, s


@pytest.mark.parametrize("shape,steps", [((24, 20, 12), 20), ((40, 12, 18), 100), ((33, 9, 5), 10)],
                         ids=["24x20x12", "40x12x18", "33x9x5"])
def test_parity_random_flow(gea, o3, shape, steps):
    """A moving stratified flow with all terms active, on sizes with ragged
    x and y blocks (33 and 9 cells: one cell past a full tile)."""
    nx, ny, nz = shape
    g = W.Grid3(nx, ny, nz, 100.0 * nx, 100.0 * ny, 100.0 * nz)
    c = W.Constants(dt=0.2, mu=1.5)
    wl = W.random_flow3(g, c, seed=11, uamp=3.0, thamp=2.0)
    so, sto, s = run_both(gea, o3, wl, steps)
    st = s.stats()
    assert st["status"] == 0 and st["steps_done"] == steps
    compare(s.get_state(), so, 1e-10)
    # the solves ran to the same tolerances in comparable iterations
    assert abs(st["jac_u"] - sto["jac_u"]) <= 2 and abs(st["jac_h"] - sto["jac_h"]) <= 2
    assert all(r <= c.cg_rtol * 1.0001 for r in st["cg_relres"])


def test_parity_prandtl_and_three_correctors(gea, o3):
    """Pr != 1 (enthalpy diffusion mu/Pr differs from the momentum's) and
    three PISO correctors."""
    g = W.Grid3(20, 12, 16, 2000.0, 1200.0, 1600.0)
    c = W.Constants(dt=0.2, mu=2.0, Pr=0.7, n_corr=3)
    wl = W.random_flow3(g, c, seed=9, uamp=3.0, thamp=2.0)
    so, sto, s = run_both(gea, o3, wl, 20)
    st = s.stats()
    assert st["status"] == 0 and len(st["cg_iters"]) == 3
    compare(s.get_state(), so, 1e-10)


@pytest.mark.parametrize("shape", [(24, 20, 12), (33, 9, 5)], ids=["24x20x12", "33x9x5"])
def test_parity_les(gea, o3, shape):
    """Smagorinsky LES (cs = 0.17, Pr = 1) on a sheared stratified flow: the
    eddy viscosity, its face means in the transport stencil and in H(u)."""
    nx, ny, nz = shape
    g = W.Grid3(nx, ny, nz, 100.0 * nx, 100.0 * ny, 100.0 * nz)
    c = W.Constants(dt=0.2, mu=0.5, cs=0.17)
    wl = W.random_flow3(g, c, seed=12, uamp=4.0, thamp=2.0)
    so, sto, s = run_both(gea, o3, wl, 20)
    st = s.stats()
    assert st["status"] == 0
    compare(s.get_state(), so, 1e-10)


def test_les_bubble_mirror_symmetry_and_mass(gea):
    """LES on the centred bubble keeps the x, y mirror symmetries and mass."""
    g = W.Grid3(64, 64, 32, 10000.0, 10000.0, 10000.0)
    c = W.Constants(dt=0.2, cs=0.17)
    wl = W.rising_bubble3(g, c, amp=2.0, rc=2000.0, xc=5000.0, yc=5000.0, zc=2000.0)
    s = gea.Solver3D(g, c)
    s.set_conservative(wl.fields)
    s.step(20)
    assert s.stats()["status"] == 0
    f = s.get_state()
    w, u, v = f["w"], f["u"], f["v"]
    sc = np.abs(w).max()
    assert sc > 1e-4
    assert np.abs(w - w[:, :, ::-1]).max() < 1e-8 * sc and np.abs(w - w[:, ::-1, :]).max() < 1e-8 * sc
    assert np.abs(u + u[:, :, ::-1]).max() < 1e-8 * sc and np.abs(v + v[:, ::-1, :]).max() < 1e-8 * sc
    m0 = wl.fields["rho"].sum()
    assert abs(f["rho"].sum() - m0) < 1e-13 * m0


def test_parity_bubble_multigrid_levels(gea, o3):
    """The rising bubble on a grid with three multigrid levels
    (48x32x16 -> 24x16x8 -> 12x8x4)."""
    g = W.Grid3(48, 32, 16, 4800.0, 3200.0, 1600.0)
    c = W.Constants(dt=0.5, mu=0.5)
    wl = W.rising_bubble3(g, c, amp=2.0, rc=800.0, xc=2000.0, yc=1500.0, zc=600.0)
    so, _, s = run_both(gea, o3, wl, 30, mg_min_cells=1)
    st = s.stats()
    assert st["mg_levels"] == 3 and st["status"] == 0
    compare(s.get_state(), so, 1e-10)


def test_y_invariant_state_matches_the_2d_library(gea):
    """An x-z state repeated along y stays y-invariant under the 3D step and
    equals the 2D library's step (two different programs)."""
    grid = W.Grid(40, 24, 4000.0, 2400.0)
    c = W.Constants(dt=0.2, mu=1.5)
    wl = W.random_flow(grid, c, seed=7, uamp=3.0, thamp=2.0)
    w3 = W.extrude3(wl, 8, 800.0)
    s2 = gea.Solver(grid, c)
    s2.set_conservative(wl.fields)
    s2.step(10)
    f2 = s2.get_full()
    s3 = gea.Solver3D(w3.grid, c)
    s3.set_conservative(w3.fields)
    s3.step(10)
    f3 = s3.get_state()
    assert np.abs(f3["v"]).max() < 1e-12 * max(1.0, np.abs(f3["u"]).max())
    for j in range(8):
        for k in ("rho", "u", "w", "T", "p", "pp"):
            err = np.abs(f3[k][:, j, :] - f2[k]).max() / np.abs(f2[k]).max()
            assert err < 1e-10, (k, j, err)


def test_rest_state_and_mass(gea):
    g = W.Grid3(20, 16, 24, 2000.0, 1600.0, 2400.0)
    c = W.Constants(dt=0.2)
    rest = W.rising_bubble3(g, c, amp=0.0)
    s = gea.Solver3D(g, c)
    s.set_conservative(rest.fields)
    s.step(20)
    f = s.get_state()
    assert max(np.abs(f[k]).max() for k in ("u", "v", "w")) < 1e-10
    wl = W.random_flow3(g, c, seed=5, uamp=2.0)
    s.set_conservative(wl.fields)
    m0 = wl.fields["rho"].sum()
    s.step(10)
    m1 = s.get_state()["rho"].sum()
    assert abs(m1 - m0) < 1e-13 * m0


def test_bubble_mirror_symmetry_at_128x128x64(gea):
    """At a size the oracle cannot follow: the centred bubble keeps its
    mirror symmetries in x and y, and mass is conserved (four multigrid
    levels, down to 16x16x8)."""
    g = W.Grid3(128, 128, 64, 10000.0, 10000.0, 10000.0)
    c = W.Constants(dt=0.1)
    wl = W.rising_bubble3(g, c, amp=2.0, rc=2000.0, xc=5000.0, yc=5000.0, zc=2000.0)
    s = gea.Solver3D(g, c, mg_min_cells=4096)
    s.set_conservative(wl.fields)
    s.step(20)
    st = s.stats()
    assert st["status"] == 0 and st["mg_levels"] == 4
    f = s.get_state()
    w, u, v = f["w"], f["u"], f["v"]
    sc = np.abs(w).max()
    assert sc > 1e-4
    assert np.abs(w - w[:, :, ::-1]).max() < 1e-8 * sc and np.abs(w - w[:, ::-1, :]).max() < 1e-8 * sc
    assert np.abs(u + u[:, :, ::-1]).max() < 1e-8 * sc and np.abs(v + v[:, ::-1, :]).max() < 1e-8 * sc
    assert np.abs(u - v.transpose(0, 2, 1)).max() < 1e-8 * sc
    m0 = wl.fields["rho"].sum()
    assert abs(f["rho"].sum() - m0) < 1e-13 * m0


def test_smallest_grid_and_device_buffers(gea, o3):
    """4x4x4 (one block, levels cannot coarsen) with torch device buffers in
    and out."""
    import torch
    g = W.Grid3(4, 4, 4, 400.0, 400.0, 400.0)
    c = W.Constants(dt=0.2, mu=1.0)
    wl = W.random_flow3(g, c, seed=2, uamp=1.0)
    q = o3.Oracle3D(g, c)
    so = q.derive(wl.fields)
    q.step(so, 5)
    s = gea.Solver3D(g, c)
    s.set_conservative({k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()})
    s.step(5)
    out = {k: torch.empty((4, 4, 4), dtype=torch.float64, device="cuda") for k in FIELDS}
    s.get_state(out)
    compare({k: v.cpu().numpy() for k, v in out.items()}, so, 1e-10)


def test_errors_are_reported(gea):
    g = W.Grid3(16, 8, 8, 1600.0, 800.0, 800.0)
    c = W.Constants(dt=0.2)
    wl = W.random_flow3(g, c, seed=1)
    s = gea.Solver3D(g, c)
    with pytest.raises(gea.GeaError) as ei:
        s.step(1)
    assert ei.value.code == gea.GEA_ERR_STATE
    bad = dict(wl.fields)
    bad["rho"] = bad["rho"].copy()
    bad["rho"][3, 2, 1] = -1.0
    with pytest.raises(gea.GeaError) as ei:
        s.set_conservative(bad)
    assert ei.value.code == gea.GEA_ERR_INVAL
    # an iteration cap that cannot be met ends the loop with NOCONV
    s2 = gea.Solver3D(g, W.Constants(dt=0.2, cg_maxit=1))
    s2.set_conservative(W.random_flow3(g, c, seed=1, uamp=3.0).fields)
    with pytest.raises(gea.GeaError) as ei:
        s2.step(1)
    assert ei.value.code == gea.GEA_ERR_NOCONV


def test_deterministic_and_multi_step_equals_single_steps(gea):
    """Two runs from the same state agree bit for bit (the reductions sum in
    a fixed order), and n steps in one call equal n calls of one step."""
    g = W.Grid3(40, 24, 16, 4000.0, 2400.0, 1600.0)
    c = W.Constants(dt=0.2, mu=0.5, cs=0.17)
    wl = W.random_flow3(g, c, seed=21, uamp=3.0, thamp=2.0)
    out = []
    for one_by_one in (False, False, True):
        s = gea.Solver3D(g, c)
        s.set_conservative(wl.fields)
        if one_by_one:
            for _ in range(6):
                s.step(1)
        else:
            s.step(6)
        assert s.stats()["steps_done"] == 6
        out.append(s.get_state())
    for k in FIELDS:
        assert np.array_equal(out[0][k], out[1][k]), k
        assert np.array_equal(out[0][k], out[2][k]), k


def test_full_size_les_bubble_properties(gea):
    """The bench's 3D workload at its full size (512 x 512 x 256, 67 M cells,
    Smagorinsky LES, two multigrid levels), where no oracle can follow: two
    steps through the graph driver keep mass to round-off and the centred
    bubble's mirror symmetries in x and y and its x <-> y symmetry."""
    wl = W.get("bubble3d_512x512x256")
    s = gea.Solver3D(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.step(2)
    st = s.stats()
    assert st["status"] == 0 and st["mg_levels"] == 2, st
    f = s.get_state()
    s.close()
    w, u, v = f["w"], f["u"], f["v"]
    sc = np.abs(w).max()
    assert sc > 1e-6
    assert np.abs(w - w[:, :, ::-1]).max() < 1e-8 * sc and np.abs(w - w[:, ::-1, :]).max() < 1e-8 * sc
    assert np.abs(u + u[:, :, ::-1]).max() < 1e-8 * sc and np.abs(v + v[:, ::-1, :]).max() < 1e-8 * sc
    assert np.abs(u - v.transpose(0, 2, 1)).max() < 1e-8 * sc
    m0 = wl.fields["rho"].sum()
    assert abs(f["rho"].sum() - m0) < 1e-12 * m0


def test_diagnostics_on_the_device(gea):
    """theta', mass and total energy of gea3d_get_diag against their
    definitions (Remark 2; Section 2.1's e = cv T + |u|^2/2 + g z) evaluated
    on the state gea3d_get_state returns, after a few steps of the bubble."""
    wl = W.get("bubble3d_64x64x32")
    s = gea.Solver3D(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.step(3)
    th, m, e = s.diagnostics(wl.theta_bar)
    st = s.get_state()
    c, g = wl.const, wl.grid
    th_ref = st["T"] * (c.p0 / st["p"]) ** (c.R / c.cp) - wl.theta_bar[:, None, None]
    assert np.abs(th - th_ref).max() < 1e-11
    assert th.max() > 0.5                     # the bubble's warm anomaly is there
    V = g.dx * g.dy * g.dz
    z = (np.arange(g.nz) + 0.5) * g.dz
    assert abs(m - st["rho"].sum() * V) / m < 1e-13
    K = 0.5 * (st["u"] ** 2 + st["v"] ** 2 + st["w"] ** 2)
    e_ref = (st["rho"] * ((c.cp - c.R) * st["T"] + K + c.g * z[:, None, None])).sum() * V
    assert abs(e - e_ref) / abs(e_ref) < 1e-12
    # theta' needs the background
    assert s.lib.gea3d_get_diag(s.h, None, th.ctypes.data, None, None) == gea.GEA_ERR_INVAL
    s.close()
