"""Pins of the three-dimensional oracle (oracle/gea_oracle3d.c) to things
other than itself: the two-dimensional oracle on y-invariant states (an
independent program whose pins are in test_oracle_pins.py), closed forms,
exact symmetries, the hydrostatic rest state and mass conservation.
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3d
    return oracle3d


def test_y_invariant_state_follows_the_2d_oracle(o3, oracle_mod):
    """An x-z state repeated along y stays y-invariant with v = 0, and its
    3D step is the 2D step (the 3D CG sees the 2D system repeated ny times:
    same iterates, sums in another order)."""
    grid = W.Grid(24, 16, 2400.0, 1600.0)
    c = W.Constants(dt=0.2, mu=1.5)
    wl = W.random_flow(grid, c, seed=7, uamp=3.0, thamp=2.0)
    w3 = W.extrude3(wl, 4, 400.0)
    o = oracle_mod.Oracle(grid, c)
    s2 = o.derive(wl.fields)
    o.step(s2, 5)
    q = o3.Oracle3D(w3.grid, c)
    s3 = q.derive(w3.fields)
    st = q.step(s3, 5)
    assert st["status"] == 0
    assert np.abs(s3["v"]).max() < 1e-12 * max(1.0, np.abs(s3["u"]).max())
    for j in range(4):
        for f in ("rho", "u", "w", "T", "pp", "p"):
            ref = s2[f]
            err = np.abs(s3[f][:, j, :] - ref).max() / np.abs(ref).max()
            assert err < 1e-10, (f, j, err)
        assert np.abs(s3["phix"][:, j, :] - s2["phix"] * 100.0).max() < 1e-10 * np.abs(s2["phix"] * 100.0).max()


def test_x_y_transpose_symmetry(o3):
    """Exchanging x and y (and u and v) on a square-based box commutes with
    the step."""
    grid = W.Grid3(12, 12, 8, 1200.0, 1200.0, 800.0)
    c = W.Constants(dt=0.2, mu=1.0)
    wl = W.random_flow3(grid, c, seed=3, uamp=2.0, thamp=1.0)
    f = wl.fields
    ft = {"rho": f["rho"].transpose(0, 2, 1).copy(), "rhou": f["rhov"].transpose(0, 2, 1).copy(),
          "rhov": f["rhou"].transpose(0, 2, 1).copy(), "rhow": f["rhow"].transpose(0, 2, 1).copy(),
          "rhoe": f["rhoe"].transpose(0, 2, 1).copy()}
    q = o3.Oracle3D(grid, c)
    a = q.derive(f)
    b = q.derive(ft)
    q.step(a, 3)
    q.step(b, 3)
    scale = max(np.abs(a["u"]).max(), np.abs(a["v"]).max())
    assert np.abs(a["u"] - b["v"].transpose(0, 2, 1)).max() < 1e-10 * scale
    assert np.abs(a["w"] - b["w"].transpose(0, 2, 1)).max() < 1e-10 * scale
    assert np.abs(a["T"] - b["T"].transpose(0, 2, 1)).max() < 1e-10 * np.abs(a["T"]).max()


def test_rest_and_mass(o3):
    grid = W.Grid3(10, 8, 12, 1000.0, 800.0, 1200.0)
    c = W.Constants(dt=0.2)
    rest = W.rising_bubble3(grid, c, amp=0.0)
    q = o3.Oracle3D(grid, c)
    s = q.derive(rest.fields)
    q.step(s, 20)
    assert max(np.abs(s[k]).max() for k in ("u", "v", "w")) < 1e-10
    wl = W.random_flow3(grid, c, seed=5, uamp=2.0)
    s = q.derive(wl.fields)
    m0, _ = q.totals(s)
    st = q.step(s, 10)
    m1, _ = q.totals(s)
    assert st["status"] == 0 and abs(m1 - m0) < 1e-13 * m0


def test_bubble_mirror_symmetry(o3):
    grid = W.Grid3(16, 16, 12, 4000.0, 4000.0, 3000.0)
    c = W.Constants(dt=0.5)
    wl = W.rising_bubble3(grid, c, amp=2.0, rc=1000.0, xc=2000.0, yc=2000.0, zc=1000.0)
    q = o3.Oracle3D(grid, c)
    s = q.derive(wl.fields)
    q.step(s, 5)
    w, u, v = s["w"], s["u"], s["v"]
    sc = max(np.abs(w).max(), 1e-30)
    assert np.abs(w - w[:, :, ::-1]).max() < 1e-9 * sc and np.abs(w - w[:, ::-1, :]).max() < 1e-9 * sc
    assert np.abs(u + u[:, :, ::-1]).max() < 1e-9 * sc and np.abs(v + v[:, ::-1, :]).max() < 1e-9 * sc
    assert np.abs(w).max() > 0


def test_laplacian_exact_on_quadratics(o3):
    grid = W.Grid3(8, 7, 6, 800.0, 700.0, 600.0)
    q = o3.Oracle3D(grid, W.Constants())
    z, y, x = np.meshgrid((np.arange(6) + 0.5) * 100.0, (np.arange(7) + 0.5) * 100.0,
                          (np.arange(8) + 0.5) * 100.0, indexing="ij")
    X = 0.3 * x * x - 0.2 * y * y + 0.7 * z * z + x * y - 4.0 * z
    for (i, j, k) in ((3, 3, 2), (1, 5, 4), (6, 2, 1)):
        assert abs(q.laplacian_cell(X, 0, i, j, k) - 2 * (0.3 - 0.2 + 0.7)) < 1e-10
