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


# ---- Smagorinsky LES in three dimensions ----

def _centres(grid):
    z = (np.arange(grid.nz) + 0.5) * grid.dz
    y = (np.arange(grid.ny) + 0.5) * grid.dy
    x = (np.arange(grid.nx) + 0.5) * grid.dx
    return np.meshgrid(z, y, x, indexing="ij")


def test_strain_exact_on_linear_fields(o3):
    """Central differences are exact on linear velocity fields: |S|^2 =
    2 S_ij S_ij in closed form at interior cells; zero for a rigid rotation."""
    grid = W.Grid3(8, 7, 6, 800.0, 700.0, 600.0)
    q = o3.Oracle3D(grid, W.Constants())
    Z, Y, X = _centres(grid)
    A = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.7], [-0.6, 0.25, -0.35]])   # grad u (rows u, v, w)
    u = A[0, 0] * X + A[0, 1] * Y + A[0, 2] * Z
    v = A[1, 0] * X + A[1, 1] * Y + A[1, 2] * Z
    w = A[2, 0] * X + A[2, 1] * Y + A[2, 2] * Z
    S = 0.5 * (A + A.T)
    expect = np.sqrt(2.0 * np.sum(S * S))
    for (i, j, k) in ((3, 3, 2), (1, 5, 4), (6, 2, 1)):
        assert abs(q.strain_cell(u, v, w, i, j, k) - expect) < 1e-12 * expect
    om = 0.01
    for (i, j, k) in ((3, 3, 2), (2, 4, 3)):
        assert abs(q.strain_cell(-om * Y, om * X, 0 * X, i, j, k)) < 1e-15


def test_variable_diffusion_reduces_to_laplacian(o3):
    """With a constant viscosity field the variable-coefficient sum is mu times
    the Laplacian, walls included, for every wall rule."""
    grid = W.Grid3(6, 5, 4, 600.0, 500.0, 400.0)
    q = o3.Oracle3D(grid, W.Constants())
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 5, 6))
    mu = np.full_like(X, 0.7)
    for bc in range(5):
        for k in range(4):
            for j in range(5):
                for i in range(6):
                    d = q.diffusion_cell(mu, X, bc, i, j, k)
                    lap = q.laplacian_cell(X, bc, i, j, k)
                    assert abs(d - 0.7 * lap) <= 1e-12 * max(1.0, abs(d)), (bc, i, j, k)


def test_variable_diffusion_conservative_and_symmetric(o3):
    """For even ghosts and any positive viscosity field the diffusion sum
    telescopes to zero over the box, is symmetric, and is negative semi-definite."""
    grid = W.Grid3(6, 5, 4, 600.0, 500.0, 400.0)
    q = o3.Oracle3D(grid, W.Constants())
    rng = np.random.default_rng(4)
    mu = 0.5 + rng.random((4, 5, 6))
    X, Y = rng.standard_normal((4, 5, 6)), rng.standard_normal((4, 5, 6))

    def D(F):
        return np.array([[[q.diffusion_cell(mu, F, 0, i, j, k) for i in range(6)] for j in range(5)]
                         for k in range(4)])
    DX, DY = D(X), D(Y)
    scale = np.abs(DX).max()
    assert abs(DX.sum()) < 1e-12 * scale * DX.size
    assert abs(np.sum(Y * DX) - np.sum(X * DY)) < 1e-11 * scale * DX.size
    assert np.sum(X * DX) < 0.0


def test_les_y_invariant_state_follows_the_2d_les_oracle(o3, oracle_mod):
    """An x-z state repeated along y with dy = sqrt(dx dz) (so the 3D filter
    width (dx dy dz)^(1/3) equals the 2D sqrt(dx dz)) follows the 2D LES
    oracle, an independently written and pinned program; and LES changes the
    result (the comparison has teeth)."""
    grid = W.Grid(24, 16, 2400.0, 1600.0)
    c = W.Constants(dt=0.2, mu=0.5, cs=0.17)
    wl = W.random_flow(grid, c, seed=8, uamp=4.0, thamp=2.0)
    ny = 4
    dy = np.sqrt(grid.dx * grid.dz)
    w3 = W.extrude3(wl, ny, ny * dy)
    o = oracle_mod.Oracle(grid, c)
    s2 = o.derive(wl.fields)
    o.step(s2, 5)
    q = o3.Oracle3D(w3.grid, c)
    s3 = q.derive(w3.fields)
    st = q.step(s3, 5)
    assert st["status"] == 0
    for j in range(ny):
        for f in ("rho", "u", "w", "T", "pp"):
            ref = s2[f]
            err = np.abs(s3[f][:, j, :] - ref).max() / np.abs(ref).max()
            assert err < 1e-10, (f, j, err)
    c0 = W.Constants(dt=0.2, mu=0.5)
    q0 = o3.Oracle3D(w3.grid, c0)
    s0 = q0.derive(w3.fields)
    q0.step(s0, 5)
    assert np.abs(s0["u"] - s3["u"]).max() > 1e-6 * np.abs(s3["u"]).max()


def test_les_rest_and_mass(o3):
    grid = W.Grid3(10, 8, 12, 1000.0, 800.0, 1200.0)
    c = W.Constants(dt=0.2, cs=0.17)
    q = o3.Oracle3D(grid, c)
    s = q.derive(W.rising_bubble3(grid, c, amp=0.0).fields)
    q.step(s, 20)
    assert max(np.abs(s[k]).max() for k in ("u", "v", "w")) < 1e-10
    s = q.derive(W.random_flow3(grid, c, seed=6, uamp=3.0).fields)
    m0, _ = q.totals(s)
    st = q.step(s, 10)
    m1, _ = q.totals(s)
    assert st["status"] == 0 and abs(m1 - m0) < 1e-13 * m0
