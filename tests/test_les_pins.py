"""Pins of the oracle's Smagorinsky LES (the eddy viscosity
mu_t = rho (cs Delta)^2 |S| with Delta = sqrt(dx dz) and the
variable-coefficient diffusion it enters): closed forms on linear fields,
exact reductions to the constant-viscosity operator, conservation and
symmetry of the discrete operator, second-order convergence to
div(mu grad X), and the physical effect (added dissipation).
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

BC_EVEN, BC_U, BC_W = 0, 1, 2


def cell_xz(grid):
    x = (np.arange(grid.nx) + 0.5) * grid.dx
    z = (np.arange(grid.nz) + 0.5) * grid.dz
    return np.meshgrid(x, z)          # X[k, i], Z[k, i]


def test_strain_rate_of_linear_fields(oracle_mod):
    grid = W.Grid(12, 10, 1200.0, 800.0)
    o = oracle_mod.Oracle(grid, W.Constants(cs=0.17))
    X, Z = cell_xz(grid)
    a, b, c, d = 0.3, -0.7, 0.2, 0.45
    u, w = a * X + b * Z, c * X + d * Z
    S = o.strain(u, w)
    ref = np.sqrt(2 * a * a + 2 * d * d + (b + c) ** 2)
    assert np.allclose(S[1:-1, 1:-1], ref, rtol=1e-12)
    # a rigid rotation has no strain
    assert np.allclose(o.strain(-Z + 400.0, X - 600.0)[1:-1, 1:-1], 0.0, atol=1e-12)


def test_smagorinsky_viscosity(oracle_mod):
    grid = W.Grid(12, 10, 1200.0, 800.0)
    cs, mu = 0.17, 0.3
    o = oracle_mod.Oracle(grid, W.Constants(cs=cs, mu=mu))
    X, Z = cell_xz(grid)
    rho = 1.0 + 0.1 * np.sin(X / 300.0)
    u, w = 0.01 * Z, np.zeros_like(X)
    m = o.smagorinsky(rho, u, w)
    ref = mu + rho * cs ** 2 * grid.dx * grid.dz * 0.01
    assert np.allclose(m[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=1e-12)


def test_diffusion_reduces_to_constant_viscosity(oracle_mod):
    grid = W.Grid(16, 12, 1600.0, 900.0)
    o = oracle_mod.Oracle(grid, W.Constants())
    rng = np.random.default_rng(3)
    Xf = rng.standard_normal((12, 16))
    for bc in (BC_EVEN, BC_U, BC_W):
        d = o.diffusion(np.full((12, 16), 0.7), Xf, bc)
        assert np.allclose(d, 0.7 * o.laplacian(Xf, bc), rtol=1e-12, atol=1e-14)


def test_diffusion_conservative_and_symmetric(oracle_mod):
    grid = W.Grid(16, 12, 1600.0, 900.0)
    o = oracle_mod.Oracle(grid, W.Constants())
    rng = np.random.default_rng(4)
    mu = 0.5 + rng.random((12, 16))
    A, B = rng.standard_normal((12, 16)), rng.standard_normal((12, 16))
    V = grid.dx * grid.dz
    dA = o.diffusion(mu, A, BC_EVEN)
    # zero-gradient walls: the face sums telescope to zero
    assert abs(np.sum(dA) * V) < 1e-12 * np.sum(np.abs(dA)) * V
    # symmetric (and negative semi-definite) bilinear form
    assert abs(np.sum(B * dA) - np.sum(A * o.diffusion(mu, B, BC_EVEN))) < 1e-12 * np.sum(np.abs(B * dA))
    assert np.sum(A * dA) < 0.0


def test_diffusion_converges_to_div_mu_grad():
    """(1/V) sum mu_f (grad X)_f A_f -> div(mu grad X) at second order for
    mu = 1 + 0.5 cos(pi x/L) cos(pi z/H), X = cos(2 pi x/L) cos(pi z/H)
    (both with zero normal derivative on the walls, BC_EVEN)."""
    import oracle as om
    L, H = 1000.0, 1000.0
    errs = []
    for n in (16, 32, 64):
        grid = W.Grid(n, n, L, H)
        o = om.Oracle(grid, W.Constants())
        X, Z = cell_xz(grid)
        kx, kz = np.pi / L, np.pi / H
        mu = 1.0 + 0.5 * np.cos(kx * X) * np.cos(kz * Z)
        f = np.cos(2 * kx * X) * np.cos(kz * Z)
        mux = -0.5 * kx * np.sin(kx * X) * np.cos(kz * Z)
        muz = -0.5 * kz * np.cos(kx * X) * np.sin(kz * Z)
        fx = -2 * kx * np.sin(2 * kx * X) * np.cos(kz * Z)
        fz = -kz * np.cos(2 * kx * X) * np.sin(kz * Z)
        lap = -(4 * kx * kx + kz * kz) * f
        ref = mux * fx + muz * fz + mu * lap
        errs.append(np.abs(o.diffusion(mu, f, BC_EVEN) - ref).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def test_les_step_at_rest_and_mass(oracle_mod):
    """At rest |S| = 0 and mu_eff = mu: the LES step keeps a hydrostatic
    atmosphere at rest and equals the constant-viscosity step to
    rounding; mass is conserved."""
    grid = W.Grid(40, 20, 4000.0, 2000.0)
    c0 = W.Constants(dt=0.2)
    c1 = W.Constants(dt=0.2, cs=0.17)
    wl = W.rest_atmosphere(grid, c0)
    outs = []
    for c in (c0, c1):
        o = oracle_mod.Oracle(grid, c)
        s = o.derive(wl.fields)
        o.step(s, 20)
        outs.append(s)
    assert np.abs(outs[1]["u"]).max() < 1e-10 and np.abs(outs[1]["w"]).max() < 1e-10
    assert np.abs(outs[1]["T"] - outs[0]["T"]).max() < 1e-10
    # mass with a moving state
    wl2 = W.random_flow(grid, c1, seed=9, uamp=3.0, thamp=1.0)
    o = oracle_mod.Oracle(grid, c1)
    s = o.derive(wl2.fields)
    m0 = np.sum(s["rho"])
    o.step(s, 10)
    assert abs(np.sum(s["rho"]) - m0) < 1e-13 * m0


def test_les_adds_dissipation(oracle_mod):
    """A shear flow loses more kinetic energy with the eddy viscosity than
    with the constant viscosity alone."""
    grid = W.Grid(48, 32, 960.0, 640.0)
    ke = []
    for cs in (0.0, 0.17):
        c = W.Constants(dt=0.2, mu=0.05, cs=cs)
        wl = W.random_flow(grid, c, seed=21, uamp=4.0, thamp=0.0)
        o = oracle_mod.Oracle(grid, c)
        s = o.derive(wl.fields)
        o.step(s, 20)
        ke.append(np.sum(s["rho"] * (s["u"] ** 2 + s["w"] ** 2)))
    assert ke[1] < ke[0] * (1 - 1e-4), ke
