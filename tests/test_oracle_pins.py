"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics, independent of the oracle's own code:

* closed forms: exactness of the stencils on polynomials and on the discrete
  eigenfunctions of the wall conditions; the Euler tendencies of Section 2.1
  (eqs. mass, mom, ent, with Remark 1's diffusion) evaluated symbolically;
* invariants: discrete hydrostatic rest (eq. mom_split), mass conservation
  (eq. mass / e1_d), mirror and transpose symmetry;
* special cases reducing to library routines: dense LU solves of the
  pressure (Step 3) and transport (Steps 1-2) systems;
* physics: the adiabatic sound speed sqrt(gamma R T) that the ideal-gas
  closure (eq. p) and the enthalpy equation (eq. over_ent) imply;
* the first-order (BDF1, Section 3) temporal part of the energy drift.
"""
import math

import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

BC_EVEN, BC_U, BC_W, BC_H = 0, 1, 2, 3


def make(oracle_mod, grid, **kw):
    return oracle_mod.Oracle(grid, W.Constants(**kw))


# ---------------------------------------------------------------------------
# stencils (Section 3: 4th-order divergence, 2nd-order Laplacian/gradient)
# ---------------------------------------------------------------------------

def test_interp4_exact_on_cubics(oracle_mod):
    """The four-point face value (-1, 7, 7, -1)/12 is the fourth-order
    finite-volume reconstruction: from cell averages of a cubic it returns
    the cubic's point value on the face. With a uniform flux through the
    interior faces the convective term is then phi (P(x_e) - P(x_w)) / V
    exactly, away from the walls."""
    grid = W.Grid(16, 12, 800.0, 300.0)
    o = make(oracle_mod, grid)
    nx, nz, dx, dz = grid.nx, grid.nz, grid.dx, grid.dz
    P = lambda s: 2.0 + 0.3 * s - 1.1e-3 * s ** 2 + 7e-7 * s ** 3
    Q = lambda s: 2.0 * s + 0.15 * s ** 2 - 1.1e-3 / 3 * s ** 3 + 7e-7 / 4 * s ** 4  # Q' = P
    avg = lambda lo, hi: (Q(hi) - Q(lo)) / (hi - lo)
    # x direction
    phix = np.zeros((nz, nx + 1)); phix[:, 1:nx] = 2.5
    phiz = np.zeros((nz + 1, nx))
    xe = (np.arange(nx) + 1.0) * dx
    xw = np.arange(nx) * dx
    X = np.broadcast_to(avg(xw, xe)[None, :], (nz, nx)).copy()
    C = o.convection(phix, phiz, X, BC_EVEN)
    want = 2.5 * (P(xe) - P(xw)) / (dx * dz)
    np.testing.assert_allclose(C[:, 2:nx - 2], np.broadcast_to(want[2:nx - 2], (nz, nx - 4)),
                               rtol=1e-11, atol=1e-11 * abs(want).max())
    # z direction
    phix = np.zeros((nz, nx + 1))
    phiz = np.zeros((nz + 1, nx)); phiz[1:nz, :] = -1.5
    zt = (np.arange(nz) + 1.0) * dz
    zb = np.arange(nz) * dz
    X = np.broadcast_to(avg(zb, zt)[:, None], (nz, nx)).copy()
    C = o.convection(phix, phiz, X, BC_EVEN)
    want = -1.5 * (P(zt) - P(zb)) / (dx * dz)
    np.testing.assert_allclose(C[2:nz - 2, :], np.broadcast_to(want[2:nz - 2, None], (nz - 4, nx)),
                               rtol=1e-11, atol=1e-11 * abs(want).max())


def test_divergence_telescopes(oracle_mod):
    """sum_i V (1/V) sum_j phi_j = 0 on a closed box for any interior fluxes."""
    rng = np.random.default_rng(1)
    grid = W.Grid(13, 9, 1300.0, 450.0)
    o = make(oracle_mod, grid)
    phix = rng.normal(size=(9, 14)); phix[:, 0] = phix[:, -1] = 0
    phiz = rng.normal(size=(10, 13)); phiz[0, :] = phiz[-1, :] = 0
    div = o.convection(phix, phiz, np.ones((9, 13)), BC_EVEN)
    assert abs(div.sum() * grid.dx * grid.dz) <= 1e-13 * np.abs(phix).sum()


def test_laplacian_exact_on_quadratics(oracle_mod):
    grid = W.Grid(11, 7, 550.0, 210.0)
    o = make(oracle_mod, grid)
    X, Z = np.meshgrid(grid.xc(), grid.zc())
    f = 3e-4 * X ** 2 - 5e-4 * Z ** 2 + 2e-4 * X * Z + 0.7 * X - 0.2 * Z + 4.0
    L = o.laplacian(f, BC_EVEN)
    np.testing.assert_allclose(L[1:-1, 1:-1], 2 * 3e-4 - 2 * 5e-4, rtol=1e-9)


@pytest.mark.parametrize("bc", [BC_EVEN, BC_U, BC_W, BC_H])
def test_wall_conditions_discrete_eigenfunctions(oracle_mod, bc):
    """Each wall condition is exact for its discrete eigenfunction: cos(m pi x/L)
    (zero gradient, even ghost) and sin(m pi x/L) (zero value, odd ghost) are
    eigenvectors of the cell-centred Laplacian with eigenvalue
    -(2/dx)^2 sin^2(k dx/2); h = -g z + cos(...) has dh/dz = -g on both
    horizontal walls."""
    grid = W.Grid(10, 8, 700.0, 400.0)
    o = make(oracle_mod, grid)
    X, Z = np.meshgrid(grid.xc(), grid.zc())
    kx, kz = 3 * np.pi / grid.lx, 2 * np.pi / grid.lz
    lx = -(2 / grid.dx) ** 2 * np.sin(kx * grid.dx / 2) ** 2
    lz = -(2 / grid.dz) ** 2 * np.sin(kz * grid.dz / 2) ** 2
    fx_even, fx_odd = np.cos(kx * X), np.sin(kx * X)
    fz_even, fz_odd = np.cos(kz * Z), np.sin(kz * Z)
    if bc == BC_EVEN:
        f = fx_even * fz_even; want = (lx + lz) * f
    elif bc == BC_U:       # odd in x, even in z
        f = fx_odd * fz_even; want = (lx + lz) * f
    elif bc == BC_W:       # even in x, odd in z
        f = fx_even * fz_odd; want = (lx + lz) * f
    else:                  # h: even in x, dh/dz = -g on the horizontal walls
        g = 9.81
        f = fx_even * fz_even - g * Z + 3e5; want = (lx + lz) * fx_even * fz_even
    L = o.laplacian(f, bc)
    np.testing.assert_allclose(L, want, atol=1e-11 * np.abs(want).max())


# ---------------------------------------------------------------------------
# linear systems vs dense LU (library routine)
# ---------------------------------------------------------------------------

def _tiny_step_dump(oracle_mod, nx=12, nz=8):
    grid = W.Grid(nx, nz, 1200.0, 640.0)
    c = W.Constants(dt=0.5)
    wl = W.random_flow(grid, c, seed=3, uamp=4.0)
    o = oracle_mod.Oracle(grid, c)
    s = o.derive(wl.fields)
    phix, phiz = s["phix"].copy(), s["phiz"].copy()
    _, d = o.step(s, 1, dump=True)
    return o, grid, c, d, phix, phiz


def test_pressure_matrix_symmetric_spd_and_cg_matches_lu(oracle_mod):
    o, grid, c, d, _, _ = _tiny_step_dump(oracle_mod)
    n = grid.cells
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        A[:, j] = o.helmholtz_apply(d["psi"], d["Dx"], d["Dz"], e.reshape(grid.nz, grid.nx)).ravel()
    assert np.array_equal(A, A.T)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    np.testing.assert_allclose(np.diag(A) - off, d["psi"].ravel() / c.dt, rtol=1e-9)
    assert np.linalg.eigvalsh(A).min() > 0
    b = d["b"].ravel()
    x_lu = np.linalg.solve(A, b)
    x_cg, it, rr = o.pcg(d["psi"], d["Dx"], d["Dz"], d["b"], np.zeros((grid.nz, grid.nx)))
    assert it > 0
    np.testing.assert_allclose(x_cg.ravel(), x_lu, rtol=1e-12)


@pytest.mark.parametrize("bc", [BC_U, BC_W, BC_H])
def test_transport_jacobi_matches_lu(oracle_mod, bc):
    """The implicit predictors (eq. step2_sd first line, eq. step3_sd) are
    affine in the unknown through the ghost layer; Jacobi must land on the
    dense solution."""
    o, grid, c, d, phix, phiz = _tiny_step_dump(oracle_mod)
    n = grid.cells
    nu = 25.0   # strong diffusion so the wall conditions matter
    shp = (grid.nz, grid.nx)
    c0 = o.transport_apply(d["rho1"], phix, phiz, nu, bc, np.zeros(shp)).ravel()
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        M[:, j] = o.transport_apply(d["rho1"], phix, phiz, nu, bc, e.reshape(shp)).ravel() - c0
    rng = np.random.default_rng(7)
    b = rng.normal(size=n) * 10 + (3e5 if bc == BC_H else 0.0)
    x_lu = np.linalg.solve(M, b - c0)
    x_j, it = o.transport_solve(d["rho1"], phix, phiz, nu, bc, b.reshape(shp), np.zeros(shp))
    assert it > 0
    np.testing.assert_allclose(x_j.ravel(), x_lu, rtol=1e-12, atol=1e-12 * np.abs(x_lu).max())


# ---------------------------------------------------------------------------
# invariants of whole steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mu", [0.15, 0.0])
def test_rest_atmosphere_stays_at_rest(oracle_mod, mu):
    """The discretely balanced neutral column (eq. mom_split with the split
    p = p' - rho g z) must not move. Round-off of p' ~ 1e5 Pa (ulp 1.5e-11 Pa)
    drives accelerations ~1e-13 m/s^2; after 100 steps (10 s) velocities stay
    below 1e-10 m/s, against 0.065 m/s gained by the 2 K bubble every step."""
    wl = W.rest_atmosphere(W.Grid(160, 80, 20000.0, 10000.0), W.Constants(dt=0.1, mu=mu))
    o = oracle_mod.Oracle(wl.grid, wl.const)
    s = o.derive(wl.fields)
    p0 = s["pp"].copy()
    st, _ = o.step(s, 100)
    assert st["status"] == 0
    th, _, _ = o.diagnostics(s, wl.theta_bar)
    assert np.abs(s["u"]).max() < 1e-10
    assert np.abs(s["w"]).max() < 1e-10
    assert np.abs(th).max() < 1e-10
    assert np.abs(s["pp"] - p0).max() / np.abs(p0).max() < 1e-12


def test_stratified_rest_inviscid(oracle_mod):
    """Any discretely balanced column is steady without diffusion (mu = 0):
    stable stratification, theta rising 3 K/km."""
    wl = W.stratified_rest(W.Grid(40, 60, 4000.0, 9000.0), W.Constants(dt=0.2, mu=0.0))
    o = oracle_mod.Oracle(wl.grid, wl.const)
    s = o.derive(wl.fields)
    T0 = s["T"].copy()
    o.step(s, 100)
    assert np.abs(s["u"]).max() < 1e-10
    assert np.abs(s["w"]).max() < 1e-10
    assert np.abs(s["T"] - T0).max() < 1e-10


def test_mass_conservation_and_continuity(oracle_mod):
    wl = W.get("bubble160x80")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    s = o.derive(wl.fields)
    _, m0, _ = o.diagnostics(s, wl.theta_bar)
    for _ in range(20):
        rho_old = s["rho"].copy()
        st, _ = o.step(s, 5)
        assert st["status"] == 0
    # continuity with the stored flux phi^{n+1} over the last step
    rho_old = s["rho"].copy()
    o.step(s, 1)
    res = o.continuity_residual(rho_old, s)
    assert np.abs(res).max() < 1e-12 * s["rho"].max() / wl.const.dt
    _, m1, _ = o.diagnostics(s, wl.theta_bar)
    assert abs(m1 - m0) / m0 < 1e-13
    # and the bubble did rise: upward flow of order g theta'/theta t
    assert s["w"].max() > 0.3


def test_mirror_symmetry(oracle_mod):
    """A bubble centred at x = L/2 stays mirror symmetric: u odd, w and T even."""
    wl = W.get("bubble160x80")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    s = o.derive(wl.fields)
    o.step(s, 60)
    u, w, T = s["u"], s["w"], s["T"]
    assert np.abs(u + u[:, ::-1]).max() <= 1e-10 * np.abs(u).max()
    assert np.abs(w - w[:, ::-1]).max() <= 1e-10 * np.abs(w).max()
    assert np.abs(T - T[:, ::-1]).max() <= 1e-12 * T.max()


def test_transpose_symmetry_without_gravity(oracle_mod):
    """With g = 0 on a square box the scheme treats x and z alike: a state
    invariant under (x, z, u, w) -> (z, x, w, u) stays so."""
    c = W.Constants(g=0.0, mu=2.0, dt=0.2)
    wl = W.transpose_symmetric(24, 1200.0, c)
    o = oracle_mod.Oracle(wl.grid, c)
    s = o.derive(wl.fields)
    o.step(s, 20)
    u, w = s["u"], s["w"]
    assert np.abs(u - w.T).max() <= 1e-11 * np.abs(u).max()
    assert np.abs(s["T"] - s["T"].T).max() <= 1e-12 * s["T"].max()
    assert np.abs(s["phix"] - s["phiz"].T).max() <= 1e-11 * np.abs(s["phix"]).max()


# ---------------------------------------------------------------------------
# consistency with the continuous equations (closed forms)
# ---------------------------------------------------------------------------

def _analytic_state():
    sp = pytest.importorskip("sympy")
    Lx, Lz = 1000.0, 600.0
    R, cp, g, p0 = 287.0, 1004.0, 9.81, 1e5
    cv = cp - R
    gam = cp / cv
    x, z, mu, Pr = sp.symbols("x z mu Pr", real=True)
    X, Z = sp.pi * x / Lx, sp.pi * z / Lz
    Tb = 300.0 - g * z / cp
    T = Tb + 3.0 * sp.cos(X) * sp.cos(Z)
    p = p0 * (Tb / 300.0) ** (cp / R) * (1 + 2e-3 * sp.cos(2 * X) * sp.cos(Z))
    rho = p / (R * T)
    u = 8.0 * sp.sin(X) * sp.cos(Z)
    w = 5.0 * sp.cos(X) * sp.sin(Z)
    h = cp * T
    e = cv * T + (u * u + w * w) / 2 + g * z
    lap = lambda f: sp.diff(f, x, 2) + sp.diff(f, z, 2)
    div = lambda fx, fz: sp.diff(fx, x) + sp.diff(fz, z)
    # Section 2.1, eqs. (mass), (mom) with Remark 1's mu Lap u, and the total
    # energy form of eq. (ent_LES): d(rho e)/dt = -div((rho e + p) u) + mu/Pr Lap h
    ex = {
        "rho": -div(rho * u, rho * w),
        "rhou": -div(rho * u * u, rho * u * w) - sp.diff(p, x) + mu * lap(u),
        "rhow": -div(rho * w * u, rho * w * w) - sp.diff(p, z) - rho * g + mu * lap(w),
        "rhoe": -div((rho * e + p) * u, (rho * e + p) * w) + mu / Pr * lap(h),
    }
    # dp/dt from p = rho R T, continuity and the enthalpy equation
    Q = mu / Pr * lap(h) - mu * (u * lap(u) + w * lap(w))
    dp = -(u * sp.diff(p, x) + w * sp.diff(p, z)) - gam * p * div(u, w) + R / cv * Q
    args = (x, z, mu, Pr)
    f = {k: sp.lambdify(args, v, "numpy") for k, v in
         dict(rho=rho, u=u, w=w, T=T, dp=dp, **{"d" + k: v for k, v in ex.items()}).items()}
    return f, (Lx, Lz, R, cp, g, p0)


def _tendency(oracle_mod, f, consts, m, mu):
    Lx, Lz, R, cp, g, p0 = consts
    grid = W.Grid(16 * m, 16 * m, Lx, Lz)
    dt = 0.02 / m ** 2
    c = W.Constants(R=R, cp=cp, g=g, p0=p0, mu=mu, Pr=1.0, dt=dt)
    XX, ZZ = np.meshgrid(grid.xc(), grid.zc())
    ev = lambda k: np.broadcast_to(np.asarray(f[k](XX, ZZ, mu, 1.0), dtype=float), XX.shape).copy()
    fields = W.conservative_from_primitive(grid, c, ev("rho"), ev("u"), ev("w"), ev("T"))
    o = oracle_mod.Oracle(grid, c)
    s = o.derive(fields)
    s.a["pold"][:] = s["p"] - dt * ev("dp")       # p^{n-1} consistent with dp/dt
    c0 = {k: v.copy() for k, v in s.conservative(g, c.cv, grid.dz).items()}
    st, _ = o.step(s, 1)
    assert st["status"] == 0
    c1 = s.conservative(g, c.cv, grid.dz)
    disc = {k: (c1[k] - c0[k]) / dt for k in c0}
    exact = {k: ev("d" + k) for k in c0}
    return disc, exact


def test_step_tendencies_converge_to_euler_equations(oracle_mod):
    """One short step from a smooth state reproduces the tendencies of the
    compressible Euler equations, at second order in the interior (dt ~ dx^2).
    A dropped term or a wrong sign leaves an O(1) error that does not shrink."""
    f, consts = _analytic_state()
    errs = []
    for m in (2, 4, 8):
        disc, exact = _tendency(oracle_mod, f, consts, m, 0.0)
        inner = (slice(3, -3), slice(3, -3))
        errs.append({k: np.abs(disc[k] - exact[k])[inner].max() / np.abs(exact[k]).max()
                     for k in exact})
    for k in errs[0]:
        assert errs[1][k] / errs[2][k] > 3.3, (k, errs)
        assert errs[0][k] / errs[1][k] > 2.8, (k, errs)
        assert errs[2][k] < 0.02, (k, errs)


def test_diffusion_tendencies(oracle_mod):
    """The difference between runs with mu and without is Remark 1's
    mu Lap u in momentum and (mu/Pr) Lap h in energy."""
    f, consts = _analytic_state()
    mu = 200.0
    errs = []
    for m in (2, 4, 8):
        d1, e1 = _tendency(oracle_mod, f, consts, m, mu)
        d0, e0 = _tendency(oracle_mod, f, consts, m, 0.0)
        inner = (slice(3, -3), slice(3, -3))
        errs.append({k: np.abs((d1[k] - d0[k]) - (e1[k] - e0[k]))[inner].max()
                     / np.abs(e1[k] - e0[k]).max() for k in ("rhou", "rhow", "rhoe")})
    for k in errs[0]:
        assert errs[2][k] < errs[1][k] < errs[0][k], (k, errs)
        assert errs[2][k] < 0.05, (k, errs)


def test_acoustic_frequency_is_adiabatic(oracle_mod):
    """With g = 0 and mu = 0 a standing wave cos(pi x / L) oscillates at
    omega = c_s k_d, c_s = sqrt(gamma R T) (gamma = cp/cv), k_d the discrete
    wavenumber (2/dx) sin(k dx/2) of the compact Laplacian; the isothermal
    speed sqrt(R T) would be 18% slower. BDF1 damping is first order in dt."""
    res = {}
    for dt in (0.02, 0.01):
        c = W.Constants(g=0.0, mu=0.0, dt=dt)
        grid = W.Grid(64, 4, 1000.0, 100.0)
        wl = W.acoustic_mode(grid, c, amp=1e-5)
        o = oracle_mod.Oracle(grid, c)
        s = o.derive(wl.fields)
        k = np.pi / grid.lx
        om = math.sqrt(c.cp / c.cv * c.R * 300.0) * 2 / grid.dx * math.sin(k * grid.dx / 2)
        period = 2 * np.pi / om
        nsteps = int(2.2 * period / dt)
        sig = np.empty(nsteps)
        for n in range(nsteps):
            o.step(s, 1)
            sig[n] = s["p"][0, 0] - s["p"][0, -1]
        t = (np.arange(nsteps) + 1) * dt
        zc = [t[i] - sig[i] * dt / (sig[i + 1] - sig[i])
              for i in range(nsteps - 1) if sig[i] * sig[i + 1] < 0]
        om_meas = 2 * np.pi / (2 * np.mean(np.diff(zc)))
        half = int(period / dt / 2)
        amp0 = np.abs(sig[:half]).max()
        amp3 = np.abs(sig[3 * half:4 * half]).max()
        res[dt] = (om_meas / om, 1 - amp3 / amp0)
    for dt, (ratio, loss) in res.items():
        assert abs(ratio - 1) < 2e-3, res
        assert loss > 0, res
    assert 1.7 < res[0.02][1] / res[0.01][1] < 2.3, res


def test_energy_drift_first_order_in_dt(oracle_mod):
    """The enthalpy form with explicit K, lagged dp/dt and rho g w does not
    conserve total energy exactly; its temporal part must be first order
    (BDF1): successive differences of the drift at dt, dt/2, dt/4 shrink by 2."""
    grid = W.Grid(80, 40, 20000.0, 10000.0)
    drift = []
    for dt in (0.4, 0.2, 0.1):
        c = W.Constants(dt=dt)
        wl = W.rising_bubble(grid, c, 300.0, "cosine", 2.0, 2000.0, 10000.0, 2000.0)
        o = oracle_mod.Oracle(grid, c)
        s = o.derive(wl.fields)
        _, _, e0 = o.diagnostics(s, wl.theta_bar)
        o.step(s, int(round(20.0 / dt)))
        _, _, e1 = o.diagnostics(s, wl.theta_bar)
        drift.append((e1 - e0) / e0)
    r = (drift[0] - drift[1]) / (drift[1] - drift[2])
    assert 1.7 < r < 2.6, (drift, r)
    assert abs(drift[2]) < 1e-7


# ---------------------------------------------------------------------------
# set-up and diagnostics
# ---------------------------------------------------------------------------

def test_derive_roundtrip(oracle_mod):
    grid = W.Grid(20, 14, 2000.0, 1400.0)
    c = W.Constants()
    wl = W.random_flow(grid, c, seed=5, uamp=6.0, thamp=3.0)
    o = oracle_mod.Oracle(grid, c)
    s = o.derive(wl.fields)
    back = s.conservative(c.g, c.cv, grid.dz)
    for k in back:
        np.testing.assert_allclose(back[k], wl.fields[k], rtol=1e-13,
                                   atol=1e-13 * np.abs(wl.fields[k]).max())
    np.testing.assert_allclose(s["p"], s["rho"] * c.R * s["T"], rtol=1e-15)
    np.testing.assert_allclose(s["h"], c.cp * s["T"], rtol=1e-15)


def test_theta_prime_of_the_bubble(oracle_mod):
    """At t = 0 the bubble sits at background pressure with
    T = T_bar (theta0 + theta'_0) / theta0, so theta' = theta_bar theta'_0 / theta0
    (eqs. theta, theta_split); the peak of the 2 K bubble is near 2 K."""
    wl = W.get("bubble160x80")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    s = o.derive(wl.fields)
    th, _, _ = o.diagnostics(s, wl.theta_bar)
    th0 = W.bubble_perturbation(wl.grid, "cosine", 2.0, 2000.0, 10000.0, 2000.0)
    np.testing.assert_allclose(th, wl.theta_bar[:, None] * th0 / 300.0, atol=1e-10)
    assert 1.98 < th.max() < 2.0


def test_lagged_kinetic_energy_reading(oracle_mod):
    """The literal reading of eq. step3_sd (reading flag 1): b~_e carries
    rho^n K^{n-1} instead of rho^n K^n, with K^{-1} := K^0.
    (a) The first step is the default reading's, bit for bit.
    (b) On a later step the enthalpy right-hand side differs from the
        default's by exactly rho^n (K^{n-1} - K^n) / dt (sign and factor of
        the one changed term), all else equal.
    (c) The reading keeps mass conservation and the rest atmosphere."""
    import dataclasses
    grid = W.Grid(24, 16, 24 * 40.0, 16 * 30.0)
    c0 = W.Constants(dt=0.2, mu=1.5)
    c1 = dataclasses.replace(c0, reading_flags=oracle_mod.READING_K_LAGGED)
    wl = W.random_flow(grid, c0, seed=12, uamp=4.0, thamp=2.0)
    o0, o1 = oracle_mod.Oracle(grid, c0), oracle_mod.Oracle(grid, c1)
    a, b = o0.derive(wl.fields), o1.derive(wl.fields)
    assert np.array_equal(a["Kold"], 0.5 * (a["u"] ** 2 + a["w"] ** 2))
    o0.step(a, 1)
    o1.step(b, 1)
    for k in oracle_mod.oracle.STATE_FIELDS:
        assert np.array_equal(a[k], b[k]), k
    # (b): from the same state after one step, K^{n-1} != K^n
    s1, s0 = b.copy(), b.copy()
    Kn = 0.5 * (b["u"] ** 2 + b["w"] ** 2)
    assert np.abs(b["Kold"] - Kn).max() > 1e-3
    _, d1 = o1.step(s1, 1, dump=True)
    _, d0 = o0.step(s0, 1, dump=True)
    expect = b["rho"] * (b["Kold"] - Kn) / c0.dt
    assert np.abs((d1["bh"] - d0["bh"]) - expect).max() <= 1e-14 * np.abs(d0["bh"]).max()
    assert np.abs(s1["u"] - s0["u"]).max() > 0.0   # the reading changes the flow
    # (c)
    _, m0, _ = o1.diagnostics(b, np.full(grid.nz, 300.0))
    o1.step(b, 10)
    _, m1, _ = o1.diagnostics(b, np.full(grid.nz, 300.0))
    assert abs(m1 - m0) / m0 < 1e-13
    rest = W.rest_atmosphere(W.Grid(32, 16, 3200.0, 1600.0), c1)
    orr = oracle_mod.Oracle(rest.grid, c1)
    sr = orr.derive(rest.fields)
    orr.step(sr, 20)
    assert np.abs(sr["u"]).max() < 1e-10 and np.abs(sr["w"]).max() < 1e-10
