"""Seeded synthetic inputs for the GEA pressure-based Euler solver.

This module only produces initial states (and the run parameters that go with
them); it holds none of the time-step arithmetic. Both the FP64 CPU oracle and
the CUDA path are fed from here, so a parity test compares the two on the
same bytes.

Set-ups follow Section 4 of Girfoglio, Quaini & Rozza (arXiv 2303.10499):

* rising thermal bubbles in a neutral atmosphere, eqs. (rho_wb), (dcEqn1)
  for the smooth cosine bubble and (dcEqn2) for the non-smooth (step) one;
* theta = T / pi, pi = (p/p0)^(R/cp), Remark 2, eq. (theta).

The background column is built so that the discrete solver sees it in exact
balance: T_bar(z) is the neutral profile theta0 - g z / cp sampled at cell
centres, and the density follows the trapezoidal hydrostatic recursion

    rho_{k+1} (R T_{k+1} + g dz/2) = rho_k (R T_k - g dz/2),

i.e. p_{k+1} - p_k = -g dz (rho_k + rho_{k+1}) / 2 with p = rho R T. The bubble
perturbs temperature at fixed background pressure, as the paper does when it
evaluates rho^0 from p with theta^0 (eq. rho_wb).

Everything returned is float64, C-contiguous, cell fields of shape (nz, nx)
with x fastest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Dict, Optional

import numpy as np


@dataclasses.dataclass
class Grid:
    nx: int
    nz: int
    lx: float
    lz: float

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dz(self) -> float:
        return self.lz / self.nz

    @property
    def cells(self) -> int:
        return self.nx * self.nz

    def xc(self) -> np.ndarray:
        return (np.arange(self.nx, dtype=np.float64) + 0.5) * self.dx

    def zc(self) -> np.ndarray:
        return (np.arange(self.nz, dtype=np.float64) + 0.5) * self.dz


@dataclasses.dataclass
class Constants:
    """Physical constants and solver settings of one run.

    mu is the constant (dynamic) artificial viscosity of Remark 1; Pr the
    Prandtl number; n_corr the number of PISO correctors. The solver
    tolerances are relative 2-norm residuals (||r|| <= rtol ||b||). The
    defaults drive every solve to round-off: the pressure right-hand side is
    dominated by the hydrostatic rho^n/dt part, so a looser pressure
    tolerance shows up directly in the velocities."""
    R: float = 287.0
    cp: float = 1004.0
    g: float = 9.81
    p0: float = 1.0e5
    mu: float = 0.15
    Pr: float = 1.0
    dt: float = 0.1
    n_corr: int = 2
    jac_rtol: float = 1e-14
    jac_maxit: int = 200
    cg_rtol: float = 1e-17
    cg_maxit: int = 400
    cs: float = 0.0        # Smagorinsky constant (0: constant viscosity only)
    reading_flags: int = 0  # 1: the literal K^{n-1} of eq. step3_sd (default K^n)

    @property
    def cv(self) -> float:
        return self.cp - self.R


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    const: Constants
    fields: Dict[str, np.ndarray]      # rho, rhou, rhow, rhoe (conservative)
    theta_bar: np.ndarray              # discrete background theta per row, shape (nz,)
    steps: int = 100


def hydrostatic_background(grid: Grid, const: Constants, theta0: float,
                           T_profile=None):
    """Discretely balanced background column at cell centres: neutral
    (T = theta0 - g z / cp) unless T_profile(z) gives another temperature.

    Returns (T_bar, rho_bar, p_bar, theta_bar), each of shape (nz,)."""
    z = grid.zc()
    R, cp, g, p0 = const.R, const.cp, const.g, const.p0
    Tb = theta0 - g * z / cp if T_profile is None else np.asarray(T_profile(z), dtype=np.float64)
    rb = np.empty_like(z)
    # bottom row from the continuous neutral profile of eq. (rho_wb)
    pz0 = p0 * (1.0 - g * z[0] / (cp * theta0)) ** (cp / R)
    rb[0] = pz0 / (R * Tb[0])
    half = 0.5 * g * grid.dz
    for k in range(grid.nz - 1):
        rb[k + 1] = rb[k] * (R * Tb[k] - half) / (R * Tb[k + 1] + half)
    pb = rb * R * Tb
    thb = Tb / (pb / p0) ** (R / cp)
    return Tb, rb, pb, thb


def bubble_perturbation(grid: Grid, kind: str, amp: float, rc: float,
                        xc: float, zc: float) -> np.ndarray:
    """theta' of the smooth (cosine, eq. dcEqn1) or non-smooth (step, eq.
    dcEqn2) bubble; amp is the peak perturbation in K."""
    X, Z = np.meshgrid(grid.xc(), grid.zc())
    r = np.sqrt((X - xc) ** 2 + (Z - zc) ** 2)
    if kind == "cosine":
        th = 0.5 * amp * (1.0 + np.cos(np.pi * r / rc))
    elif kind == "step":
        th = np.full_like(r, amp)
    else:
        raise ValueError(kind)
    return np.where(r <= rc, th, 0.0)


def conservative_from_primitive(grid: Grid, const: Constants, rho, u, w, T):
    """(rho, rho u, rho w, rho e) with e = cv T + |u|^2/2 + g z (Section 2.1)."""
    z = grid.zc()[:, None]
    e = const.cv * T + 0.5 * (u * u + w * w) + const.g * z
    f = {
        "rho": np.ascontiguousarray(rho, dtype=np.float64),
        "rhou": np.ascontiguousarray(rho * u, dtype=np.float64),
        "rhow": np.ascontiguousarray(rho * w, dtype=np.float64),
        "rhoe": np.ascontiguousarray(rho * e, dtype=np.float64),
    }
    return f


def rising_bubble(grid: Grid, const: Constants, theta0: float = 300.0,
                  kind: str = "cosine", amp: float = 2.0, rc: float = 2000.0,
                  xc: float = 10000.0, zc: float = 2000.0,
                  name: str = "bubble", steps: int = 100) -> Workload:
    """Bubble at rest in the balanced background: the perturbed temperature
    is T = T_bar * (theta0 + theta') / theta0 at the background pressure."""
    Tb, rb, pb, thb = hydrostatic_background(grid, const, theta0)
    thp = bubble_perturbation(grid, kind, amp, rc, xc, zc)
    T = Tb[:, None] * (theta0 + thp) / theta0
    rho = pb[:, None] / (const.R * T)
    zero = np.zeros_like(T)
    f = conservative_from_primitive(grid, const, rho, zero, zero, T)
    return Workload(name, grid, const, f, thb.copy(), steps)


def rest_atmosphere(grid: Grid, const: Constants, theta0: float = 300.0) -> Workload:
    """The balanced background alone (theta' = 0, fluid at rest)."""
    w = rising_bubble(grid, const, theta0, amp=0.0, name="rest")
    return w


def stratified_rest(grid: Grid, const: Constants, theta0: float = 300.0,
                    dtheta_dz: float = 0.003) -> Workload:
    """Stably stratified column at rest: theta(z) = theta0 + dtheta_dz z, with
    T(z) = theta(z) (1 - g z / (cp theta0)), in discrete hydrostatic balance."""
    prof = lambda z: (theta0 + dtheta_dz * z) * (1.0 - const.g * z / (const.cp * theta0))
    Tb, rb, pb, thb = hydrostatic_background(grid, const, theta0, prof)
    T = np.repeat(Tb[:, None], grid.nx, axis=1)
    rho = np.repeat(rb[:, None], grid.nx, axis=1)
    zero = np.zeros_like(T)
    f = conservative_from_primitive(grid, const, rho, zero, zero, T)
    return Workload("stratified_rest", grid, const, f, thb.copy(), 100)


def transpose_symmetric(n: int, L: float, const: Constants, T0: float = 300.0,
                        rho0: float = 1.1, uamp: float = 3.0, Tamp: float = 2.0) -> Workload:
    """State on an n x n square box that is unchanged by swapping x with z
    together with u with w (for use with g = 0)."""
    grid = Grid(n, n, L, L)
    X, Z = np.meshgrid(grid.xc() / L, grid.zc() / L)
    pi = np.pi
    T = T0 + Tamp * (np.cos(pi * X) * np.cos(2 * pi * Z) + np.cos(2 * pi * X) * np.cos(pi * Z))
    rho = rho0 * (1.0 + 0.01 * np.cos(pi * X) * np.cos(pi * Z))
    u = uamp * np.sin(pi * X) * np.cos(2 * pi * Z)
    w = uamp * np.cos(2 * pi * X) * np.sin(pi * Z)
    f = conservative_from_primitive(grid, const, rho, u, w, T)
    return Workload("transpose_symmetric", grid, const, f, np.full(n, T0), 20)


def acoustic_mode(grid: Grid, const: Constants, T0: float = 300.0,
                  rho0: float = 1.2, amp: float = 1e-6) -> Workload:
    """Small-amplitude standing sound wave cos(pi x / lx) in a uniform gas at
    rest, for use with g = 0: isentropic perturbation rho = rho0 (1 + a c),
    T = T0 (1 + a c)^(gamma-1), so p = rho R T (1 + a c)^gamma."""
    X = np.broadcast_to(grid.xc()[None, :], (grid.nz, grid.nx))
    c = np.cos(np.pi * X / grid.lx)
    gam = const.cp / const.cv
    rho = rho0 * (1.0 + amp * c)
    T = T0 * (1.0 + amp * c) ** (gam - 1.0)
    zero = np.zeros_like(T)
    f = conservative_from_primitive(grid, const, rho, zero, zero, T)
    thb = np.full(grid.nz, T0 * (const.p0 / (rho0 * const.R * T0)) ** (const.R / const.cp))
    return Workload("acoustic", grid, const, f, thb, 100)


def random_flow(grid: Grid, const: Constants, seed: int = 0, theta0: float = 300.0,
                uamp: float = 1.0, thamp: float = 1.0) -> Workload:
    """Bubble-like state with a smooth seeded velocity field that is zero in
    the wall-normal direction at every wall (for operator tests that need a
    moving fluid). Velocity is a sum of a few random Fourier modes."""
    rng = np.random.default_rng(seed)
    Tb, rb, pb, thb = hydrostatic_background(grid, const, theta0)
    X, Z = np.meshgrid(grid.xc() / grid.lx, grid.zc() / grid.lz)
    u = np.zeros_like(X)
    w = np.zeros_like(X)
    th = np.zeros_like(X)
    for _ in range(3):
        m, n = rng.integers(1, 4, size=2)
        a, b, c = rng.uniform(-1, 1, size=3)
        u += a * np.sin(m * np.pi * X) * np.cos(n * np.pi * Z)
        w += b * np.cos(m * np.pi * X) * np.sin(n * np.pi * Z)
        th += c * np.cos(m * np.pi * X) * np.cos(n * np.pi * Z)
    u *= uamp
    w *= uamp
    T = Tb[:, None] * (theta0 + thamp * th) / theta0
    rho = pb[:, None] / (const.R * T)
    f = conservative_from_primitive(grid, const, rho, u, w, T)
    return Workload("random_flow", grid, const, f, thb.copy(), 10)


# ---------------------------------------------------------------------------
# Named workloads. Sizes and constants follow the run configurations this
# library is measured on; see the design notes for the recipe of each.
# ---------------------------------------------------------------------------

def smooth_bubble_20km(nx: int = 160, nz: int = 80, dt: float = 0.1,
                       steps: int = 100, **kw) -> Workload:
    """Smooth cosine bubble, 2 K peak, radius 2 km, centred (10, 2) km, in a
    20 km x 10 km box, theta0 = 300 K, p0 = 1e5 Pa, R = 287, cp = 1004,
    g = 9.81, mu = 0.15, Pr = 1."""
    grid = Grid(nx, nz, 20000.0, 10000.0)
    const = Constants(dt=dt, **kw)
    return rising_bubble(grid, const, 300.0, "cosine", 2.0, 2000.0, 10000.0, 2000.0,
                         name=f"smooth_bubble_{nx}x{nz}", steps=steps)


def paper_smooth_bubble(res: float = 10.0, **kw) -> Workload:
    """Section 4.1: [0,1000]^2 m, cosine theta' of 0.5 K, r_c = 250 m,
    centre (500, 350) m, dt = 0.1, mu = 0.15, Pr = 1, cv = 715.5, R = 287."""
    n = int(round(1000.0 / res))
    grid = Grid(n, n, 1000.0, 1000.0)
    kw.setdefault("mu", 0.15)
    const = Constants(cp=287.0 + 715.5, dt=0.1, **kw)
    return rising_bubble(grid, const, 300.0, "cosine", 0.5, 250.0, 500.0, 350.0,
                         name=f"paper_smooth_{n}x{n}", steps=6000)


def paper_nonsmooth_bubble(res: float = 10.0, **kw) -> Workload:
    """Section 4.2: as Section 4.1 but theta' = 0.5 K inside r_c (step),
    centre (500, 260) m, mu = 0.3."""
    n = int(round(1000.0 / res))
    grid = Grid(n, n, 1000.0, 1000.0)
    kw.setdefault("mu", 0.3)
    const = Constants(cp=287.0 + 715.5, dt=0.1, **kw)
    return rising_bubble(grid, const, 300.0, "step", 0.5, 250.0, 500.0, 260.0,
                         name=f"paper_nonsmooth_{n}x{n}", steps=6000)


def les_member(n: int, amp: float = 0.5, xc: float = 500.0, zc: float = 260.0, cs: float = 0.17,
               name: str = "") -> Workload:
    """One member of the LES ensemble: the Section 4.2 non-smooth bubble
    (1 km box, theta' = amp inside r_c = 250 m centred (xc, zc), mu = 0.3,
    Pr = 1, dt = 0.1, c_v = 715.5) on n x n cells with the Smagorinsky
    eddy viscosity of constant cs added."""
    grid = Grid(n, n, 1000.0, 1000.0)
    const = Constants(cp=287.0 + 715.5, dt=0.1, mu=0.3, cs=cs)
    return rising_bubble(grid, const, 300.0, "step", amp, 250.0, xc, zc,
                         name=name or f"les_bubble_{n}x{n}", steps=100)


def les_ensemble(n_members: int = 256, seed: int = 0, sizes=(100, 200, 400),
                 cs: float = 0.17) -> List[Workload]:
    """The batched LES ensemble: non-smooth bubbles with seeded amplitudes
    uniform in [0.3, 0.7] K and centres jittered uniformly by up to 50 m in
    x and z, member m on sizes[m % len(sizes)] cells per side."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_members):
        n = int(sizes[m % len(sizes)])
        amp = float(rng.uniform(0.3, 0.7))
        xc = 500.0 + float(rng.uniform(-50.0, 50.0))
        zc = 260.0 + float(rng.uniform(-50.0, 50.0))
        out.append(les_member(n, amp, xc, zc, cs, name=f"les_member{m}_{n}x{n}"))
    return out


# ---------------------------------------------------------------------------
# Three dimensions: x, y horizontal, z up; fields are nz x ny x nx arrays
# (cell (i, j, k) at [k, j, i]).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Grid3:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def dz(self) -> float:
        return self.lz / self.nz

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def column(self) -> Grid:
        """The x-z grid with this grid's vertical levels."""
        return Grid(self.nx, self.nz, self.lx, self.lz)


def conservative3(grid: Grid3, const: Constants, rho, u, v, w, T):
    """(rho, rho u, rho v, rho w, rho e), e = cv T + |u|^2/2 + g z."""
    z = ((np.arange(grid.nz) + 0.5) * grid.dz)[:, None, None]
    e = const.cv * T + 0.5 * (u * u + v * v + w * w) + const.g * z
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    return {"rho": c(rho), "rhou": c(rho * u), "rhov": c(rho * v), "rhow": c(rho * w), "rhoe": c(rho * e)}


def rising_bubble3(grid: Grid3, const: Constants, theta0: float = 300.0, amp: float = 2.0,
                   rc: float = 2000.0, xc: float = 5000.0, yc: float = 5000.0, zc: float = 2000.0,
                   name: str = "bubble3d", steps: int = 200) -> Workload:
    """Spherical cosine bubble at rest in the balanced background (the
    smooth bubble of Section 4.1 in three dimensions)."""
    Tb, rb, pb, thb = hydrostatic_background(grid.column(), const, theta0)
    x = (np.arange(grid.nx) + 0.5) * grid.dx
    y = (np.arange(grid.ny) + 0.5) * grid.dy
    z = (np.arange(grid.nz) + 0.5) * grid.dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt((X - xc) ** 2 + (Y - yc) ** 2 + (Z - zc) ** 2)
    thp = np.where(r <= rc, 0.5 * amp * (1.0 + np.cos(np.pi * r / rc)), 0.0)
    T = Tb[:, None, None] * (theta0 + thp) / theta0
    rho = pb[:, None, None] / (const.R * T)
    zero = np.zeros_like(T)
    return Workload(name, grid, const, conservative3(grid, const, rho, zero, zero, zero, T), thb.copy(), steps)


def random_flow3(grid: Grid3, const: Constants, seed: int = 0, theta0: float = 300.0,
                 uamp: float = 1.0, thamp: float = 1.0) -> Workload:
    """A smooth seeded velocity field, zero in the wall-normal direction at
    every wall, and a temperature perturbation, in the balanced background."""
    rng = np.random.default_rng(seed)
    Tb, rb, pb, thb = hydrostatic_background(grid.column(), const, theta0)
    x = (np.arange(grid.nx) + 0.5) / grid.nx
    y = (np.arange(grid.ny) + 0.5) / grid.ny
    z = (np.arange(grid.nz) + 0.5) / grid.nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u, v, w, th = (np.zeros_like(X) for _ in range(4))
    for _ in range(3):
        l, m, n = rng.integers(1, 4, size=3)
        a, b, c, d = rng.uniform(-1, 1, size=4)
        u += a * np.sin(l * np.pi * X) * np.cos(m * np.pi * Y) * np.cos(n * np.pi * Z)
        v += b * np.cos(l * np.pi * X) * np.sin(m * np.pi * Y) * np.cos(n * np.pi * Z)
        w += c * np.cos(l * np.pi * X) * np.cos(m * np.pi * Y) * np.sin(n * np.pi * Z)
        th += d * np.cos(l * np.pi * X) * np.cos(m * np.pi * Y) * np.cos(n * np.pi * Z)
    T = Tb[:, None, None] * (theta0 + thamp * th) / theta0
    rho = pb[:, None, None] / (const.R * T)
    return Workload("random_flow3", grid, const,
                    conservative3(grid, const, rho, uamp * u, uamp * v, uamp * w, T), thb.copy(), 10)


def extrude3(wl: Workload, ny: int, ly: float) -> Workload:
    """A two-dimensional x-z workload repeated along y (v = 0): its
    three-dimensional evolution stays y-invariant and equals the x-z one."""
    g = wl.grid
    grid = Grid3(g.nx, ny, g.nz, g.lx, ly, g.lz)
    f = wl.fields
    rep = lambda a: np.ascontiguousarray(np.repeat(a[:, None, :], ny, axis=1))
    fields = {"rho": rep(f["rho"]), "rhou": rep(f["rhou"]), "rhov": np.zeros((g.nz, ny, g.nx)),
              "rhow": rep(f["rhow"]), "rhoe": rep(f["rhoe"])}
    return Workload(wl.name + f"_y{ny}", grid, wl.const, fields, wl.theta_bar, wl.steps)


def bubble3d(nx: int, ny: int, nz: int, dt: float = 0.05, steps: int = 200) -> Workload:
    """The 3D rising thermal bubble: 10 km x 10 km x 10 km, theta0 = 300 K,
    spherical cosine bubble of 2 K, radius 2 km, centred (5, 5, 2) km, at
    rest, mu = 0.15, Smagorinsky LES with cs = 0.17 (Pr = 1)."""
    return rising_bubble3(Grid3(nx, ny, nz, 10000.0, 10000.0, 10000.0), Constants(dt=dt, cs=0.17), 300.0, 2.0,
                          2000.0, 5000.0, 5000.0, 2000.0, name=f"bubble3d_{nx}x{ny}x{nz}", steps=steps)


WORKLOADS = {
    # 160 x 80 cells (125 m), dt = 0.1 s, 100 steps: the small parity case
    "bubble160x80": lambda: smooth_bubble_20km(160, 80, 0.1, 100),
    # 640 x 320 cells (31.25 m), dt = 0.05 s
    "bubble640x320": lambda: smooth_bubble_20km(640, 320, 0.05, 100),
    # 4096 x 2048 cells (about 4.9 m), dt = 0.05 s: larger than L2 at FP64
    "bubble4096x2048": lambda: smooth_bubble_20km(4096, 2048, 0.05, 3),
    # the non-smooth bubble with Smagorinsky LES on the ensemble's grid sizes
    "les100": lambda: les_member(100),
    "les200": lambda: les_member(200),
    "les400": lambda: les_member(400),
    # three dimensions
    "bubble3d_64x64x32": lambda: bubble3d(64, 64, 32, 0.05, 20),
    "bubble3d_192x192x96": lambda: bubble3d(192, 192, 96, 0.05, 20),
    "bubble3d_512x512x256": lambda: bubble3d(512, 512, 256, 0.05, 200),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]()
