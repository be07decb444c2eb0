"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances. Every solve is driven to round-off, so the two sides differ by
rounding order only. The velocity fields carry round-off noise of the
near-hydrostatic state (p' ~ 1e5 Pa resolved to ~1e-11 Pa), measured on the
oracle by perturbing the initial density by one ulp: relative L2 changes of
6e-12 (160x80) and 1.1e-11 (640x320) in rho u after 100 steps. The bar is
1e-10 relative L2 per field after 100 steps. In short runs the horizontal
velocity is still tiny (1e-4 m/s after three steps) and its round-off noise
is ~1e-10 of itself, so there velocity components, momenta and face fluxes
are measured against the norm of their vector; stage fields after one step
are compared element by element against the largest value of the field or
of its vector.
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


def run_both(gea, oracle_mod, wl, steps, **solver_kw):
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, steps)
    s = gea.Solver(wl.grid, wl.const, **solver_kw)
    s.set_conservative(wl.fields)
    s.step(steps)
    return so, s


def compare_state(gea_state, so, tol, const, grid, fields=None, vector_norm=False):
    """Relative L2 error per field. vector_norm: velocity components,
    momenta and face fluxes are measured against the norm of their vector
    (for short runs in which one component is still at round-off level)."""
    out = {}
    cv = const.cp - const.R
    co = so.conservative(const.g, cv, grid.dz)
    z = (np.arange(grid.nz) + 0.5)[:, None] * grid.dz
    gs = gea_state
    cg = {"rho": gs["rho"], "rhou": gs["rho"] * gs["u"], "rhow": gs["rho"] * gs["w"],
          "rhoe": gs["rho"] * (cv * gs["T"] + 0.5 * (gs["u"] ** 2 + gs["w"] ** 2) + const.g * z)}
    vec = {}
    if vector_norm:
        m = np.hypot(np.linalg.norm(co["rhou"]), np.linalg.norm(co["rhow"]))
        f = np.hypot(np.linalg.norm(so["phix"]), np.linalg.norm(so["phiz"]))
        vec = {"rhou": m, "rhow": m, "phix": f, "phiz": f}
    for k in ("rho", "rhou", "rhow", "rhoe"):
        out[k] = np.linalg.norm(cg[k] - co[k]) / vec[k] if k in vec else rel_l2(cg[k], co[k])
    for k in fields or ("T", "h", "p", "pp", "pold", "phix", "phiz"):
        out[k] = np.linalg.norm(gs[k] - so[k]) / vec[k] if k in vec else rel_l2(gs[k], so[k])
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, (bad, out)
    return out


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_stage_parity_one_step(gea, oracle_mod, graph):
    """Every intermediate field of one step (one corrector) element by
    element, on a moving stratified state so that all terms are active."""
    grid = W.Grid(160, 80, 16000.0, 6000.0)
    c = W.Constants(dt=0.2, n_corr=1, mu=2.0)
    wl = W.random_flow(grid, c, seed=4, uamp=5.0, thamp=2.0)
    o = oracle_mod.Oracle(grid, c)
    so = o.derive(wl.fields)
    _, d = o.step(so, 1, dump=True)
    s = gea.Solver(grid, c, graph=graph)
    s.set_conservative(wl.fields)
    s.step(1)
    # element-wise, relative to the largest value of the field or its vector
    scale = {"u1": ("u1", "w1"), "w1": ("u1", "w1"), "Hx": ("Hx", "Hz"), "Hz": ("Hx", "Hz")}
    for name, tol in (("rho1", 1e-14), ("u1", 1e-12), ("w1", 1e-12), ("h1", 1e-14),
                      ("rho2", 1e-14), ("Dx", 1e-13), ("Dz", 1e-13), ("Hx", 1e-12),
                      ("Hz", 1e-12), ("b", 1e-13)):
        g = s.field(name)
        ref = d[name]
        sc = max(np.abs(d[k]).max() for k in scale.get(name, (name,)))
        err = np.abs(g - ref).max() / sc
        assert err <= tol, (name, err)
    compare_state(s.get_full(), so, 1e-11, c, grid)
    st = s.stats()
    assert st["status"] == 0 and st["steps_done"] == 1
    assert st["cg_relres"][0] <= c.cg_rtol


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("name", ["bubble160x80", "bubble640x320"])
def test_parity_100_steps(gea, oracle_mod, name, graph):
    wl = W.get(name)
    so, s = run_both(gea, oracle_mod, wl, 100, graph=graph)
    errs = compare_state(s.get_full(), so, 1e-10, wl.const, wl.grid)
    th_g, m_g, e_g = s.diagnostics(wl.theta_bar)
    th_o, m_o, e_o = oracle_mod.Oracle(wl.grid, wl.const).diagnostics(so, wl.theta_bar)
    assert np.abs(th_g - th_o).max() < 1e-9
    # totals differ by summation order over ~1e5 terms (the oracle adds
    # sequentially: error up to N eps)
    assert abs(m_g - m_o) / m_o < 1e-11 and abs(e_g - e_o) / e_o < 1e-11
    print(name, errs, s.stats())


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("nx,nz,ncorr", [(37, 23, 2), (50, 34, 2), (4, 4, 1), (66, 130, 3),
                                          (128, 96, 2)])
def test_parity_ragged_sizes(gea, oracle_mod, nx, nz, ncorr, graph):
    """Sizes that are not multiples of the 32 x 8 tile, odd sizes (a
    single multigrid level), the smallest grid, and several corrector
    counts, on a moving stratified state."""
    grid = W.Grid(nx, nz, 40.0 * nx, 30.0 * nz)
    c = W.Constants(dt=0.2, n_corr=ncorr, mu=1.5)
    wl = W.random_flow(grid, c, seed=nx * 1000 + nz, uamp=3.0, thamp=2.0)
    so, s = run_both(gea, oracle_mod, wl, 20, graph=graph)
    compare_state(s.get_full(), so, 1e-10, c, grid)


@pytest.mark.parametrize("kw", [dict(g=0.0), dict(mu=0.0), dict(Pr=0.7, mu=3.0)])
def test_parity_constants(gea, oracle_mod, kw):
    grid = W.Grid(48, 40, 2400.0, 2000.0)
    c = W.Constants(dt=0.1, **kw)
    wl = W.random_flow(grid, c, seed=11, uamp=2.0)
    so, s = run_both(gea, oracle_mod, wl, 20)
    compare_state(s.get_full(), so, 1e-10, c, grid)


def test_rest_atmosphere_on_gpu(gea):
    wl = W.rest_atmosphere(W.Grid(160, 80, 20000.0, 10000.0), W.Constants(dt=0.1))
    s = gea.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.step(100)
    st = s.get_full()
    assert np.abs(st["u"]).max() < 1e-10 and np.abs(st["w"]).max() < 1e-10
    th, _, _ = s.diagnostics(wl.theta_bar)
    assert np.abs(th).max() < 1e-10


def test_checkpoint_roundtrip_bitwise(gea):
    """FULL get + set continues bit for bit."""
    wl = W.get("bubble160x80")
    a = gea.Solver(wl.grid, wl.const)
    a.set_conservative(wl.fields)
    a.step(7)
    ck = a.get_full()
    a.step(5)
    ref = a.get_full()
    b = gea.Solver(wl.grid, wl.const)
    b.set_full(ck)
    b.step(5)
    got = b.get_full()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


def test_checkpoint_file_resumes_bitwise(gea, tmp_path):
    """A checkpoint file of the full state (Solver.save_checkpoint) loaded
    into a new context continues bit for bit."""
    wl = W.get("bubble160x80")
    a = gea.Solver(wl.grid, wl.const)
    a.set_conservative(wl.fields)
    a.step(6)
    path = str(tmp_path / "bubble.npz")
    a.save_checkpoint(path)
    a.step(4)
    ref = a.get_full()
    b = gea.Solver(wl.grid, wl.const)
    ck = b.load_checkpoint(path)
    assert ck["steps_done"] == 6
    b.step(4)
    got = b.get_full()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


def test_deterministic(gea):
    wl = W.get("bubble160x80")
    out = []
    for _ in range(2):
        s = gea.Solver(wl.grid, wl.const)
        s.set_conservative(wl.fields)
        s.step(10)
        out.append(s.get_full())
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_noconv_keeps_last_state(gea, graph):
    """A pressure solve that hits its iteration cap reports GEA_ERR_NOCONV
    and leaves the last completed state in place."""
    wl = W.get("bubble160x80")
    wl.const.cg_maxit = 1
    s = gea.Solver(wl.grid, wl.const, graph=graph)
    s.set_conservative(wl.fields)
    before = s.get_full()
    with pytest.raises(gea.GeaError) as ei:
        s.step(3)
    assert ei.value.code == gea.GEA_ERR_NOCONV
    after = s.get_full()
    for k in before:
        assert np.array_equal(before[k], after[k]), k


def test_set_state_rejects_bad_input(gea):
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    f = {k: v.copy() for k, v in wl.fields.items()}
    f["rho"][3, 4] = -1.0
    with pytest.raises(gea.GeaError) as ei:
        s.set_conservative(f)
    assert ei.value.code == gea.GEA_ERR_INVAL
    with pytest.raises(gea.GeaError):
        s.step(1)


def test_device_tensors_in_and_out(gea):
    import torch
    wl = W.get("bubble160x80")
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.fields.items()}
    s = gea.Solver(wl.grid, wl.const, stream=torch.cuda.current_stream())
    s.set_conservative(dev)
    s.step(2)
    host = s.get_full()
    nx, nz = wl.grid.nx, wl.grid.nz
    out = {k: torch.empty((nz, nx), dtype=torch.float64, device="cuda") for k in host}
    out["phix"] = torch.empty((nz, nx + 1), dtype=torch.float64, device="cuda")
    out["phiz"] = torch.empty((nz + 1, nx), dtype=torch.float64, device="cuda")
    s.get_full(out)
    torch.cuda.synchronize()
    for k in host:
        assert np.array_equal(out[k].cpu().numpy(), host[k]), k


def roundoff_floor_4096():
    """Per-field round-off floor of one oracle step on the 4096 x 2048 bubble
    (tests/golden/roundoff_floor_bubble4096x2048.txt, written by
    make_roundoff_floor.py from the oracle alone): the larger of the
    differences caused by reversing the oracle's reduction order and by
    moving every input value by one ulp at random."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "roundoff_floor_bubble4096x2048.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, rev, ulp = line.split()
        out[k] = max(float(rev), float(ulp))
    return out


def test_full_size_one_step(gea, oracle_mod):
    """4096 x 2048 (larger than L2 at FP64): one step against the oracle,
    plus mass conservation and mirror symmetry of the GPU state.

    The bar comes from the oracle's own round-off floor F (file above). One
    step leaves velocities of ~3e-3 m/s that the near-hydrostatic state makes
    sensitive to rounding: moving each input value by one ulp moves rho u,
    rho w by 2-3e-10 and the face fluxes by 4-5e-10 of their vector norm. The
    GPU rounds differently in every stage of the step (the derivation of p',
    both predictors, the EOS update, the assembly, each CG iteration and the
    correction of both correctors: about ten independent injections of
    one-ulp differences), and independent perturbations add in quadrature,
    so the expected difference is about sqrt(10) F ~ 3 F. The bar is 4 F,
    with F the larger of the two components of a vector (they share its
    norm), and 64 ulps (1.4e-14) for scalar fields, whose floor is a few
    ulps."""
    wl = W.get("bubble4096x2048")
    so, s = run_both(gea, oracle_mod, wl, 1)
    g = s.get_full()
    F = roundoff_floor_4096()
    eps = np.finfo(np.float64).eps
    mom = 4.0 * max(F["rhou"], F["rhow"])
    flx = 4.0 * max(F["phix"], F["phiz"])
    bars = {k: max(4.0 * v, 64 * eps) for k, v in F.items()}
    bars.update({"rhou": mom, "rhow": mom, "phix": flx, "phiz": flx})
    errs = compare_state(g, so, 1.0, wl.const, wl.grid, vector_norm=True)
    ratio = {k: errs[k] / bars[k] for k in errs}
    print("4096x2048 one step:", errs, "error / bar:", ratio)
    bad = {k: (errs[k], bars[k]) for k in errs if not errs[k] <= bars[k]}
    assert not bad, bad
    _, m1, _ = s.diagnostics(wl.theta_bar)
    s2 = gea.Solver(wl.grid, wl.const)
    s2.set_conservative(wl.fields)
    _, m0, _ = s2.diagnostics(wl.theta_bar)
    assert abs(m1 - m0) / m0 < 1e-13
    u, w = g["u"], g["w"]
    vmax = max(np.abs(u).max(), np.abs(w).max())
    assert np.abs(u + u[:, ::-1]).max() <= 1e-9 * vmax
    assert np.abs(w - w[:, ::-1]).max() <= 1e-9 * vmax


def test_persistent_and_graph_paths_agree(gea):
    """The two step drivers run the same tile functions; only the order of
    the reduction sums differs (block count), so they agree to round-off."""
    wl = W.get("bubble640x320")
    out = []
    for graph in (False, True):
        s = gea.Solver(wl.grid, wl.const, graph=graph)
        s.set_conservative(wl.fields)
        s.step(20)
        assert s.stats()["driver"] == ("graph" if graph else "persistent")
        out.append(s.get_full())
    for k in ("rho", "T", "pp"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-13 * np.abs(out[1][k]).max(), k
    for k in ("u", "w"):
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-10 * np.abs(out[1]["w"]).max(), k


def test_multi_step_launch_matches_single_steps(gea):
    """n steps in one persistent launch equal n launches of one step."""
    wl = W.get("bubble160x80")
    a = gea.Solver(wl.grid, wl.const)
    a.set_conservative(wl.fields)
    a.step(6)
    b = gea.Solver(wl.grid, wl.const)
    b.set_conservative(wl.fields)
    for _ in range(6):
        b.step(1)
    ra, rb = a.get_full(), b.get_full()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


@pytest.mark.parametrize("device_out", [False, True], ids=["host", "device"])
def test_conservative_get_on_device(gea, oracle_mod, device_out):
    """gea_get_state(CONSERVATIVE) computes rho, rho u, rho w and
    rho e = rho (cv T + |u|^2/2 + g z) (Section 2.1) on the device: a
    conservative set followed by a conservative get returns the input to
    round-off, and after 20 steps it matches the oracle's conservative
    fields like every other field (1e-10 relative L2)."""
    import torch
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    nx, nz = wl.grid.nx, wl.grid.nz
    out = None
    if device_out:
        out = {k: torch.empty((nz, nx), dtype=torch.float64, device="cuda")
               for k in ("rho", "rhou", "rhow", "rhoe")}
    got = s.get_conservative(out)
    got = {k: (v.cpu().numpy() if device_out else v) for k, v in got.items()}
    for k in ("rho", "rhoe"):
        assert np.abs(got[k] - wl.fields[k]).max() <= 1e-14 * np.abs(wl.fields[k]).max(), k
    for k in ("rhou", "rhow"):
        assert np.abs(got[k] - wl.fields[k]).max() <= 1e-14 * np.abs(wl.fields["rho"]).max(), k
    s.step(20)
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, 20)
    co = so.conservative(wl.const.g, wl.const.cp - wl.const.R, wl.grid.dz)
    got = s.get_conservative(out)
    got = {k: (v.cpu().numpy() if device_out else v) for k, v in got.items()}
    m = np.hypot(np.linalg.norm(co["rhou"]), np.linalg.norm(co["rhow"]))
    for k in ("rho", "rhoe"):
        assert rel_l2(got[k], co[k]) <= 1e-10, k
    for k in ("rhou", "rhow"):
        assert np.linalg.norm(got[k] - co[k]) / m <= 1e-10, k
