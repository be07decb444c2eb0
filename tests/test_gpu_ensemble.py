"""Ensembles of independent contexts in one cooperative launch
(gea_ensemble_*): members of different sizes and constants, each on its own
share of the blocks with its own barrier and reductions.

A member's step is its persistent-driver step with the reduction sums taken
over fewer blocks (a different summation order), so it matches the member
stepped alone to rounding (bound 1e-12 relative L2; the solves run to
round-off) and the oracle at the parity bound.
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def members():
    """LES bubbles of the three ensemble sizes, a constant-viscosity bubble
    and a ragged random flow."""
    out = W.les_ensemble(6, seed=3)
    out.append(W.get("bubble160x80"))
    out.append(W.random_flow(W.Grid(37, 23, 370.0, 230.0), W.Constants(dt=0.2, mu=1.5), seed=5,
                             uamp=3.0, thamp=2.0))
    return out


def test_ensemble_matches_members_stepped_alone(gea, oracle_mod):
    wls = members()
    steps = 10
    solo = []
    for wl in wls:
        s = gea.Solver(wl.grid, wl.const)
        s.set_conservative(wl.fields)
        s.step(steps)
        solo.append(s.get_full())
        s.close()
    ens = [gea.Solver(wl.grid, wl.const) for wl in wls]
    for s, wl in zip(ens, wls):
        s.set_conservative(wl.fields)
    E = gea.Ensemble(ens)
    nb = E.blocks()
    assert min(nb) >= 1
    E.step(steps // 2)
    E.step(steps - steps // 2)
    for k, (s, ref) in enumerate(zip(ens, solo)):
        st = s.stats()
        assert st["status"] == 0 and st["steps_done"] == steps, (k, st)
        g = s.get_full()
        vel = np.hypot(np.linalg.norm(ref["u"]), np.linalg.norm(ref["w"]))
        for f in ("rho", "T", "pp"):
            assert rel(g[f], ref[f]) < 1e-12, (k, f)
        for f in ("u", "w"):
            assert np.linalg.norm(g[f] - ref[f]) / vel < 1e-9, (k, f)
    # the smallest LES member against the oracle; after ten steps the
    # velocities are ~1e-5 m/s and their round-off noise ~1e-10 of the
    # vector norm (measured 1.1e-10), so the bound is 5e-10 here
    wl = wls[0]
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, steps)
    g = ens[0].get_full()
    vel = np.hypot(np.linalg.norm(so["u"]), np.linalg.norm(so["w"]))
    assert rel(g["rho"], so["rho"]) < 1e-10
    assert np.linalg.norm(g["w"] - so["w"]) / vel < 5e-10


def test_ensemble_is_deterministic(gea):
    wls = W.les_ensemble(9, seed=11)
    out = []
    for _ in range(2):
        ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
        for s, wl in zip(ss, wls):
            s.set_conservative(wl.fields)
        E = gea.Ensemble(ss)
        E.step(5)
        out.append([s.get_full() for s in ss])
        E.close()
    for a, b in zip(*out):
        for f in a:
            assert np.array_equal(a[f], b[f]), f


def test_ensemble_rejects_unsuitable_members(gea):
    wl = W.get("les100")
    a = gea.Solver(wl.grid, wl.const)
    b = gea.Solver(wl.grid, wl.const, mixed=True)
    with pytest.raises(gea.GeaError):
        gea.Ensemble([a, b])
    with pytest.raises(gea.GeaError):
        gea.Ensemble([a, a])
    E = gea.Ensemble([a])
    with pytest.raises(gea.GeaError) as ei:
        E.step(1)                       # no state set
    assert ei.value.code == gea.GEA_ERR_STATE


def test_weights_and_autotune(gea):
    """Blocks follow the weights (at least one per member, at most one per
    tile); the autotuner returns a working partition and its trial times."""
    import torch
    from paper_2303_10499_gb300 import ensemble
    wls = W.les_ensemble(6, seed=2)
    ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
    for s, wl in zip(ss, wls):
        s.set_conservative(wl.fields)
    tiles = [((wl.grid.nx + 31) // 32) * ((wl.grid.nz + 7) // 8) for wl in wls]
    w = np.ones(len(wls))
    w[2] = 1e6                      # one 400 x 400 member takes (almost) everything
    E = gea.Ensemble(ss, weights=w)
    nb = E.blocks()
    assert all(b >= 1 for b in nb) and all(b <= t for b, t in zip(nb, tiles))
    assert nb[2] == max(nb) and nb[2] > 10 * max(nb[:2])
    E.close()
    E, rep = ensemble.autotune(ss, stream=torch.cuda.current_stream(), betas=(0.0, 1.0), trial_steps=1)
    by = rep["ms_per_step_by_shape_and_beta"]
    assert set(by) == {"32x8", "16x16", "64x4"} and all(set(v) == {"0.0", "1.0"} for v in by.values())
    assert rep["tile_shape"] in by
    E.step(1)
    steps = ss[0].stats()["steps_done"]
    # one step to measure the iterations, one per shape and weight, one more
    assert steps == 1 + 3 * 2 + 1 and all(s.stats()["status"] == 0 for s in ss)


def test_ensemble_graph_launch_equals_direct_launch(gea):
    """The ensemble step as a replayed CUDA graph (one cooperative kernel node
    with its own device copy of the arguments) gives the direct launch's
    states bit for bit, over 1-step and 2-step calls and both slot parities;
    members at different parities fall back to the direct launch."""
    wls = W.les_ensemble(5, seed=4)

    def members():
        ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
        for s, wl in zip(ss, wls):
            s.set_conservative(wl.fields)
        return ss

    out = []
    for graph in (True, False):
        ss = members()
        E = gea.Ensemble(ss)
        E.set_graph(graph)
        for n in (1, 1, 2, 1, 2):
            E.step(n)
        E.close()
        out.append([s.get_full() for s in ss])
        assert all(s.stats()["steps_done"] == 7 and s.stats()["status"] == 0 for s in ss)
    for a, b in zip(*out):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    # parities apart: member 0 one step ahead
    ss = members()
    ss[0].step(1)
    E = gea.Ensemble(ss)
    E.step(2)
    E.close()
    assert ss[0].stats()["steps_done"] == 3 and ss[1].stats()["steps_done"] == 2
    ref = gea.Solver(wls[0].grid, wls[0].const)
    ref.set_conservative(wls[0].fields)
    ref.step(3)
    a, b = ss[0].get_full(), ref.get_full()
    for k in ("rho", "T", "pp"):
        assert np.abs(a[k] - b[k]).max() <= 1e-13 * np.abs(b[k]).max(), k


def test_ensemble_graph_follows_member_settings(gea):
    """A captured ensemble graph carries the members' argument blocks; when a
    member's smoother weight changes between steps the next launch uses the
    new weight, so graph and direct launches stay equal bit for bit."""
    wls = W.les_ensemble(3, seed=6)
    out = []
    for graph in (True, False):
        ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
        for s, wl in zip(ss, wls):
            s.set_conservative(wl.fields)
        E = gea.Ensemble(ss)
        E.set_graph(graph)
        E.step(1)
        ss[1].set_smoother_weight(0.8)
        E.step(1)
        E.step(1)
        E.close()
        out.append([s.get_full() for s in ss])
    for a, b in zip(*out):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def test_mixed_precision_ensemble(gea):
    """Mixed-precision members (FP64 state, FP32 inner solves) in one launch:
    each member's result is its own mixed persistent run's up to the order of
    the sums, and FP64 and mixed members cannot share a launch. In the
    ensemble a member runs on fewer blocks than alone, so its FP32 reductions
    add in another order and the inner solves (stopped at 1e-5 of their
    initial residual) take other iterates within that tolerance: velocities
    agree to 1e-6 of their maximum (a tenth of the inner tolerance), theta'
    to 1e-7 K (the mixed step's own bar against the oracle), scalars to
    1e-11."""
    wls = W.les_ensemble(4, seed=5)
    ss = []
    for wl in wls:
        s = gea.Solver(wl.grid, wl.const, mixed=True)
        s.set_conservative(wl.fields)
        ss.append(s)
    E = gea.Ensemble(ss)
    E.step(4)
    E.close()
    for s, wl in zip(ss, wls):
        assert s.stats()["status"] == 0 and s.stats()["steps_done"] == 4
        ref = gea.Solver(wl.grid, wl.const, mixed=True)
        ref.set_conservative(wl.fields)
        ref.step(4)
        a, b = s.get_full(), ref.get_full()
        for k in ("rho", "T", "pp"):
            assert np.abs(a[k] - b[k]).max() <= 1e-11 * np.abs(b[k]).max(), k
        vmax = max(np.abs(b["u"]).max(), np.abs(b["w"]).max())
        for k in ("u", "w"):
            assert np.abs(a[k] - b[k]).max() <= 1e-6 * vmax, k
        assert np.abs(s.diagnostics(wl.theta_bar)[0] - ref.diagnostics(wl.theta_bar)[0]).max() <= 1e-7
    f = gea.Solver(wls[0].grid, wls[0].const)
    f.set_conservative(wls[0].fields)
    with pytest.raises(gea.GeaError) as ei:
        gea.Ensemble([f, ss[1]])
    assert ei.value.code == gea.GEA_ERR_INVAL


def test_small_members_share_blocks(gea):
    """Members whose weight share is below one block are packed onto blocks
    they share and run in turn, each as a one-block grid: an ensemble may
    then hold more members than there are co-resident blocks, and every
    member still matches its own persistent driver to rounding."""
    wls = [W.random_flow(W.Grid(24, 16, 240.0, 160.0), W.Constants(dt=0.2, mu=1.5), seed=s, uamp=2.0,
                         thamp=1.0) for s in range(600)]
    wls.append(W.get("les400"))      # one large member beside them
    steps = 4
    ss = [gea.Solver(wl.grid, wl.const) for wl in wls]
    for s, wl in zip(ss, wls):
        s.set_conservative(wl.fields)
    E = gea.Ensemble(ss)
    nb = E.blocks()
    assert len(nb) == len(wls) > 456 and all(b == 1 for b in nb[:-1]) and nb[-1] > 1
    E.step(steps)
    E.sync()
    for k in list(range(0, 600, 37)) + [599, 600]:
        st = ss[k].stats()
        assert st["status"] == 0 and st["steps_done"] == steps, (k, st)
        ref = gea.Solver(wls[k].grid, wls[k].const)
        ref.set_conservative(wls[k].fields)
        ref.step(steps)
        a, b = ss[k].get_full(), ref.get_full()
        vel = np.hypot(np.linalg.norm(b["u"]), np.linalg.norm(b["w"]))
        for f in ("rho", "T", "pp"):
            assert rel(a[f], b[f]) < 1e-12, (k, f)
        for f in ("u", "w"):
            assert np.linalg.norm(a[f] - b[f]) / vel < 1e-9, (k, f)
        ref.close()
    E.close()
