"""The learned network inside the pressure solve (gea_attach_net): as the
initial guess and as a flexible-CG preconditioner stage.

The guess only changes where each solve starts: x + alpha e with the A-norm
optimal alpha, then the same solve to the same tolerance. So with any
network, trained or not, the FP64 step still matches the oracle at the
parity bound, and the mixed step stays within its bounds. The stage only
shapes the search directions of a solve that runs to the same tolerance.
"""
import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea as G
    from paper_2303_10499_gb300 import learned
    return torch, G, learned


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_untrained_guess_keeps_parity(env, oracle_mod, mixed):
    torch, G, learned = env
    wl = W.get("bubble160x80")
    net = G.Net(1, 80, 160, relu=False)
    net.set_params(learned.initial_params(3) * 0.5)
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, 30)
    s = G.Solver(wl.grid, wl.const, mixed=mixed)
    s.set_conservative(wl.fields)
    s.attach_net(net)
    s.step(30)
    st = s.stats()
    assert st["status"] == 0 and st["driver"] == ("mixed" if mixed else "graph")
    g = s.get_full()
    bound = 5e-9 if mixed else 1e-10
    for k in ("rho", "T", "pp"):
        assert rel_l2(g[k], so[k]) < (1e-11 if mixed else 1e-10), k
    vel = np.hypot(np.linalg.norm(so["u"]), np.linalg.norm(so["w"]))
    for k in ("u", "w"):
        assert np.linalg.norm(g[k] - so[k]) / vel < bound, k
    s.attach_net(None, 0)
    s.step(1)
    assert s.stats()["status"] == 0


def test_attach_rejects_grids_off_the_network(env):
    torch, G, learned = env
    net = G.Net(1, 80, 160)
    wl = W.random_flow(W.Grid(37, 23, 370.0, 230.0), W.Constants(), seed=1)
    s = G.Solver(wl.grid, wl.const)
    with pytest.raises(G.GeaError) as ei:
        s.attach_net(net)
    assert ei.value.code == G.GEA_ERR_INVAL
    big = W.get("bubble640x320")
    s2 = G.Solver(big.grid, big.const)
    with pytest.raises(G.GeaError):
        s2.attach_net(net)        # 640 x 320 does not fit an 80 x 160 network


def test_kept_residual_is_b_minus_a_p(env, oracle_mod):
    """GEA_FLAG_KEEP_R0 keeps r0 = b - A p'^n of the first corrector: with one
    corrector, b is that corrector's right-hand side (GEA_FIELD_B) and A the
    step's operator (GEA_FIELD_HC/HAX/HAZ)."""
    torch, G, learned = env
    from oracle import unet
    grid = W.Grid(64, 32, 6400.0, 3200.0)
    c = W.Constants(dt=0.2, n_corr=1)
    wl = W.random_flow(grid, c, seed=5, uamp=3.0, thamp=2.0)
    s = G.Solver(grid, c, keep_r0=True)
    s.set_conservative(wl.fields)
    pp0 = s.get_full()["pp"]
    s.step(1)
    r0, b = s.field("r0"), s.field("b")
    Ap = unet.helmholtz_apply(pp0, s.field("hc"), s.field("hax"), s.field("haz"))
    assert np.abs(r0 - (b - Ap)).max() <= 1e-9 * np.abs(b).max()


def test_trained_guess_saves_iterations_at_4096(env):
    """The network trained on the 4096 x 2048 bubble's own pressure systems
    makes the first corrector's solve to 1e-8 (relative to b) start within
    its tolerance: over six steps the plain MG-CG needs one iteration per
    step there, the learned start (measured) none in five of six."""
    import copy
    torch, G, learned = env
    wl = W.get("bubble4096x2048")
    samples = learned.collect(wl, 8, every=2)
    net = G.Net(8, 1024, 1024, relu=False)
    net.set_params(learned.initial_params(1) * 0.5)
    res = learned.train(net, samples, 400, n=8, h=256, w=256, lr=2e-3)
    assert np.mean(res["losses"][-20:]) < res["losses"][0]
    c = copy.copy(wl.const)
    c.cg_rtol = 1e-8
    its = {}
    for use in (False, True):
        s = G.Solver(wl.grid, c, graph=True)
        s.set_conservative(wl.fields)
        if use:
            s.attach_net(net)
        its[use] = []
        for _ in range(6):
            s.step(1)
            its[use].append(sum(s.stats()["cg_iters"]))
        s.close()
    print(its)
    assert sum(its[True]) < sum(its[False])


@pytest.fixture(scope="module")
def small_net(env):
    """A network trained briefly on the 160 x 80 bubble's own pressure
    systems."""
    torch, G, learned = env
    wl = W.get("bubble160x80")
    samples = learned.collect(wl, 6, every=1)
    net = G.Net(4, 80, 160, relu=False)
    net.set_params(learned.initial_params(2) * 0.5)
    learned.train(net, samples, 150, n=4, h=80, w=160, lr=2e-3)
    return net


@pytest.mark.parametrize("mode", [2, 3], ids=["stage", "guess+stage"])
def test_network_preconditioner_keeps_parity(env, oracle_mod, small_net, mode):
    """Flexible CG with the two-stage preconditioner (the network, then a
    V-cycle on the residual its step leaves; mode 2, and with the learned
    initial guess as well, mode 3): the network only shapes the search
    directions, and each solve still runs to the same tolerance, so the FP64
    step matches the oracle at the parity bound."""
    torch, G, learned = env
    wl = W.get("bubble160x80")
    steps = 20
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, steps)
    s = G.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.attach_net(small_net, mode)
    its = []
    for _ in range(steps):
        s.step(1)
        st = s.stats()
        assert st["status"] == 0, st
        its.append(st["cg_iters"])
    assert st["driver"] == "graph"
    assert all(i[0] > 0 for i in its), its
    g = s.get_full()
    for k in ("rho", "T", "pp"):
        assert rel_l2(g[k], so[k]) < 1e-10, k
    vel = np.hypot(np.linalg.norm(so["u"]), np.linalg.norm(so["w"]))
    for k in ("u", "w"):
        assert np.linalg.norm(g[k] - so[k]) / vel < 1e-10, k
    print(mode, its)


def test_network_preconditioner_is_fp64_only(env):
    torch, G, learned = env
    wl = W.get("bubble160x80")
    net = G.Net(1, 80, 160, relu=False)
    s = G.Solver(wl.grid, wl.const, mixed=True)
    with pytest.raises(G.GeaError) as ei:
        s.attach_net(net, 2)
    assert ei.value.code == G.GEA_ERR_INVAL
    s.attach_net(net, 1)          # the guess is fine for the mixed step
    with pytest.raises(G.GeaError) as ei:
        s.attach_net(net, 4)      # modes are 0..3
    assert ei.value.code == G.GEA_ERR_INVAL
