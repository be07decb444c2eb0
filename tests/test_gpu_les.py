"""Smagorinsky LES on the GPU (gea_constants.cs > 0) against the oracle's
LES step, on the non-smooth bubble of the ensemble workload (Section 4.2
set-up, 1 km box, theta' step of 0.5 K, mu = 0.3, cs = 0.17).

The eddy viscosity enters only as stencil coefficients, so the FP64 step
stays at the parity bound of the constant-viscosity step (relative L2 1e-10
per field after 100 steps); the mixed step within its own bounds.
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


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
def test_les_parity_100_steps(gea, oracle_mod, graph):
    wl = W.get("les100")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, 100)
    s = gea.Solver(wl.grid, wl.const, graph=graph)
    s.set_conservative(wl.fields)
    s.step(100)
    st = s.stats()
    assert st["status"] == 0 and st["driver"] == ("graph" if graph else "persistent")
    g = s.get_full()
    errs = {k: rel(g[k], so[k]) for k in ("rho", "T", "p", "pp", "u", "w", "phix", "phiz")}
    print(errs, st)
    assert max(errs.values()) < 1e-10, errs
    # the eddy viscosity acts: the LES state differs from the constant-mu one
    c0 = W.Constants(cp=wl.const.cp, dt=wl.const.dt, mu=wl.const.mu)
    s0 = gea.Solver(wl.grid, c0, graph=graph)
    s0.set_conservative(wl.fields)
    s0.step(100)
    assert rel(s0.get_full()["w"], g["w"]) > 1e-4


def test_les_mixed(gea, oracle_mod):
    wl = W.get("les100")
    o = oracle_mod.Oracle(wl.grid, wl.const)
    so = o.derive(wl.fields)
    o.step(so, 50)
    s = gea.Solver(wl.grid, wl.const, mixed=True)
    s.set_conservative(wl.fields)
    s.step(50)
    g = s.get_full()
    vel = np.hypot(np.linalg.norm(so["u"]), np.linalg.norm(so["w"]))
    assert rel(g["rho"], so["rho"]) < 1e-11 and rel(g["T"], so["T"]) < 1e-11
    for k in ("u", "w"):
        assert np.linalg.norm(g[k] - so[k]) / vel < 5e-8, k


def test_les_rejects_prandtl_not_one(gea):
    wl = W.get("les100")
    c = W.Constants(cp=wl.const.cp, dt=0.1, mu=0.3, cs=0.17, Pr=0.7)
    with pytest.raises(gea.GeaError) as ei:
        gea.Solver(wl.grid, c)
    assert ei.value.code == gea.GEA_ERR_INVAL
