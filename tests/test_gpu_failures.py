"""Failure detection on the GPU, in forms that fault and hang nothing.

* A bounded wait that runs out: the persistent step kernel's grid barriers
  poll an arrival counter with an iteration limit. gea_set_wait_limit(0)
  makes every block that is not the last to arrive give up at its first
  poll, so the step stops at a phase boundary with GEA_ERR_TIMEOUT; the
  state stays at the last completed step and the context works again after
  the next set_state.
* A NaN loaded through a host FULL set_state: the residual norms fold the
  check for non-finite values into their reductions (GEA_ERR_NONFINITE), and
  the state stays as loaded.
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


def same_state(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_barrier_wait_limit_reports_timeout_and_keeps_state(gea, mixed):
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const, mixed=mixed)
    s.set_conservative(wl.fields)
    s.step(3)
    assert s.stats()["driver"] == ("mixed_persistent" if mixed else "persistent")
    before = s.get_full()
    steps_before = s.stats()["steps_done"]
    s.set_wait_limit(0)
    with pytest.raises(gea.GeaError) as ei:
        s.step(2)
    assert ei.value.code == gea.GEA_ERR_TIMEOUT
    same_state(s.get_full(), before)
    assert s.stats()["steps_done"] == steps_before
    # the error is sticky until the next set_state
    s.set_wait_limit(-1)
    with pytest.raises(gea.GeaError):
        s.step(1)
    # after a set_state with the default limit the context steps again, bit
    # for bit like an uninterrupted run
    s.set_full(before)
    s.step(2)
    ref = gea.Solver(wl.grid, wl.const, mixed=mixed)
    ref.set_conservative(wl.fields)
    ref.step(5)
    same_state(s.get_full(), ref.get_full())


def test_ensemble_member_timeout(gea):
    """An ensemble member whose barrier gives up reports GEA_ERR_TIMEOUT; the
    other member, with its own barrier, completes its steps."""
    members = []
    for nx in (64, 96):
        grid = W.Grid(nx, 32, 40.0 * nx, 30.0 * 32)
        c = W.Constants(dt=0.2, mu=1.5)
        wl = W.random_flow(grid, c, seed=nx, uamp=2.0)
        s = gea.Solver(grid, c)
        s.set_conservative(wl.fields)
        members.append((s, wl))
    members[0][0].set_wait_limit(0)
    ens = gea.Ensemble([m[0] for m in members])
    ens.step_async(2)
    with pytest.raises(gea.GeaError) as ei:
        ens.sync()
    assert ei.value.code == gea.GEA_ERR_TIMEOUT
    assert members[0][0].stats()["steps_done"] == 0
    assert members[1][0].stats()["steps_done"] == 2
    ens.close()


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("field", ["T", "rho"])
def test_nan_in_state_reports_nonfinite_and_keeps_state(gea, graph, field):
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const, graph=graph)
    s.set_conservative(wl.fields)
    s.step(1)
    st = s.get_full()
    st[field][40, 80] = np.nan
    s.set_full(st)
    with pytest.raises(gea.GeaError) as ei:
        s.step(1)
    assert ei.value.code == gea.GEA_ERR_NONFINITE
    same_state(s.get_full(), st)
    assert s.stats()["status"] == gea.GEA_ERR_NONFINITE


def test_rejected_set_state_keeps_context(gea):
    """A set_state whose arguments are rejected (a missing FULL field) leaves
    the context as it was: same state, and the following steps equal an
    uninterrupted run. A conservative state that fails its check (rho <= 0
    in a cell) leaves no state, so the next step is refused."""
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.step(2)
    before = s.get_full()
    partial = {k: v for k, v in before.items() if k != "T"}
    with pytest.raises(gea.GeaError) as ei:
        s.set_full(partial)
    assert ei.value.code == gea.GEA_ERR_INVAL
    same_state(s.get_full(), before)
    assert s.stats()["steps_done"] == 2
    s.step(1)
    ref = gea.Solver(wl.grid, wl.const)
    ref.set_conservative(wl.fields)
    ref.step(3)
    same_state(s.get_full(), ref.get_full())

    bad = {k: np.array(v, copy=True) for k, v in wl.fields.items()}
    bad["rho"][10, 20] = -1.0
    with pytest.raises(gea.GeaError) as ei:
        s.set_conservative(bad)
    assert ei.value.code == gea.GEA_ERR_INVAL
    with pytest.raises(gea.GeaError) as ei:
        s.step(1)
    assert ei.value.code == gea.GEA_ERR_STATE
