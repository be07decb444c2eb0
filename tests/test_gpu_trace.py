"""Phase trace of the persistent step kernel (gea_set_trace).

The trace records, per grid barrier of a step, every block's arrival and
release. A barrier releases no block before the last one has arrived, so
every release of barrier k comes after every arrival at it; barrier k + 1
follows barrier k in every block; the number of barriers is the step's
phase count, which follows from its Jacobi sweeps and CG iterations
(Section 3: Steps 1-2, then per PISO corrector the right-hand side, the
preconditioned CG and the correction). Tracing must not change the step.
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


def expected_barriers(st, n_corr):
    """Grid barriers of one FP64 persistent step with a one-level
    preconditioner: Step 1 with the first momentum sweep, the other sweeps,
    Step 2 with the first enthalpy sweep, the other sweeps, the EOS update
    with H(u); per corrector H(u) (after the first), the right-hand side, the
    first preconditioning (when the solve is not already converged), two per
    CG iteration, the correction (but the last, which the step end covers);
    the step end."""
    n = 1 + (st["jac_u"] - 1) + 1 + (st["jac_h"] - 1) + 1
    for c in range(n_corr):
        its = st["cg_iters"][c]
        n += (1 if c > 0 else 0) + 1 + (1 if its > 0 else 0) + 2 * its
        n += 1 if c + 1 < n_corr else 0
    return n + 1


def test_trace_of_a_persistent_step(gea):
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    ref = gea.Solver(wl.grid, wl.const)
    for x in (s, ref):
        x.set_conservative(wl.fields)
        x.step(2)
    assert s.stats()["driver"] == "persistent"
    tr = s.trace_step()
    ref.step(1)
    st = s.stats()
    assert st["status"] == 0
    nb, nbar = tr["blocks"], tr["barriers"]
    assert nb > 0 and tr["arrive"].shape == (nbar, nb)
    assert nbar == expected_barriers(st, wl.const.n_corr), (nbar, st)
    a, r = tr["arrive"], tr["release"]
    assert (tr["entry"] >= 0).all() and (a[0] >= tr["entry"]).all()
    assert (r >= a).all()
    # no release before the last arrival at the same barrier
    assert (r.min(axis=1) >= a.max(axis=1)).all()
    # the next barrier's arrival after this one's release, block by block
    assert (a[1:] >= r[:-1]).all()
    assert ((tr["sm"] >= 0) & (tr["sm"] < 1024)).all()
    # the traced step is the same step
    g, h = s.get_full(), ref.get_full()
    for k in ("rho", "u", "w", "T", "pp", "phix", "phiz"):
        assert np.array_equal(g[k], h[k]), k
    # tracing is off again
    s.step(1)
    ref.step(1)
    assert np.array_equal(s.get_full()["pp"], ref.get_full()["pp"])
    s.close()
    ref.close()


def test_trace_rejects_bad_arguments(gea):
    import ctypes as C
    import torch
    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    nb = C.c_int32(0)
    assert s.lib.gea_set_trace(s.h, None, 0, 0, C.byref(nb)) == gea.GEA_OK and nb.value > 0
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    # too small for 2 x (1 + 1) x blocks values
    assert s.lib.gea_set_trace(s.h, C.c_void_p(buf.data_ptr()), 1, 16, None) == gea.GEA_ERR_INVAL
    assert s.lib.gea_set_trace(s.h, C.c_void_p(buf.data_ptr()), 0, 16, None) == gea.GEA_ERR_INVAL
    s.close()
