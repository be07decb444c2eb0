"""gea_mass_energy_noalloc: mass and energy totals with no device allocation.

Some callers cannot allocate device memory (their memory belongs to a
framework's caching allocator or a fixed arena, or they must not call
cudaMalloc). For them the library offers one context-free entry point whose
reduction scratch is a fixed device array inside the library. This test
calls it through the C ABI twice in a row on a state produced by the solver
and checks both results against the context's own diagnostics
(gea_get_diag), which allocate their scratch with the context.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2303_10499_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_diagnostics_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea

    wl = W.get("bubble160x80")
    s = gea.Solver(wl.grid, wl.const)
    s.set_conservative(wl.fields)
    s.step(5)
    _, mass, energy = s.diagnostics(wl.theta_bar)
    st = s.get_full()
    dev = {k: torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in ("rho", "u", "w", "T")}
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")

    lib = gea.library()
    f = lib.gea_mass_energy_noalloc
    f.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double,
                  C.c_double] + [C.c_void_p] * 6
    f.restype = C.c_int
    c = wl.const
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        out.fill_(float("nan"))
        rc = f(wl.grid.nx, wl.grid.nz, wl.grid.lx, wl.grid.lz, c.cp, c.R, c.g,
               dev["rho"].data_ptr(), dev["u"].data_ptr(), dev["w"].data_ptr(),
               dev["T"].data_ptr(), out.data_ptr(), stream)
        assert rc == gea.GEA_OK
        torch.cuda.synchronize()
        m2, e2 = out.cpu().tolist()
        # same sums in another block order: agreement to 1e-12 relative
        assert abs(m2 - mass) <= 1e-12 * abs(mass), (m2, mass)
        assert abs(e2 - energy) <= 1e-12 * abs(energy), (e2, energy)
        results.append((m2, e2))
    assert results[0] == results[1]

    # sizes beyond the fixed scratch are rejected before anything is launched
    rc = f(4096, 4097, 1.0, 1.0, c.cp, c.R, c.g, dev["rho"].data_ptr(), dev["u"].data_ptr(),
           dev["w"].data_ptr(), dev["T"].data_ptr(), out.data_ptr(), stream)
    assert rc == gea.GEA_ERR_INVAL
