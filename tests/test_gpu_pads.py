"""Pad checking in place of a device memory checker (GEA_FLAG_DEBUG_PADS).

In a debug-pads context every array has NaN-poisoned row padding, an
unused tail and a guard band behind it. These tests run the library's
kernels at sizes whose edges cut through the 32 x 8 tiles and the coarse
multigrid levels (tiny, odd, ragged; FP64 and mixed precision; LES), check
every pad after every kernel launch of eagerly launched steps and after
steps of both drivers, and require the results to equal, bit for bit, those
of the same context without the flag: a kernel that wrote out of bounds
would have changed a pad, and one that read out of bounds would have drawn a
NaN into its results.
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


# nx, nz, Solver keywords, Constants keywords
CASES = {
    "4x4": (4, 4, {}, {}),
    "7x9": (7, 9, {}, {}),
    "17x33": (17, 33, {}, {}),
    "33x17": (33, 17, {}, {}),
    "65x31": (65, 31, {}, {}),
    "96x64_5levels": (96, 64, {"mg_min_cells": 64}, {}),
    "37x23_mixed": (37, 23, {"mixed": True}, {}),
    "64x48_mixed_4levels": (64, 48, {"mixed": True, "mg_min_cells": 48}, {}),
    "40x40_les": (40, 40, {}, {"cs": 0.17, "mu": 0.3}),
}


def workload(nx, nz, ckw):
    grid = W.Grid(nx, nz, 40.0 * nx, 30.0 * nz)
    c = W.Constants(dt=0.2, mu=ckw.pop("mu", 1.5), **ckw)
    return W.random_flow(grid, c, seed=nx * 100 + nz, uamp=3.0, thamp=2.0)


def run(gea, wl, skw, graph, debug):
    s = gea.Solver(wl.grid, wl.const, graph=graph, debug_pads=debug, **skw)
    s.set_conservative(wl.fields)
    reports = []
    for _ in range(2):
        if debug:
            reports.append(s.debug_step())
        else:
            s.profile_step()
    s.step(3)
    return s, reports


@pytest.mark.parametrize("graph", [False, True], ids=["persistent", "graph"])
@pytest.mark.parametrize("case", list(CASES))
def test_no_kernel_touches_a_pad(gea, case, graph):
    nx, nz, skw, ckw = CASES[case]
    wl = workload(nx, nz, dict(ckw))
    s, reports = run(gea, wl, skw, graph, True)
    for r in reports:
        assert r["launch"] == -1 and r["bad"] == 0, r
    final = s.debug_check_pads()
    assert final["bad"] == 0, final
    assert s.stats()["status"] == 0
    ref, _ = run(gea, wl, skw, graph, False)
    got, want = s.get_full(), ref.get_full()
    for k in want:
        assert np.array_equal(got[k], want[k]), k
        assert np.isfinite(got[k]).all(), k


def test_regions_describe_the_layout(gea):
    nx, nz = 96, 64
    wl = workload(nx, nz, {})
    s = gea.Solver(wl.grid, wl.const, mg_min_cells=64, debug_pads=True)
    regs = {r["name"]: r for r in s.debug_pad_regions()}
    pitch = (nx + 1 + 31) // 32 * 32
    assert regs["S0.u"]["pitch"] == pitch and (regs["S0.u"]["rows"], regs["S0.u"]["cols"]) == (nz, nx)
    assert (regs["S1.phix"]["rows"], regs["S1.phix"]["cols"]) == (nz, nx + 1)
    assert (regs["S1.phiz"]["rows"], regs["S1.phiz"]["cols"]) == (nz + 1, nx)
    assert (regs["L3.c"]["rows"], regs["L3.c"]["cols"]) == (8, 12)
    assert (regs["L3.ax"]["rows"], regs["L3.ax"]["cols"]) == (8, 13)
    assert (regs["L4.az"]["rows"], regs["L4.az"]["cols"]) == (5, 6)
    assert regs["gz"]["cols"] == 2 * nz + 1
    # arrays do not overlap: each one's span ends where the next begins
    order = sorted(regs.values(), key=lambda r: r["ptr"])
    for a, b in zip(order, order[1:]):
        assert a["ptr"] + a["span"] * a["elem_bytes"] <= b["ptr"], (a["name"], b["name"])
        # every array ends in a guard band of at least GEA_PAD_GUARD_BYTES
        used = ((a["rows"] - 1) * a["pitch"] + a["cols"]) * a["elem_bytes"]
        assert a["span"] * a["elem_bytes"] - used >= 512
    assert s.debug_check_pads()["bad"] == 0


class _Dev:
    """A device buffer given by its address, for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


@pytest.mark.parametrize("where", ["row_padding", "guard_band", "fp32_row_padding"])
def test_a_changed_pad_is_found_and_named(gea, where):
    """The checker itself: one pad element overwritten from the host (a
    write inside the context's allocation, to a pad no kernel uses) is
    counted and located; poisoning again clears it."""
    import torch
    nx, nz = 33, 17
    wl = workload(nx, nz, {})
    s = gea.Solver(wl.grid, wl.const, debug_pads=True, mixed=where.startswith("fp32"))
    s.set_conservative(wl.fields)
    s.step(1)
    regs = {r["name"]: r for r in s.debug_pad_regions()}
    if where == "row_padding":
        name, row, col = "S0.u", 2, nx + 3
    elif where == "guard_band":
        r = regs["S1.phiz"]
        e = r["span"] - 1
        name, row, col = "S1.phiz", e // r["pitch"], e % r["pitch"]
    else:
        name, row, col = "F.L0.r", 5, nx
    r = regs[name]
    e = row * r["pitch"] + col
    assert e < r["span"] and (row >= r["rows"] or col >= r["cols"])
    torch.cuda.synchronize()
    t = torch.as_tensor(_Dev(r["ptr"] + e * r["elem_bytes"], 1, "<f8" if r["elem_bytes"] == 8 else "<f4"),
                        device="cuda")
    t.fill_(1.0)
    torch.cuda.synchronize()
    rep = s.debug_check_pads()
    assert (rep["bad"], rep["array"], rep["row"], rep["col"]) == (1, name, row, col), rep
    s.debug_poison()
    assert s.debug_check_pads()["bad"] == 0


def test_pad_calls_need_the_flag(gea):
    wl = workload(16, 16, {})
    s = gea.Solver(wl.grid, wl.const)
    with pytest.raises(gea.GeaError) as ei:
        s.debug_check_pads()
    assert ei.value.code == gea.GEA_ERR_INVAL
