"""The C-ABI library builds for sm_103a and exports every entry point that
include/gea.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    """Every function declared in include/*.h."""
    out = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            out.update(re.findall(r"\b(gea_[a-z_0-9]+)\s*\(", src))
    return sorted(out)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("gea_create", "gea_set_state", "gea_step", "gea_get_state", "gea_destroy"):
        assert s in syms


def test_library_builds_and_exports_every_symbol():
    from paper_2303_10499_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_struct_sizes_match_header():
    """The ctypes structs mirror the C structs (checked with the host C
    compiler against include/gea.h)."""
    import subprocess
    import tempfile
    from paper_2303_10499_gb300 import gea
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "gea.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gea_grid), sizeof(gea_constants),
 sizeof(gea_state_view), sizeof(gea_stats), sizeof(gea_pad_region), sizeof(gea_pad_report)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(gea._Grid), ctypes.sizeof(gea._Const),
                     ctypes.sizeof(gea._View), ctypes.sizeof(gea._Stats),
                     ctypes.sizeof(gea._PadRegion), ctypes.sizeof(gea._PadReport)]


def test_binding_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W
    wl = W.get("bubble160x80")
    with pytest.raises(gea.GeaError):
        gea.Solver(wl.grid, wl.const)


def test_create_rejects_bad_flags_and_mixed_tolerance():
    """Argument checks run before any CUDA call, so they answer on a
    machine without a GPU too."""
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W
    wl = W.get("bubble160x80")
    for kw in (dict(mixed=True, mp_rtol=2.0), dict(mixed=True, mp_rtol=1e-9),
               dict(mixed=True, mp_rtol=-1e-3)):
        with pytest.raises(gea.GeaError) as ei:
            gea.Solver(wl.grid, wl.const, **kw)
        assert ei.value.code == gea.GEA_ERR_INVAL, kw
    # more tiles (32 x 8 cells) than the grid sums' 4096 groups of 1024
    # blocks cover, though within the cell limit: 33 columns are two tiles wide
    big = W.Grid(33, (1 << 30) // 33 // 8 * 8, 33.0, 1e6)
    with pytest.raises(gea.GeaError) as ei:
        gea.Solver(big, wl.const)
    assert ei.value.code == gea.GEA_ERR_INVAL


def test_grid3_struct_matches_header():
    import subprocess
    import tempfile
    from paper_2303_10499_gb300 import gea
    code = r'''
#include <stdio.h>
#include "gea3d.h"
int main(void){printf("%zu\n", sizeof(gea3d_grid)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        size = int(subprocess.check_output([exe]))
    assert size == ctypes.sizeof(gea._Grid3)


def test_create3_rejects_bad_arguments():
    """gea3d_create validates sizes and constants before any CUDA call."""
    from paper_2303_10499_gb300 import gea
    from paper_2303_10499_gb300 import workloads as W
    c = W.Constants(dt=0.2)
    for g in (W.Grid3(3, 8, 8, 1.0, 1.0, 1.0), W.Grid3(8, 8, 2, 1.0, 1.0, 1.0),
              W.Grid3(8, 8, 8, 1.0, -1.0, 1.0)):
        with pytest.raises(gea.GeaError) as ei:
            gea.Solver3D(g, c)
        assert ei.value.code == gea.GEA_ERR_INVAL
    # only GEA_FLAG_MIXED, with 1e-7 <= mp_rtol < 1 (or 0), and mp_rtol only with it
    for kw in (dict(mixed=True, mp_rtol=2.0), dict(mixed=True, mp_rtol=1e-9), dict(mp_rtol=1e-4)):
        with pytest.raises(gea.GeaError) as ei:
            gea.Solver3D(W.Grid3(8, 8, 8, 1.0, 1.0, 1.0), W.Constants(dt=0.2), **kw)
        assert ei.value.code == gea.GEA_ERR_INVAL, kw
    # LES needs Pr = 1 (one viscosity field for momentum and enthalpy), and cs >= 0
    for kw in (dict(cs=0.17, Pr=0.7), dict(cs=-0.1)):
        with pytest.raises(gea.GeaError) as ei:
            gea.Solver3D(W.Grid3(8, 8, 8, 1.0, 1.0, 1.0), W.Constants(dt=0.2, **kw))
        assert ei.value.code == gea.GEA_ERR_INVAL, kw
