"""Argument checks of the Python binding (no GPU needed).

The library reads or writes a fixed number of elements behind every pointer
it is given (nz x nx values of a state field, n x h x w of a network input,
...). The binding therefore refuses, with GeaError(GEA_ERR_INVAL), any array
of the wrong element type, layout, size or memory before the call is made,
so a caller's mistake cannot turn into an out-of-bounds access on the host
or the GPU. These checks are explicit (not `assert`), so they also hold
under `python -O`.
"""
import numpy as np
import pytest
import torch

from paper_2303_10499_gb300 import gea


def refused(fn):
    with pytest.raises(gea.GeaError) as ei:
        fn()
    assert ei.value.code == gea.GEA_ERR_INVAL


def test_numpy_arrays():
    a = np.zeros((8, 16))
    assert gea._buf(a, 128, "a") == a.ctypes.data
    assert gea._buf(a, 128, "a", device=False) == a.ctypes.data
    refused(lambda: gea._buf(a, 127, "a"))                          # size
    refused(lambda: gea._buf(a.astype(np.float32), 128, "a"))       # element type
    refused(lambda: gea._buf(np.zeros((16, 8)).T, 128, "a"))        # layout
    refused(lambda: gea._buf(a, 128, "a", device=True))             # memory
    refused(lambda: gea._buf(np.zeros(4, dtype=np.int16), 4, "x", "bf16"))
    i = np.zeros(5, dtype=np.int64)
    assert gea._buf(i, 5, "tiles", "int64") == i.ctypes.data


def test_torch_tensors_on_the_host():
    t = torch.zeros((4, 6), dtype=torch.float64)
    assert gea._buf(t, 24, "t") == t.data_ptr()
    assert gea._buf(t, 24, "t", device=False) == t.data_ptr()
    refused(lambda: gea._buf(t, 24, "t", device=True))
    refused(lambda: gea._buf(t.t(), 24, "t"))
    refused(lambda: gea._buf(t, 23, "t"))
    refused(lambda: gea._buf(t.float(), 24, "t"))
    for dt in (torch.bfloat16, torch.int16):
        b = torch.zeros(8, dtype=dt)
        assert gea._buf(b, 8, "x", "bf16") == b.data_ptr()
    refused(lambda: gea._buf(torch.zeros(8), 8, "x", "bf16"))
    refused(lambda: gea._buf([0.0] * 8, 8, "x"))


def test_ensemble_plan_checks_its_arrays():
    refused(lambda: gea.ensemble_plan(np.ones(3), np.array([4, 4]), 16))
    plan = gea.ensemble_plan(np.ones(3), np.array([4, 4, 4]), 16)
    assert plan["used_blocks"] <= 16
