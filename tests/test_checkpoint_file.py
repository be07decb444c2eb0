"""Checkpoint files of the full state (write_checkpoint / read_checkpoint):
the arrays come back bit for bit with their grid, constants and step count,
and a file of another grid, another format version or a field of the wrong
shape is refused. (The resumed run continuing bit for bit on the GPU is in
test_gpu_parity.py.)"""
import json

import numpy as np
import pytest

from paper_2303_10499_gb300 import gea
from paper_2303_10499_gb300 import workloads as W


def fake_state(nx, nz, seed=0):
    rng = np.random.default_rng(seed)
    st = {k: rng.standard_normal((nz, nx)) for k in ("rho", "u", "w", "T", "h", "p", "pp", "pold")}
    st["phix"] = rng.standard_normal((nz, nx + 1))
    st["phiz"] = rng.standard_normal((nz + 1, nx))
    return st


def test_roundtrip(tmp_path):
    grid = W.Grid(24, 16, 240.0, 160.0)
    const = W.Constants(dt=0.2, mu=1.5, cs=0.17)
    st = fake_state(24, 16)
    path = str(tmp_path / "ck.npz")
    gea.write_checkpoint(path, grid, const, st, steps_done=42)
    ck = gea.read_checkpoint(path, grid)
    assert ck["steps_done"] == 42 and ck["grid"] == [24, 16, 240.0, 160.0]
    assert ck["constants"]["dt"] == 0.2 and ck["constants"]["cs"] == 0.17
    assert set(ck["state"]) == set(st)
    for k in st:
        assert ck["state"][k].dtype == np.float64 and np.array_equal(ck["state"][k], st[k]), k


def test_refuses_mismatches(tmp_path):
    grid = W.Grid(24, 16, 240.0, 160.0)
    const = W.Constants()
    path = str(tmp_path / "ck.npz")
    gea.write_checkpoint(path, grid, const, fake_state(24, 16))
    with pytest.raises(gea.GeaError):
        gea.read_checkpoint(path, W.Grid(32, 16, 320.0, 160.0))
    bad = fake_state(24, 16)
    bad["phix"] = bad["phix"][:, :-1]
    gea.write_checkpoint(path, grid, const, bad)
    with pytest.raises(gea.GeaError):
        gea.read_checkpoint(path)
    # another format version
    with np.load(path) as z:
        arrays = {k: z[k] for k in z.files}
    meta = json.loads(str(arrays.pop("meta")))
    meta["version"] = 99
    with open(path, "wb") as f:
        np.savez(f, meta=np.array(json.dumps(meta)), **arrays)
    with pytest.raises(gea.GeaError):
        gea.read_checkpoint(path)
