"""Thin ctypes binding of the CUDA library (include/gea.h).

Argument marshalling only: every step of the time step runs in the
library's kernels. There is no fallback: if the shared library is missing,
or no CUDA device is present, the calls raise.

Arrays are float64 with the layouts of include/gea.h: cell fields (nz, nx),
phix (nz, nx+1), phiz (nz+1, nx). Host arrays are numpy arrays; device
arrays may be torch CUDA tensors (their data pointers are passed through).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional

import numpy as np

from .build import LIB

GEA_OK, GEA_ERR_INVAL, GEA_ERR_NOMEM, GEA_ERR_CUDA, GEA_ERR_NOCONV, GEA_ERR_NONFINITE, \
    GEA_ERR_STATE, GEA_ERR_TIMEOUT = range(8)
STATE_CONSERVATIVE, STATE_FULL = 0, 1
FLAG_GRAPH, FLAG_MIXED, FLAG_KEEP_R0, FLAG_DEBUG_PADS = 1, 2, 4, 8
PAD_POISON64, PAD_POISON32 = 0x7FF4BAD0DEAD0BAD, 0x7FA0BAD0
MEM_HOST, MEM_DEVICE = 0, 1
FIELDS = {"rho1": 0, "u1": 1, "w1": 2, "h1": 3, "rho2": 4, "Hx": 5, "Hz": 6, "b": 7,
          "Dx": 8, "Dz": 9, "hc": 10, "hax": 11, "haz": 12, "r0": 13}
FULL_FIELDS = ("rho", "u", "w", "T", "h", "p", "pp", "pold", "phix", "phiz", "Kold")
READING_K_LAGGED = 1   # gea_constants.reading_flags: the literal K^{n-1} of eq. step3_sd
# tile shapes of the persistent kernels (gea_set_tile_shape): cells in x by z
TILE_SHAPES = {0: "32x8", 1: "16x16", 2: "64x4"}


class GeaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gea error {code}: {msg}")
        self.code = code


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("lx", C.c_double), ("lz", C.c_double)]


class _Const(C.Structure):
    _fields_ = [("R", C.c_double), ("cp", C.c_double), ("g", C.c_double), ("p0", C.c_double),
                ("mu", C.c_double), ("Pr", C.c_double), ("dt", C.c_double),
                ("n_corr", C.c_int32), ("jac_rtol", C.c_double), ("jac_maxit", C.c_int32),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32),
                ("mg_min_cells", C.c_int32), ("flags", C.c_int32), ("mp_rtol", C.c_double), ("cs", C.c_double),
                ("reading_flags", C.c_uint32)]


class _View(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mem", C.c_int32)] + [
        (n, C.c_void_p) for n in ("rho", "rhou", "rhow", "rhoe", "u", "w", "T", "h", "p", "pp",
                                  "pold", "phix", "phiz", "Kold")]


class _Grid3(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("jac_u", C.c_int32), ("jac_h", C.c_int32),
                ("cg_iters", C.c_int32 * 4), ("cg_relres", C.c_double * 4),
                ("status", C.c_int32), ("mg_levels", C.c_int32), ("launches", C.c_int64),
                ("driver", C.c_int32), ("reserved", C.c_int32)]


class _KTime(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_int32), ("cells", C.c_int64),
                ("ms", C.c_double)]


class _PadRegion(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("ptr", C.c_void_p), ("elem_bytes", C.c_int32),
                ("pitch", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32), ("span", C.c_int64)]


class _PadReport(C.Structure):
    _fields_ = [("bad", C.c_int64), ("launch", C.c_int32), ("kernel", C.c_char * 40),
                ("array", C.c_char * 24), ("row", C.c_int32), ("col", C.c_int32)]


_lib = None


def library() -> C.CDLL:
    """Load libgea.so (built by paper_2303_10499_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library {LIB} is not built; call "
                               "paper_2303_10499_gb300.build.build() first")
        lib = C.CDLL(LIB)
        P = C.c_void_p
        lib.gea_create.argtypes = [C.POINTER(_Grid), C.POINTER(_Const), C.POINTER(P)]
        lib.gea_set_stream.argtypes = [P, P]
        lib.gea_set_state.argtypes = [P, C.POINTER(_View)]
        lib.gea_step.argtypes = [P, C.c_int32]
        lib.gea_step_async.argtypes = [P, C.c_int32]
        lib.gea_sync.argtypes = [P]
        lib.gea_get_state.argtypes = [P, C.POINTER(_View)]
        lib.gea_get_diag.argtypes = [P, P, P, P, P]
        lib.gea_get_stats.argtypes = [P, C.POINTER(_Stats)]
        lib.gea_get_field.argtypes = [P, C.c_int32, P]
        lib.gea_last_pressure_ms.argtypes = [P]
        lib.gea_last_pressure_ms.restype = C.c_double
        lib.gea_profile_step.argtypes = [P, C.POINTER(_KTime), C.c_int32, C.POINTER(C.c_int32)]
        lib.gea_debug_pad_regions.argtypes = [P, C.POINTER(_PadRegion), C.c_int32, C.POINTER(C.c_int32)]
        lib.gea_debug_poison.argtypes = [P]
        lib.gea_debug_check_pads.argtypes = [P, C.POINTER(_PadReport)]
        lib.gea_debug_step.argtypes = [P, C.POINTER(_PadReport)]
        lib.gea_last_error.argtypes = [P]
        lib.gea_last_error.restype = C.c_char_p
        lib.gea_destroy.argtypes = [P]
        lib.gea_destroy.restype = None
        I = C.c_int32
        lib.gea_conv3x3.argtypes = [I, I, I, I, I, I, I, P, P, P, P, P, P, P]
        lib.gea_attach_net.argtypes = [P, P, I]
        lib.gea_set_tiles_per_block.argtypes = [P, I]
        lib.gea_set_wait_limit.argtypes = [P, C.c_int64]
        lib.gea_set_trace.argtypes = [P, P, I, C.c_int64, C.POINTER(I)]
        lib.gea_set_tile_shape.argtypes = [P, I]
        lib.gea_set_smoother_weight.argtypes = [P, C.c_double]
        lib.gea_apply_precond.argtypes = [P, P, P]
        lib.gea_probe_fma.argtypes = [I, I, I, P, P]
        lib.gea_probe_barrier.argtypes = [I, I, I, P, P]
        lib.gea_ensemble_create.argtypes = [C.POINTER(P), I, P, C.POINTER(P)]
        lib.gea_ensemble_set_stream.argtypes = [P, P]
        lib.gea_ensemble_blocks.argtypes = [P, I]
        lib.gea_ensemble_plan.argtypes = [P, P, I, I, P, P, C.POINTER(I), C.POINTER(I)]
        lib.gea_ensemble_step.argtypes = [P, I]
        lib.gea_ensemble_set_graph.argtypes = [P, I]
        lib.gea_ensemble_sync.argtypes = [P]
        lib.gea_ensemble_destroy.argtypes = [P]
        lib.gea_ensemble_destroy.restype = None
        lib.gea_net_param_count.restype = C.c_int64
        lib.gea_net_layout.argtypes = [P]
        lib.gea_net_create.argtypes = [I, I, I, I, C.POINTER(P)]
        lib.gea_net_set_stream.argtypes = [P, P]
        lib.gea_net_set_params.argtypes = [P, P, I]
        lib.gea_net_get_params.argtypes = [P, P, I]
        lib.gea_net_forward.argtypes = [P, I, I, I, P, P]
        lib.gea_net_energy.argtypes = [P, P, P, P, P, C.POINTER(C.c_float)]
        lib.gea_net_backward.argtypes = [P, P, P]
        lib.gea_net_adam.argtypes = [P, P, C.c_float]
        lib.gea_net_train_step.argtypes = [P, I, I, I, P, P, P, P, C.c_float, C.POINTER(C.c_float)]
        lib.gea_net_destroy.argtypes = [P]
        lib.gea3d_create.argtypes = [C.POINTER(_Grid3), C.POINTER(_Const), C.POINTER(P)]
        lib.gea3d_set_stream.argtypes = [P, P]
        lib.gea3d_set_conservative.argtypes = [P, P, P, P, P, P, I]
        lib.gea3d_step_async.argtypes = [P, I]
        lib.gea3d_sync.argtypes = [P]
        lib.gea3d_step.argtypes = [P, I]
        lib.gea3d_get_state.argtypes = [P, P, P, P, P, P, P, P, I]
        lib.gea3d_get_stats.argtypes = [P, C.POINTER(_Stats)]
        lib.gea3d_get_diag.argtypes = [P, P, P, P, P]
        lib.gea3d_profile_step.argtypes = [P, C.POINTER(_KTime), I, C.POINTER(I)]
        lib.gea3d_last_error.argtypes = [P]
        lib.gea3d_last_error.restype = C.c_char_p
        lib.gea3d_destroy.argtypes = [P]
        lib.gea_net_destroy.restype = None
        _lib = lib
    return _lib


def _buf(a, count: int, what: str, dtype: str = "float64", device: Optional[bool] = None) -> int:
    """Data pointer of `a`, a numpy array or a torch tensor, after checking
    that it is C-contiguous, of element type `dtype` ("float64", "float32",
    "int32"; "bf16" for bfloat16 bit patterns: torch.bfloat16 or 16-bit
    integers), holds exactly `count` elements and, with device True/False,
    lives on the GPU/the host. The library reads or writes that many elements
    behind the pointer, so anything else raises GeaError(GEA_ERR_INVAL)."""
    if isinstance(a, np.ndarray):
        ok = (dtype != "bf16" and a.dtype == np.dtype(dtype) and a.flags.c_contiguous and a.size == count
              and device is not True)
        if not ok:
            raise GeaError(GEA_ERR_INVAL, f"{what}: need a C-contiguous {dtype} array of {count} elements"
                           f"{' on the device' if device else ''}, got {a.dtype} {a.shape}")
        return a.ctypes.data
    kind = str(getattr(a, "dtype", type(a).__name__))
    types = ("torch.bfloat16", "torch.int16", "torch.uint16") if dtype == "bf16" else ("torch." + dtype,)
    ok = (kind in types and hasattr(a, "data_ptr") and a.is_contiguous() and a.numel() == count
          and (device is None or bool(a.is_cuda) == device))
    if not ok:
        shape = tuple(getattr(a, "shape", ()))
        where = {None: "", True: " on the device", False: " on the host"}[device]
        raise GeaError(GEA_ERR_INVAL, f"{what}: need a contiguous {dtype} tensor of {count} elements{where}, "
                       f"got {kind} {shape}")
    return a.data_ptr()


def _addr(a, count: int, what: str) -> int:
    """Data pointer of a float64 field (host or device) of `count` values."""
    return _buf(a, count, what)


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def ensemble_plan(weights, tiles, blocks: int) -> Dict:
    """The block partition of an ensemble launch (gea_ensemble_plan),
    computed on the host: per member its blocks and group, the number of
    groups and of blocks used."""
    lib = library()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    t = np.ascontiguousarray(tiles, dtype=np.int64)
    n = w.size
    nb = np.zeros(n, dtype=np.int32)
    grp = np.zeros(n, dtype=np.int32)
    ng, used = C.c_int32(0), C.c_int32(0)
    rc = lib.gea_ensemble_plan(_buf(w, n, "weights"), _buf(t, n, "tiles", "int64"), n, int(blocks),
                               nb.ctypes.data, grp.ctypes.data, C.byref(ng), C.byref(used))
    if rc != GEA_OK:
        raise GeaError(rc, "gea_ensemble_plan failed")
    return {"blocks": nb, "group": grp, "groups": ng.value, "used_blocks": used.value}


CHECKPOINT_VERSION = 1


def write_checkpoint(path: str, grid, const, state: Dict[str, np.ndarray], steps_done: int = 0) -> None:
    """Write a FULL state (Solver.get_full) to `path` as an .npz file: the
    state arrays, and as JSON the grid (nx, nz, lx, lz), the constants' fields
    and the number of steps done. Reading it back and setting it continues
    the run bit for bit (gea_set_state with the FULL view)."""
    import dataclasses
    import json
    meta = {"version": CHECKPOINT_VERSION, "grid": [int(grid.nx), int(grid.nz), float(grid.lx), float(grid.lz)],
            "constants": dataclasses.asdict(const) if dataclasses.is_dataclass(const) else dict(vars(const)),
            "steps_done": int(steps_done), "fields": sorted(state)}
    arrays = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in state.items()}
    with open(path, "wb") as f:
        np.savez(f, meta=np.array(json.dumps(meta)), **arrays)


def read_checkpoint(path: str, grid=None) -> Dict:
    """Read a checkpoint written by write_checkpoint: {"state", "grid",
    "constants", "steps_done"}. With `grid`, the checkpoint must be of that
    grid (GeaError GEA_ERR_INVAL otherwise); the arrays' shapes are checked
    against the grid either way."""
    import json
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        if meta.get("version") != CHECKPOINT_VERSION:
            raise GeaError(GEA_ERR_INVAL, f"checkpoint version {meta.get('version')} is not {CHECKPOINT_VERSION}")
        state = {k: np.array(z[k]) for k in meta["fields"]}
    nx, nz, lx, lz = meta["grid"]
    if grid is not None and (nx, nz) != (grid.nx, grid.nz):
        raise GeaError(GEA_ERR_INVAL, f"checkpoint of a {nx} x {nz} grid, not {grid.nx} x {grid.nz}")
    shapes = {"phix": (nz, nx + 1), "phiz": (nz + 1, nx)}
    for k, v in state.items():
        if v.shape != shapes.get(k, (nz, nx)):
            raise GeaError(GEA_ERR_INVAL, f"checkpoint field {k} has shape {v.shape}")
    return {"state": state, "grid": meta["grid"], "constants": meta["constants"],
            "steps_done": meta["steps_done"]}


class Solver:
    """One context of the library: a grid, its constants and device state."""

    def __init__(self, grid, const, mg_min_cells: int = 0, stream=None, graph: bool = False,
                 mixed: bool = False, mp_rtol: float = 0.0, keep_r0: bool = False,
                 debug_pads: bool = False):
        """graph=True runs each step as a CUDA graph of per-phase kernels
        instead of the persistent cooperative kernel (GEA_FLAG_GRAPH).
        mixed=True selects the mixed-precision step (GEA_FLAG_MIXED): FP32
        inner solves for FP64 increments, to ||r|| <= mp_rtol ||r0|| (0: the
        library default). debug_pads=True lays the arrays out with guard
        bands and NaN-poisoned pads (GEA_FLAG_DEBUG_PADS; debug_* methods)."""
        self.lib = library()
        self.grid, self.const = grid, const
        g = _Grid(grid.nx, grid.nz, grid.lx, grid.lz)
        flags = (FLAG_GRAPH if graph else 0) | (FLAG_MIXED if mixed else 0) | \
            (FLAG_KEEP_R0 if keep_r0 else 0) | (FLAG_DEBUG_PADS if debug_pads else 0)
        c = _Const(const.R, const.cp, const.g, const.p0, const.mu, const.Pr, const.dt,
                   const.n_corr, const.jac_rtol, const.jac_maxit, const.cg_rtol, const.cg_maxit,
                   mg_min_cells, flags, mp_rtol, getattr(const, "cs", 0.0),
                   getattr(const, "reading_flags", 0))
        h = C.c_void_p()
        rc = self.lib.gea_create(C.byref(g), C.byref(c), C.byref(h))
        if rc != GEA_OK:
            raise GeaError(rc, "gea_create failed")
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            self.lib.gea_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != GEA_OK:
            msg = self.lib.gea_last_error(self.h)
            raise GeaError(rc, msg.decode() if msg else "")

    def _count(self, field: str) -> int:
        """Values of a state field: nz x (nx + 1) x-face fluxes, (nz + 1) x nx
        z-face fluxes, nz x nx cell values otherwise."""
        nx, nz = self.grid.nx, self.grid.nz
        return {"phix": nz * (nx + 1), "phiz": (nz + 1) * nx}.get(field, nz * nx)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer or None."""
        self._stream = stream if hasattr(stream, "cuda_stream") else None
        s = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.gea_set_stream(self.h, C.c_void_p(s or 0)))

    # -- state -------------------------------------------------------------
    def set_conservative(self, fields: Dict):
        v = _View()
        v.kind = STATE_CONSERVATIVE
        v.mem = MEM_DEVICE if _is_device(fields["rho"]) else MEM_HOST
        for k in ("rho", "rhou", "rhow", "rhoe"):
            setattr(v, k, _addr(fields[k], self._count(k), k))
        self._check(self.lib.gea_set_state(self.h, C.byref(v)))

    def set_full(self, state: Dict):
        v = _View()
        v.kind = STATE_FULL
        v.mem = MEM_DEVICE if _is_device(state["rho"]) else MEM_HOST
        for k in FULL_FIELDS:
            # Kold (K^{n-1}) is part of the state only with READING_K_LAGGED
            setattr(v, k, _addr(state[k], self._count(k), k) if k in state else None)
        self._check(self.lib.gea_set_state(self.h, C.byref(v)))

    def full_fields(self):
        """The fields of this context's FULL state: K^{n-1} (Kold) belongs to it
        only with READING_K_LAGGED."""
        lagged = getattr(self.const, "reading_flags", 0) & READING_K_LAGGED
        return FULL_FIELDS if lagged else FULL_FIELDS[:-1]

    def save_checkpoint(self, path: str) -> None:
        """The full state (get_full) with the grid, constants and steps done,
        as an .npz file (write_checkpoint)."""
        write_checkpoint(path, self.grid, self.const, self.get_full(), self.stats()["steps_done"])

    def load_checkpoint(self, path: str) -> Dict:
        """Set the full state from a checkpoint of this grid (read_checkpoint);
        the steps that follow continue the checkpointed run bit for bit.
        Returns the checkpoint's metadata."""
        ck = read_checkpoint(path, self.grid)
        self.set_full(ck["state"])
        return ck

    def get_full(self, out: Optional[Dict] = None) -> Dict[str, np.ndarray]:
        nx, nz = self.grid.nx, self.grid.nz
        fields = self.full_fields()
        if out is None:
            out = {k: np.empty((nz, nx)) for k in fields}
            out["phix"] = np.empty((nz, nx + 1))
            out["phiz"] = np.empty((nz + 1, nx))
        v = _View()
        v.kind = STATE_FULL
        v.mem = MEM_DEVICE if _is_device(out["rho"]) else MEM_HOST
        for k in fields:
            setattr(v, k, _addr(out[k], self._count(k), k))
        self._check(self.lib.gea_get_state(self.h, C.byref(v)))
        return out

    def get_conservative(self, out: Optional[Dict] = None) -> Dict[str, np.ndarray]:
        """rho, rho u, rho w, rho e of the current state, computed by the
        library on the device (gea_get_state with kind CONSERVATIVE)."""
        nx, nz = self.grid.nx, self.grid.nz
        if out is None:
            out = {k: np.empty((nz, nx)) for k in ("rho", "rhou", "rhow", "rhoe")}
        v = _View()
        v.kind = STATE_CONSERVATIVE
        v.mem = MEM_DEVICE if _is_device(out["rho"]) else MEM_HOST
        for k in ("rho", "rhou", "rhow", "rhoe"):
            setattr(v, k, _addr(out[k], self._count(k), k))
        self._check(self.lib.gea_get_state(self.h, C.byref(v)))
        return out

    # -- stepping ----------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self.lib.gea_step(self.h, int(n)))

    def step_async(self, n: int = 1):
        self._check(self.lib.gea_step_async(self.h, int(n)))

    def sync(self):
        self._check(self.lib.gea_sync(self.h))

    # -- diagnostics -------------------------------------------------------
    def diagnostics(self, theta_bar: np.ndarray):
        tb = np.ascontiguousarray(theta_bar, dtype=np.float64)
        th = np.empty((self.grid.nz, self.grid.nx))
        m = C.c_double()
        e = C.c_double()
        self._check(self.lib.gea_get_diag(self.h, _buf(tb, self.grid.nz, "theta_bar", device=False),
                                          th.ctypes.data, C.addressof(m), C.addressof(e)))
        return th, m.value, e.value

    def stats(self) -> Dict:
        s = _Stats()
        self._check(self.lib.gea_get_stats(self.h, C.byref(s)))
        n = self.const.n_corr
        return {"steps_done": s.steps_done, "jac_u": s.jac_u, "jac_h": s.jac_h,
                "cg_iters": list(s.cg_iters)[:n], "cg_relres": list(s.cg_relres)[:n],
                "status": s.status, "mg_levels": s.mg_levels, "launches": s.launches,
                "driver": {0: "graph", 1: "persistent", 2: "mixed", 3: "mixed_persistent"}[s.driver]}

    def field(self, name: str) -> np.ndarray:
        nx, nz = self.grid.nx, self.grid.nz
        shape = {"Dx": (nz, nx + 1), "Dz": (nz + 1, nx), "hax": (nz, nx + 1),
                 "haz": (nz + 1, nx)}.get(name, (nz, nx))
        out = np.empty(shape)
        self._check(self.lib.gea_get_field(self.h, FIELDS[name], out.ctypes.data))
        return out

    def apply_precond(self, r: np.ndarray) -> np.ndarray:
        """z = M r with the pressure solve's multigrid preconditioner of the
        last completed step (gea_apply_precond)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty((self.grid.nz, self.grid.nx))
        self._check(self.lib.gea_apply_precond(self.h, _buf(r, z.size, "r", device=False), z.ctypes.data))
        return z

    def set_wait_limit(self, polls: int):
        """Grid-barrier poll limit of the persistent kernels (gea_set_wait_limit;
        < 0: the default)."""
        self._check(self.lib.gea_set_wait_limit(self.h, int(polls)))

    def trace_step(self, max_barriers: int = 512) -> Dict:
        """One step of the persistent driver with its phase trace
        (gea_set_trace). Returns the grid's blocks, each block's SM and entry
        time, and per grid barrier of the step (rows) every block's arrival
        and release (columns), in ns after the earliest block entry; only the
        barriers the step passed are kept."""
        import torch
        nb = C.c_int32(0)
        self._check(self.lib.gea_set_trace(self.h, None, 0, 0, C.byref(nb)))
        if nb.value <= 0:
            raise GeaError(GEA_ERR_INVAL, "the phase trace needs the persistent driver")
        cap = 2 * (max_barriers + 1) * nb.value
        buf = torch.zeros(cap, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        self._check(self.lib.gea_set_trace(self.h, C.c_void_p(buf.data_ptr()), int(max_barriers), cap,
                                           C.byref(nb)))
        try:
            self.step(1)
        finally:
            self.lib.gea_set_trace(self.h, None, 0, 0, None)
        t = buf.cpu().numpy().view(np.uint64).reshape(max_barriers + 1, nb.value, 2)
        entry = t[0, :, 0].astype(np.int64)
        used = int(np.count_nonzero(t[1:, 0, 0]))
        t0 = entry.min()
        arrive = t[1:1 + used, :, 0].astype(np.int64) - t0
        release = t[1:1 + used, :, 1].astype(np.int64) - t0
        return {"blocks": nb.value, "sm": t[0, :, 1].astype(np.int64), "entry": entry - t0,
                "arrive": arrive, "release": release, "barriers": used}

    def pressure_ms(self) -> float:
        return float(self.lib.gea_last_pressure_ms(self.h))

    def attach_net(self, net, mode: int = 1):
        """Use a Net in the pressure solves: as their learned initial guess
        (mode 1), as the preconditioner of a flexible CG in place of the
        multigrid V-cycle (mode 2, FP64 step only), or both (mode 3); mode 0
        (net None) detaches it."""
        self._check(self.lib.gea_attach_net(self.h, net.h if net is not None else None, mode))
        self._net = net if mode else None   # keep it alive while attached

    def set_smoother_weight(self, omega: float):
        """Weight of the preconditioner's Jacobi sweeps (gea_set_smoother_weight)."""
        self._check(self.lib.gea_set_smoother_weight(self.h, float(omega)))

    def set_tiles_per_block(self, n: int):
        """Tiles a block walks in the per-phase kernels with a grid reduction
        (gea_set_tiles_per_block; 0: the size rule)."""
        self._check(self.lib.gea_set_tiles_per_block(self.h, int(n)))

    def tune_tiles(self, candidates=(1, 2, 4, 8), steps: int = 3) -> Dict:
        """Tile-column autotuner of the graph driver's per-phase kernels: for
        each candidate number of tiles a block walks, one untimed step (which
        records the step graph) and `steps` timed steps (gea_step
        synchronises, so host time brackets the device work); keeps the
        fastest. The state advances by len(candidates) x (steps + 1) steps."""
        import time
        times = {}
        for n in candidates:
            self.set_tiles_per_block(n)
            self.step(1)
            t0 = time.perf_counter()
            self.step(steps)
            times[int(n)] = (time.perf_counter() - t0) / steps * 1e3
        best = min(times, key=times.get)
        self.set_tiles_per_block(best)
        return {"ms_per_step": times, "tiles_per_block": best}

    def set_tile_shape(self, shape: int):
        """Tile shape of the persistent kernels (gea_set_tile_shape): one of
        TILE_SHAPES' keys."""
        self._check(self.lib.gea_set_tile_shape(self.h, int(shape)))
        self.tile_shape = int(shape)

    def tune_tile_shape(self, candidates=None, steps: int = 3) -> Dict:
        """Tile-shape autotuner of the persistent kernels: for each candidate
        shape, one untimed step and `steps` steps timed with CUDA events on
        the context's stream; keeps the fastest. The state advances by
        len(candidates) x (steps + 1) steps."""
        import torch
        candidates = tuple(TILE_SHAPES) if candidates is None else tuple(candidates)
        stream = getattr(self, "_stream", None) or torch.cuda.current_stream()
        times = {}
        for sh in candidates:
            self.set_tile_shape(sh)
            self.step(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.step_async(steps)
            e1.record(stream)
            self.sync()
            times[TILE_SHAPES[sh]] = e0.elapsed_time(e1) / steps
        best = min(candidates, key=lambda sh: times[TILE_SHAPES[sh]])
        self.set_tile_shape(best)
        return {"ms_per_step": times, "tile_shape": TILE_SHAPES[best]}

    def profile_step(self) -> Dict[str, Dict]:
        """Advance one step with every kernel launch timed by CUDA events on
        the context's stream; returns {kernel: {launches, cells, ms}}."""
        buf = (_KTime * 64)()
        n = C.c_int32()
        self._check(self.lib.gea_profile_step(self.h, buf, 64, C.byref(n)))
        return {buf[i].name.decode(): {"launches": buf[i].launches, "cells": buf[i].cells,
                                       "ms": buf[i].ms} for i in range(min(n.value, 64))}

    # ---- pad checking (debug_pads=True) ----
    def debug_pad_regions(self) -> List[Dict]:
        """The context's arrays: name, device pointer, element bytes, pitch,
        rows and columns in use, span (elements up to the next array)."""
        buf = (_PadRegion * 1024)()
        n = C.c_int32()
        self._check(self.lib.gea_debug_pad_regions(self.h, buf, 1024, C.byref(n)))
        return [{"name": r.name.decode(), "ptr": r.ptr, "elem_bytes": r.elem_bytes, "pitch": r.pitch,
                 "rows": r.rows, "cols": r.cols, "span": r.span} for r in buf[:min(n.value, 1024)]]

    def debug_poison(self):
        self._check(self.lib.gea_debug_poison(self.h))

    @staticmethod
    def _pad_report(r) -> Dict:
        return {"bad": r.bad, "launch": r.launch, "kernel": r.kernel.decode(), "array": r.array.decode(),
                "row": r.row, "col": r.col}

    def debug_check_pads(self) -> Dict:
        """Pad elements that no longer hold the poison, and the first one."""
        r = _PadReport()
        self._check(self.lib.gea_debug_check_pads(self.h, C.byref(r)))
        return self._pad_report(r)

    def debug_step(self) -> Dict:
        """One eagerly launched step with every pad checked after every
        launch; names the first launch that changed a pad."""
        r = _PadReport()
        self._check(self.lib.gea_debug_step(self.h, C.byref(r)))
        return self._pad_report(r)


def probe_fma(bits: int = 64, blocks: int = 608, iters: int = 16384, stream=None, repeats: int = 5) -> Dict:
    """Measured FMA rate (gea_probe_fma): the best of `repeats` CUDA-event
    timed launches on `stream`, in TFLOP/s (an FMA counts 2 flops)."""
    import torch
    lib = library()
    stream = stream or torch.cuda.current_stream()
    dt = torch.float64 if bits == 64 else torch.float32
    out = torch.empty(blocks * 256, dtype=dt, device="cuda")
    flops = blocks * 256 * 8 * iters * 2.0
    _chk(lib.gea_probe_fma(bits, blocks, max(1, iters // 16), out.data_ptr(), stream.cuda_stream),
         "gea_probe_fma")   # warm-up
    best = None
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _chk(lib.gea_probe_fma(bits, blocks, iters, out.data_ptr(), stream.cuda_stream), "gea_probe_fma")
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    assert torch.isfinite(out).all()
    return {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "blocks": blocks, "iters": iters,
            "flops": flops}


def probe_barrier(blocks: int = 456, iters: int = 20000, read_status: bool = True, stream=None,
                  repeats: int = 3) -> Dict:
    """Measured cost of one grid barrier of the persistent kernels' protocol
    (gea_probe_barrier): the best of `repeats` CUDA-event timed launches of
    `iters` barriers on `blocks` co-resident blocks, in microseconds per
    barrier."""
    import torch
    lib = library()
    stream = stream or torch.cuda.current_stream()
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    _chk(lib.gea_probe_barrier(blocks, max(1, iters // 10), int(read_status), scratch.data_ptr(),
                               stream.cuda_stream), "gea_probe_barrier")   # warm-up
    best = None
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _chk(lib.gea_probe_barrier(blocks, iters, int(read_status), scratch.data_ptr(), stream.cuda_stream),
             "gea_probe_barrier")
        e1.record(stream)
        e1.synchronize()
        if int(scratch[2].item()) != 0:
            raise GeaError(GEA_ERR_TIMEOUT, "gea_probe_barrier: a bounded wait gave up")
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return {"us_per_barrier": best * 1e3 / iters, "ms": best, "blocks": blocks, "iters": iters,
            "read_status": bool(read_status)}


CONV_PLAIN, CONV_POOL, CONV_UPADD = 0, 1, 2
CONV_RELU, CONV_OUT_F32 = 1, 2


def _ptr(t):
    return None if t is None else t.data_ptr()


def conv3x3(x0, wt, y, n, h, w, cin, cout, mode=CONV_PLAIN, flags=0, x1=None, bias=None,
            status=None, stream=None):
    """3x3 convolution on the tensor cores (gea_conv3x3): device tensors,
    bfloat16 activations and weights (N x H x W x C, [cout][3][3][cin]),
    FP32 bias; y is bfloat16 or, with CONV_OUT_F32, float32. Enqueued on
    `stream` (a torch stream or None for the current one)."""
    import torch
    st = (stream or torch.cuda.current_stream()).cuda_stream
    n, h, w, cin, cout = int(n), int(h), int(w), int(cin), int(cout)
    # with arguments the library accepts, every tensor must hold exactly what
    # it reads or writes (x0 at twice the size for POOL, x1 at half for UPADD)
    if n >= 1 and h >= 1 and w >= 1 and cin in (16, 32, 64) and cout in (16, 32, 64) and mode in (0, 1, 2):
        f = 4 if mode == CONV_POOL else 1
        _buf(x0, n * h * w * cin * f, "x0", "bf16", device=True)
        if mode == CONV_UPADD and x1 is not None:
            _buf(x1, n * (h // 2) * (w // 2) * cin, "x1", "bf16", device=True)
        _buf(wt, cout * 9 * cin, "wt", "bf16", device=True)
        if bias is not None:
            _buf(bias, cout, "bias", "float32", device=True)
        _buf(y, n * h * w * cout, "y", "float32" if flags & CONV_OUT_F32 else "bf16", device=True)
        if status is not None:
            _buf(status, 1, "status", "int32", device=True)
    rc = library().gea_conv3x3(n, h, w, cin, cout, mode, flags, _ptr(x0), _ptr(x1), _ptr(wt),
                               _ptr(bias), _ptr(y), _ptr(status), st)
    if rc != GEA_OK:
        raise GeaError(rc, "gea_conv3x3 failed")


NET_RELU = 1
NET_LAYERS = 15


def net_param_count() -> int:
    return int(library().gea_net_param_count())


def net_layout() -> np.ndarray:
    """Per layer: cin, cout, k, activation, input kind, level."""
    d = np.zeros(6 * NET_LAYERS, dtype=np.int32)
    _chk(library().gea_net_layout(d.ctypes.data), "gea_net_layout")
    return d.reshape(NET_LAYERS, 6)


def _chk(rc, what):
    if rc != GEA_OK:
        raise GeaError(rc, f"{what} failed")


class Net:
    """The learned pressure-correction network (include/gea_net.h). Tensor
    arguments are contiguous float32 CUDA tensors."""

    def __init__(self, n_max: int, h_max: int, w_max: int, relu: bool = True, stream=None):
        import torch
        self.lib = library()
        h = C.c_void_p()
        _chk(self.lib.gea_net_create(n_max, h_max, w_max, NET_RELU if relu else 0, C.byref(h)),
             "gea_net_create")
        self.h = h
        self.np = net_param_count()
        self.stream = stream or torch.cuda.current_stream()
        _chk(self.lib.gea_net_set_stream(self.h, self.stream.cuda_stream), "gea_net_set_stream")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gea_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        if isinstance(theta, np.ndarray):
            t = np.ascontiguousarray(theta, dtype=np.float32)
            _chk(self.lib.gea_net_set_params(self.h, _buf(t, self.np, "theta", "float32"), MEM_HOST),
                 "gea_net_set_params")
        else:
            _chk(self.lib.gea_net_set_params(self.h, _buf(theta, self.np, "theta", "float32", device=True),
                                             MEM_DEVICE), "gea_net_set_params")

    def get_params(self) -> np.ndarray:
        t = np.empty(self.np, dtype=np.float32)
        _chk(self.lib.gea_net_get_params(self.h, t.ctypes.data, MEM_HOST), "gea_net_get_params")
        return t

    def _operators(self, n, hh, ww, c, ax, az):
        """Pointers of the Helmholtz coefficients of n samples of hh x ww."""
        return (_buf(c, n * hh * ww, "c", "float32", device=True),
                _buf(ax, n * hh * (ww + 1), "ax", "float32", device=True),
                _buf(az, n * (hh + 1) * ww, "az", "float32", device=True))

    def forward(self, r, y):
        n, hh, ww = (int(d) for d in r.shape)
        pr = _buf(r, n * hh * ww, "r", "float32", device=True)
        py = _buf(y, n * hh * ww, "y", "float32", device=True)
        _chk(self.lib.gea_net_forward(self.h, n, hh, ww, pr, py), "gea_net_forward")
        self._last = (n, hh, ww)

    def energy(self, c, ax, az, dy) -> float:
        """Energy loss of the last forward pass (its n, h, w size the arrays)."""
        n, hh, ww = getattr(self, "_last", (0, 0, 0))
        if not n:
            raise GeaError(GEA_ERR_STATE, "gea_net_energy: no forward pass")
        pc, pax, paz = self._operators(n, hh, ww, c, ax, az)
        loss = C.c_float()
        _chk(self.lib.gea_net_energy(self.h, pc, pax, paz, _buf(dy, n * hh * ww, "dy", "float32", device=True),
                                     C.byref(loss)), "gea_net_energy")
        return float(loss.value)

    def backward(self, dy, grad):
        n, hh, ww = getattr(self, "_last", (0, 0, 0))
        if not n:
            raise GeaError(GEA_ERR_STATE, "gea_net_backward: no forward pass")
        _chk(self.lib.gea_net_backward(self.h, _buf(dy, n * hh * ww, "dy", "float32", device=True),
                                       _buf(grad, self.np, "grad", "float32", device=True)), "gea_net_backward")

    def adam(self, grad, lr: float):
        _chk(self.lib.gea_net_adam(self.h, _buf(grad, self.np, "grad", "float32", device=True), lr), "gea_net_adam")

    def train_step(self, r, c, ax, az, lr: float) -> float:
        n, hh, ww = (int(d) for d in r.shape)
        pr = _buf(r, n * hh * ww, "r", "float32", device=True)
        pc, pax, paz = self._operators(n, hh, ww, c, ax, az)
        loss = C.c_float()
        _chk(self.lib.gea_net_train_step(self.h, n, hh, ww, pr, pc, pax, paz, lr, C.byref(loss)),
             "gea_net_train_step")
        self._last = (n, hh, ww)
        return float(loss.value)


class Ensemble:
    """Independent solvers advanced together by one cooperative launch per
    call (gea_ensemble_*). The solvers stay usable for get/diagnostics; step
    them only through the ensemble while it exists."""

    def __init__(self, solvers, stream=None, weights=None):
        """weights: optional per-member work weights (blocks in proportion;
        default the members' tile counts)."""
        self.lib = library()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[sv.h.value for sv in self.solvers])
        w = None
        if weights is not None:
            self._w = np.ascontiguousarray(weights, dtype=np.float64)
            w = _buf(self._w, len(self.solvers), "weights", device=False)
        h = C.c_void_p()
        _chk(self.lib.gea_ensemble_create(arr, len(self.solvers), w, C.byref(h)), "gea_ensemble_create")
        self.h = h
        if stream is not None:
            _chk(self.lib.gea_ensemble_set_stream(self.h, stream.cuda_stream), "gea_ensemble_set_stream")

    def blocks(self):
        return [int(self.lib.gea_ensemble_blocks(self.h, m)) for m in range(len(self.solvers))]

    def set_graph(self, on: bool):
        """Launch through captured CUDA graphs (default) or directly."""
        _chk(self.lib.gea_ensemble_set_graph(self.h, 1 if on else 0), "gea_ensemble_set_graph")

    def step_async(self, n: int = 1):
        _chk(self.lib.gea_ensemble_step(self.h, int(n)), "gea_ensemble_step")

    def sync(self):
        _chk(self.lib.gea_ensemble_sync(self.h), "gea_ensemble_sync")

    def step(self, n: int = 1):
        self.step_async(n)
        self.sync()

    def close(self):
        if getattr(self, "h", None):
            self.lib.gea_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATE3_FIELDS = ("rho", "u", "v", "w", "T", "p", "pp")


class Solver3D:
    """One context of the three-dimensional step (include/gea3d.h): cell
    fields are (nz, ny, nx) float64 arrays, x fastest."""

    def __init__(self, grid, const, mg_min_cells: int = 0, stream=None, mixed: bool = False,
                 mp_rtol: float = 0.0):
        """mixed=True selects the mixed-precision step (GEA_FLAG_MIXED) with
        inner tolerance mp_rtol (0: the library default)."""
        self.lib = library()
        self.grid, self.const = grid, const
        g = _Grid3(grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, grid.lz)
        c = _Const(const.R, const.cp, const.g, const.p0, const.mu, const.Pr, const.dt,
                   const.n_corr, const.jac_rtol, const.jac_maxit, const.cg_rtol, const.cg_maxit,
                   mg_min_cells, FLAG_MIXED if mixed else 0, mp_rtol, getattr(const, "cs", 0.0),
                   getattr(const, "reading_flags", 0))
        h = C.c_void_p()
        rc = self.lib.gea3d_create(C.byref(g), C.byref(c), C.byref(h))
        if rc != GEA_OK:
            raise GeaError(rc, "gea3d_create failed")
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            self.lib.gea3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != GEA_OK:
            msg = self.lib.gea3d_last_error(self.h)
            raise GeaError(rc, msg.decode() if msg else "")

    def set_stream(self, stream):
        s = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.gea3d_set_stream(self.h, C.c_void_p(s or 0)))

    def set_conservative(self, fields: Dict):
        mem = MEM_DEVICE if _is_device(fields["rho"]) else MEM_HOST
        n = self.grid.nx * self.grid.ny * self.grid.nz
        ptrs = [_buf(fields[k], n, k, device=mem == MEM_DEVICE) for k in ("rho", "rhou", "rhov", "rhow", "rhoe")]
        self._check(self.lib.gea3d_set_conservative(self.h, *ptrs, mem))

    def get_state(self, out: Optional[Dict] = None) -> Dict:
        g = self.grid
        if out is None:
            out = {k: np.empty((g.nz, g.ny, g.nx)) for k in STATE3_FIELDS}
        mem = MEM_DEVICE if _is_device(next(iter(out.values()))) else MEM_HOST
        n = g.nx * g.ny * g.nz
        ptrs = [_buf(out[k], n, k, device=mem == MEM_DEVICE) if k in out else None for k in STATE3_FIELDS]
        self._check(self.lib.gea3d_get_state(self.h, *ptrs, mem))
        return out

    def diagnostics(self, theta_bar: np.ndarray):
        """theta' (nz, ny, nx), mass and total energy of the current state,
        computed on the device (gea3d_get_diag)."""
        tb = np.ascontiguousarray(theta_bar, dtype=np.float64)
        g = self.grid
        th = np.empty((g.nz, g.ny, g.nx))
        m = C.c_double()
        e = C.c_double()
        self._check(self.lib.gea3d_get_diag(self.h, _buf(tb, g.nz, "theta_bar", device=False), th.ctypes.data,
                                            C.addressof(m), C.addressof(e)))
        return th, m.value, e.value

    def step(self, n: int = 1):
        self._check(self.lib.gea3d_step(self.h, int(n)))

    def step_async(self, n: int = 1):
        self._check(self.lib.gea3d_step_async(self.h, int(n)))

    def sync(self):
        self._check(self.lib.gea3d_sync(self.h))

    def stats(self) -> Dict:
        s = _Stats()
        self._check(self.lib.gea3d_get_stats(self.h, C.byref(s)))
        n = self.const.n_corr
        return {"steps_done": s.steps_done, "jac_u": s.jac_u, "jac_h": s.jac_h,
                "cg_iters": list(s.cg_iters)[:n], "cg_relres": list(s.cg_relres)[:n],
                "status": s.status, "mg_levels": s.mg_levels, "launches": s.launches,
                "driver": {0: "graph", 2: "mixed"}[s.driver]}

    def set_tile_shape(self, shape: int):
        """Tile shape of the persistent kernels (gea_set_tile_shape): one of
        TILE_SHAPES' keys."""
        self._check(self.lib.gea_set_tile_shape(self.h, int(shape)))
        self.tile_shape = int(shape)

    def tune_tile_shape(self, candidates=None, steps: int = 3) -> Dict:
        """Tile-shape autotuner of the persistent kernels: for each candidate
        shape, one untimed step and `steps` steps timed with CUDA events on
        the context's stream; keeps the fastest. The state advances by
        len(candidates) x (steps + 1) steps."""
        import torch
        candidates = tuple(TILE_SHAPES) if candidates is None else tuple(candidates)
        stream = getattr(self, "_stream", None) or torch.cuda.current_stream()
        times = {}
        for sh in candidates:
            self.set_tile_shape(sh)
            self.step(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.step_async(steps)
            e1.record(stream)
            self.sync()
            times[TILE_SHAPES[sh]] = e0.elapsed_time(e1) / steps
        best = min(candidates, key=lambda sh: times[TILE_SHAPES[sh]])
        self.set_tile_shape(best)
        return {"ms_per_step": times, "tile_shape": TILE_SHAPES[best]}

    def profile_step(self) -> Dict[str, Dict]:
        """One eagerly launched step with per-kernel CUDA-event totals."""
        buf = (_KTime * 32)()
        n = C.c_int32()
        self._check(self.lib.gea3d_profile_step(self.h, buf, 32, C.byref(n)))
        return {buf[i].name.decode(): {"launches": buf[i].launches, "cells": buf[i].cells, "ms": buf[i].ms}
                for i in range(min(n.value, 32))}
