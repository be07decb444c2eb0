"""ctypes binding of the plain-C FP64 three-dimensional oracle
(gea_oracle3d.c).

TEST INFRASTRUCTURE: only tests/ and the benchmark's CPU legs may import
this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gea_oracle3d.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgea_oracle3d.so")

B3_EVEN, B3_U, B3_V, B3_W, B3_H = 0, 1, 2, 3, 4
FIELDS = ("rho", "u", "v", "w", "T", "h", "p", "pp", "pold", "phix", "phiy", "phiz")

_lock = threading.Lock()
_lib = None


def build_oracle3d(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("R", C.c_double), ("cp", C.c_double), ("g", C.c_double), ("p0", C.c_double),
                ("mu", C.c_double), ("Pr", C.c_double), ("dt", C.c_double),
                ("n_corr", C.c_int32), ("jac_rtol", C.c_double), ("jac_maxit", C.c_int32),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32), ("cs", C.c_double)]


_P = C.POINTER(C.c_double)


class _State(C.Structure):
    _fields_ = [(n, _P) for n in FIELDS]


class _Stats(C.Structure):
    _fields_ = [("jac_u", C.c_int32), ("jac_h", C.c_int32), ("cg_iters", C.c_int32 * 4),
                ("cg_relres", C.c_double * 4), ("status", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle3d())
            P = C.c_void_p
            lib.o3_derive.argtypes = [C.POINTER(_Cfg), P, P, P, P, P, C.POINTER(_State)]
            lib.o3_step.argtypes = [C.POINTER(_Cfg), C.POINTER(_State), C.c_int32, C.POINTER(_Stats)]
            lib.o3_totals.argtypes = [C.POINTER(_Cfg), C.POINTER(_State), P, P]
            lib.o3_laplacian_cell.argtypes = [C.POINTER(_Cfg), P, C.c_int, C.c_int, C.c_int, C.c_int]
            lib.o3_laplacian_cell.restype = C.c_double
            lib.o3_divergence_cell.argtypes = [C.POINTER(_Cfg), P, P, P, C.c_int, C.c_int, C.c_int]
            lib.o3_divergence_cell.restype = C.c_double
            lib.o3_strain_cell.argtypes = [C.POINTER(_Cfg), P, P, P, C.c_int, C.c_int, C.c_int]
            lib.o3_strain_cell.restype = C.c_double
            lib.o3_smagorinsky.argtypes = [C.POINTER(_Cfg), P, P, P, P, P]
            lib.o3_diffusion_cell.argtypes = [C.POINTER(_Cfg), P, P, C.c_int, C.c_int, C.c_int, C.c_int]
            lib.o3_diffusion_cell.restype = C.c_double
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data


class State3(dict):
    """Full 3D state: cell fields nz x ny x nx, face fluxes phix
    nz x ny x (nx+1), phiy nz x (ny+1) x nx, phiz (nz+1) x ny x nx."""

    def __init__(self, grid):
        super().__init__()
        nx, ny, nz = grid.nx, grid.ny, grid.nz
        for f in FIELDS[:9]:
            self[f] = np.zeros((nz, ny, nx))
        self["phix"] = np.zeros((nz, ny, nx + 1))
        self["phiy"] = np.zeros((nz, ny + 1, nx))
        self["phiz"] = np.zeros((nz + 1, ny, nx))

    def view(self):
        return _State(*[C.cast(self[f].ctypes.data, _P) for f in FIELDS])

    def conservative(self, g, cv, dz):
        z = ((np.arange(self["rho"].shape[0]) + 0.5) * dz)[:, None, None]
        r = self["rho"]
        K = 0.5 * (self["u"] ** 2 + self["v"] ** 2 + self["w"] ** 2)
        return {"rho": r, "rhou": r * self["u"], "rhov": r * self["v"], "rhow": r * self["w"],
                "rhoe": r * (cv * self["T"] + K + g * z)}


class Oracle3D:
    def __init__(self, grid, const):
        self.lib = _load()
        self.grid, self.const = grid, const
        self.cfg = _Cfg(grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, grid.lz, const.R, const.cp, const.g,
                        const.p0, const.mu, const.Pr, const.dt, const.n_corr, const.jac_rtol,
                        const.jac_maxit, const.cg_rtol, const.cg_maxit, getattr(const, "cs", 0.0))

    def derive(self, fields: Dict[str, np.ndarray]) -> State3:
        s = State3(self.grid)
        a = [np.ascontiguousarray(fields[k], dtype=np.float64) for k in ("rho", "rhou", "rhov", "rhow", "rhoe")]
        v = s.view()
        if self.lib.o3_derive(C.byref(self.cfg), *[_ptr(x) for x in a], C.byref(v)):
            raise ValueError("rho <= 0 or T <= 0")
        return s

    def step(self, s: State3, n: int = 1) -> Dict:
        st = _Stats()
        v = s.view()
        rc = self.lib.o3_step(C.byref(self.cfg), C.byref(v), n, C.byref(st))
        return {"status": rc, "jac_u": st.jac_u, "jac_h": st.jac_h,
                "cg_iters": list(st.cg_iters)[:self.const.n_corr],
                "cg_relres": list(st.cg_relres)[:self.const.n_corr]}

    def totals(self, s: State3):
        m, e = C.c_double(), C.c_double()
        v = s.view()
        self.lib.o3_totals(C.byref(self.cfg), C.byref(v), C.addressof(m), C.addressof(e))
        return m.value, e.value

    def laplacian_cell(self, X, bc, i, j, k):
        x = np.ascontiguousarray(X, dtype=np.float64)
        return self.lib.o3_laplacian_cell(C.byref(self.cfg), _ptr(x), bc, i, j, k)

    def strain_cell(self, u, v, w, i, j, k):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (u, v, w)]
        return self.lib.o3_strain_cell(C.byref(self.cfg), *[_ptr(x) for x in a], i, j, k)

    def smagorinsky(self, rho, u, v, w):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, u, v, w)]
        out = np.empty_like(a[0])
        self.lib.o3_smagorinsky(C.byref(self.cfg), *[_ptr(x) for x in a], _ptr(out))
        return out

    def diffusion_cell(self, mu, X, bc, i, j, k):
        m = np.ascontiguousarray(mu, dtype=np.float64)
        x = np.ascontiguousarray(X, dtype=np.float64)
        return self.lib.o3_diffusion_cell(C.byref(self.cfg), _ptr(m), _ptr(x), bc, i, j, k)
