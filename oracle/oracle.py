"""ctypes binding of the plain-C FP64 oracle (gea_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.

The oracle is compiled with the host C compiler (gcc -O2, no intrinsics,
single-threaded) into oracle/_build/ on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gea_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgea_oracle.so")

BC_EVEN, BC_U, BC_W, BC_H = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("lx", C.c_double), ("lz", C.c_double),
                ("R", C.c_double), ("cp", C.c_double), ("g", C.c_double), ("p0", C.c_double),
                ("mu", C.c_double), ("Pr", C.c_double), ("dt", C.c_double),
                ("n_corr", C.c_int32), ("jac_rtol", C.c_double), ("jac_maxit", C.c_int32),
                ("cg_rtol", C.c_double), ("cg_maxit", C.c_int32), ("cs", C.c_double),
                ("reading_flags", C.c_uint32)]


_P = C.POINTER(C.c_double)


class _State(C.Structure):
    _fields_ = [(n, _P) for n in ("rho", "u", "w", "T", "h", "p", "pp", "pold", "phix", "phiz", "Kold")]


class _Stats(C.Structure):
    _fields_ = [("jac_u", C.c_int32), ("jac_w", C.c_int32), ("jac_h", C.c_int32),
                ("cg_iters", C.c_int32 * 4), ("cg_relres", C.c_double * 4),
                ("status", C.c_int32)]


class _Dump(C.Structure):
    _fields_ = [(n, _P) for n in ("rho1", "u1", "w1", "h1", "T1", "rho2", "psi",
                                  "Hx", "Hz", "b", "Dx", "Dz", "bh")]


def _bind(path: str):
    """Load an oracle build and declare its entry points."""
    lib = C.CDLL(path)
    i32 = C.c_int32
    lib.orc_derive.argtypes = [C.POINTER(_Cfg), _P, _P, _P, _P, C.POINTER(_State)]
    lib.orc_derive.restype = C.c_int
    lib.orc_step.argtypes = [C.POINTER(_Cfg), C.POINTER(_State), i32,
                             C.POINTER(_Stats), C.POINTER(_Dump)]
    lib.orc_step.restype = C.c_int
    lib.orc_diagnostics.argtypes = [C.POINTER(_Cfg), C.POINTER(_State), _P, _P, _P, _P]
    lib.orc_continuity_residual.argtypes = [C.POINTER(_Cfg), _P, C.POINTER(_State), _P]
    lib.orc_convection.argtypes = [C.POINTER(_Cfg), _P, _P, _P, C.c_int, _P]
    lib.orc_laplacian.argtypes = [C.POINTER(_Cfg), _P, C.c_int, _P]
    lib.orc_strain.argtypes = [C.POINTER(_Cfg), _P, _P, _P]
    lib.orc_smagorinsky.argtypes = [C.POINTER(_Cfg), _P, _P, _P, _P]
    lib.orc_diffusion.argtypes = [C.POINTER(_Cfg), _P, _P, C.c_int, _P]
    lib.orc_face_forces.argtypes = [C.POINTER(_Cfg), _P, _P, _P, _P]
    lib.orc_helmholtz_apply.argtypes = [C.POINTER(_Cfg), _P, _P, _P, _P, _P]
    lib.orc_pcg.argtypes = [C.POINTER(_Cfg), _P, _P, _P, _P, _P, _P]
    lib.orc_pcg.restype = C.c_int
    lib.orc_transport_apply.argtypes = [C.POINTER(_Cfg), _P, _P, _P, C.c_double,
                                        C.c_int, _P, _P]
    lib.orc_transport_solve.argtypes = [C.POINTER(_Cfg), _P, _P, _P, C.c_double,
                                        C.c_int, _P, _P]
    lib.orc_transport_solve.restype = C.c_int
    lib.orc_set_reverse_sums.argtypes = [C.c_int]
    return lib


def set_reverse_sums(on: bool):
    """Evaluate the oracle's reductions (norms, CG dot products) in reverse
    index order (on) or in index order (off, the default): two correct
    evaluations whose difference is a round-off floor."""
    _lib_handle().orc_set_reverse_sums(1 if on else 0)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build_oracle())
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


STATE_FIELDS = ("rho", "u", "w", "T", "h", "p", "pp", "pold", "phix", "phiz", "Kold")
# reading flags (Constants.reading_flags): the literal K^{n-1} of eq. step3_sd
READING_K_LAGGED = 1


class OracleState:
    """Full solver state as float64 numpy arrays: cell fields (nz, nx),
    phix (nz, nx+1), phiz (nz+1, nx)."""

    def __init__(self, nx: int, nz: int, arrays: Optional[Dict[str, np.ndarray]] = None):
        self.nx, self.nz = nx, nz
        shapes = {f: (nz, nx) for f in STATE_FIELDS}
        shapes["phix"] = (nz, nx + 1)
        shapes["phiz"] = (nz + 1, nx)
        self.a = {}
        for f in STATE_FIELDS:
            if arrays is not None:
                v = np.ascontiguousarray(arrays[f], dtype=np.float64).copy()
                assert v.shape == shapes[f], (f, v.shape, shapes[f])
            else:
                v = np.zeros(shapes[f])
            self.a[f] = v

    def __getitem__(self, k):
        return self.a[k]

    def copy(self) -> "OracleState":
        return OracleState(self.nx, self.nz, self.a)

    def cstruct(self) -> _State:
        return _State(*[_ptr(self.a[f]) for f in STATE_FIELDS])

    def conservative(self, g: float, cv: float, dz: float) -> Dict[str, np.ndarray]:
        z = (np.arange(self.nz) + 0.5)[:, None] * dz
        rho, u, w, T = self.a["rho"], self.a["u"], self.a["w"], self.a["T"]
        return {"rho": rho, "rhou": rho * u, "rhow": rho * w,
                "rhoe": rho * (cv * T + 0.5 * (u * u + w * w) + g * z)}


class Oracle:
    """One grid + constant set. Mirrors the library's create/set/step/get."""

    def __init__(self, grid, const, lib_path: Optional[str] = None):
        """lib_path selects another build of the oracle source (the tests use
        this to check that planted mistakes are caught)."""
        self.grid, self.const = grid, const
        self.cfg = _Cfg(grid.nx, grid.nz, grid.lx, grid.lz, const.R, const.cp, const.g,
                        const.p0, const.mu, const.Pr, const.dt, const.n_corr,
                        const.jac_rtol, const.jac_maxit, const.cg_rtol, const.cg_maxit,
                        getattr(const, "cs", 0.0), getattr(const, "reading_flags", 0))
        self.lib = _lib_handle() if lib_path is None else _bind(lib_path)
        self.last_stats = None

    # -- state ------------------------------------------------------------
    def derive(self, fields: Dict[str, np.ndarray]) -> OracleState:
        """Full state from conservative fields (rho, rhou, rhow, rhoe)."""
        s = OracleState(self.grid.nx, self.grid.nz)
        f = {k: np.ascontiguousarray(fields[k], dtype=np.float64) for k in
             ("rho", "rhou", "rhow", "rhoe")}
        st = s.cstruct()
        rc = self.lib.orc_derive(C.byref(self.cfg), _ptr(f["rho"]), _ptr(f["rhou"]),
                                 _ptr(f["rhow"]), _ptr(f["rhoe"]), C.byref(st))
        if rc != 0:
            raise ValueError("non-positive density or temperature")
        return s

    def step(self, s: OracleState, n: int = 1, dump: bool = False):
        """Advance s in place by n steps. Returns (stats dict, dump dict|None)."""
        st = _Stats()
        d = None
        dptr = None
        if dump:
            nx, nz = self.grid.nx, self.grid.nz
            d = {k: np.zeros((nz, nx)) for k in ("rho1", "u1", "w1", "h1", "T1", "rho2",
                                                 "psi", "Hx", "Hz", "b", "bh")}
            d["Dx"] = np.zeros((nz, nx + 1))
            d["Dz"] = np.zeros((nz + 1, nx))
            dptr = _Dump(*[_ptr(d[k]) for k in ("rho1", "u1", "w1", "h1", "T1", "rho2", "psi",
                                                  "Hx", "Hz", "b", "Dx", "Dz", "bh")])
        cs = s.cstruct()
        self.lib.orc_step(C.byref(self.cfg), C.byref(cs), int(n), C.byref(st),
                          C.byref(dptr) if dptr is not None else None)
        stats = {"jac_u": st.jac_u, "jac_w": st.jac_w, "jac_h": st.jac_h,
                 "cg_iters": list(st.cg_iters)[: self.const.n_corr],
                 "cg_relres": list(st.cg_relres)[: self.const.n_corr],
                 "status": st.status}
        self.last_stats = stats
        return stats, d

    def diagnostics(self, s: OracleState, theta_bar: np.ndarray):
        th = np.zeros((self.grid.nz, self.grid.nx))
        m = C.c_double()
        e = C.c_double()
        tb = np.ascontiguousarray(theta_bar, dtype=np.float64)
        cs = s.cstruct()
        self.lib.orc_diagnostics(C.byref(self.cfg), C.byref(cs), _ptr(tb), _ptr(th),
                                 C.cast(C.pointer(m), _P), C.cast(C.pointer(e), _P))
        return th, m.value, e.value

    def continuity_residual(self, rho_old: np.ndarray, s: OracleState) -> np.ndarray:
        out = np.zeros((self.grid.nz, self.grid.nx))
        ro = np.ascontiguousarray(rho_old, dtype=np.float64)
        cs = s.cstruct()
        self.lib.orc_continuity_residual(C.byref(self.cfg), _ptr(ro), C.byref(cs), _ptr(out))
        return out

    # -- operators (for the pins) -----------------------------------------
    def convection(self, phix, phiz, X, bc) -> np.ndarray:
        out = np.zeros((self.grid.nz, self.grid.nx))
        args = [np.ascontiguousarray(a, dtype=np.float64) for a in (phix, phiz, X)]
        self.lib.orc_convection(C.byref(self.cfg), _ptr(args[0]), _ptr(args[1]),
                                _ptr(args[2]), bc, _ptr(out))
        return out

    def laplacian(self, X, bc) -> np.ndarray:
        out = np.zeros((self.grid.nz, self.grid.nx))
        x = np.ascontiguousarray(X, dtype=np.float64)
        self.lib.orc_laplacian(C.byref(self.cfg), _ptr(x), bc, _ptr(out))
        return out

    def strain(self, u, w) -> np.ndarray:
        """|S| = sqrt(2 S_ij S_ij) per cell (Smagorinsky model)."""
        out = np.zeros((self.grid.nz, self.grid.nx))
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (u, w)]
        self.lib.orc_strain(C.byref(self.cfg), _ptr(a[0]), _ptr(a[1]), _ptr(out))
        return out

    def smagorinsky(self, rho, u, w) -> np.ndarray:
        """mu + rho (cs Delta)^2 |S| per cell."""
        out = np.zeros((self.grid.nz, self.grid.nx))
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, u, w)]
        self.lib.orc_smagorinsky(C.byref(self.cfg), _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(out))
        return out

    def diffusion(self, mu, X, bc) -> np.ndarray:
        """(1/V) sum_f mu_f (grad X)_f . A_f with face-mean viscosities."""
        out = np.zeros((self.grid.nz, self.grid.nx))
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (mu, X)]
        self.lib.orc_diffusion(C.byref(self.cfg), _ptr(a[0]), _ptr(a[1]), bc, _ptr(out))
        return out

    def face_forces(self, pp, rho):
        nx, nz = self.grid.nx, self.grid.nz
        Gx = np.zeros((nz, nx + 1))
        Gz = np.zeros((nz + 1, nx))
        a = np.ascontiguousarray(pp, dtype=np.float64)
        b = np.ascontiguousarray(rho, dtype=np.float64)
        self.lib.orc_face_forces(C.byref(self.cfg), _ptr(a), _ptr(b), _ptr(Gx), _ptr(Gz))
        return Gx, Gz

    def helmholtz_apply(self, psi, Dx, Dz, x) -> np.ndarray:
        out = np.zeros((self.grid.nz, self.grid.nx))
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (psi, Dx, Dz, x)]
        self.lib.orc_helmholtz_apply(C.byref(self.cfg), *[_ptr(v) for v in a], _ptr(out))
        return out

    def pcg(self, psi, Dx, Dz, b, x0):
        x = np.ascontiguousarray(x0, dtype=np.float64).copy()
        rr = C.c_double()
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (psi, Dx, Dz, b)]
        it = self.lib.orc_pcg(C.byref(self.cfg), *[_ptr(v) for v in a], _ptr(x),
                              C.cast(C.pointer(rr), _P))
        return x, it, rr.value

    def transport_apply(self, rho1, phix, phiz, nu, bc, X) -> np.ndarray:
        out = np.zeros((self.grid.nz, self.grid.nx))
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho1, phix, phiz)]
        x = np.ascontiguousarray(X, dtype=np.float64)
        self.lib.orc_transport_apply(C.byref(self.cfg), *[_ptr(v) for v in a], float(nu),
                                     bc, _ptr(x), _ptr(out))
        return out

    def transport_solve(self, rho1, phix, phiz, nu, bc, b, X0):
        x = np.ascontiguousarray(X0, dtype=np.float64).copy()
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho1, phix, phiz, b)]
        it = self.lib.orc_transport_solve(C.byref(self.cfg), _ptr(a[0]), _ptr(a[1]),
                                          _ptr(a[2]), float(nu), bc, _ptr(a[3]), _ptr(x))
        return x, it
