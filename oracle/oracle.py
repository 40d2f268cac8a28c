"""ctypes loader for the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import dataclasses
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpdata_oracle.c")
_BUILD = os.path.join(_HERE, "_build", platform.machine())
_LIB = None
_LIB_OMP = None


def lib_path(omp: bool = False) -> str:
    return os.path.join(_BUILD, "libmpdata_oracle_omp.so" if omp else "libmpdata_oracle.so")


def build(force: bool = False, src: str = _SRC, out: str | None = None, omp: bool = False) -> str:
    """Compile the oracle (or a copy of its source) into a shared library.

    omp=True builds the same source with -fopenmp: the per-cell loops run on
    all host cores and return the serial build's bits."""
    out = out or lib_path(omp)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared"]
        if omp:
            cmd.append("-fopenmp")
        subprocess.check_call(cmd + [src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("iterations", ctypes.c_int),
                ("nonoscillatory", ctypes.c_int), ("eps", ctypes.c_double),
                ("extrema", ctypes.c_int)]


class _Stages(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("psi1", "v1", "v2", "v3", "beta_up", "beta_dn", "vm1", "vm2", "vm3")]


@dataclasses.dataclass
class Config:
    nx: int
    ny: int
    nz: int
    periodic: tuple = (1, 1, 1)
    iterations: int = 2
    nonoscillatory: int = 1
    eps: float = 1e-15
    extrema: int = 0  # 0: psi^n and the corrected field; 1: the corrected field only

    def c(self) -> _Cfg:
        return _Cfg(self.nx, self.ny, self.nz, (ctypes.c_int * 3)(*self.periodic),
                    self.iterations, self.nonoscillatory, self.eps, self.extrema)


def load(path: str | None = None, omp: bool = False):
    """Load the oracle library (building it first if needed); omp=True loads
    the OpenMP build."""
    global _LIB, _LIB_OMP
    if path is None and omp and _LIB_OMP is not None:
        return _LIB_OMP
    if path is None and not omp and _LIB is not None:
        return _LIB
    lib = ctypes.CDLL(path or build(omp=omp))
    P = ctypes.c_void_p
    lib.oracle_step.argtypes = [ctypes.POINTER(_Cfg), P, P, P, P, P, P, ctypes.POINTER(_Stages)]
    lib.oracle_step.restype = ctypes.c_int
    lib.oracle_run.argtypes = [ctypes.POINTER(_Cfg), P, P, P, P, P, ctypes.c_int]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_mass.argtypes = [ctypes.c_long, P, P]
    lib.oracle_mass.restype = ctypes.c_double
    lib.oracle_threads.argtypes = []
    lib.oracle_threads.restype = ctypes.c_int
    if path is None and omp:
        _LIB_OMP = lib
    elif path is None:
        _LIB = lib
    return lib


def threads(lib=None) -> int:
    """Threads the library's per-cell loops use (1 for the serial build)."""
    return int((lib or load()).oracle_threads())


def _arr(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def step(cfg: Config, h, psi, u1, u2, u3, lib=None) -> np.ndarray:
    """One MPDATA step; returns psi^{n+1} (float64 [nz][ny][nx])."""
    lib = lib or load()
    shp = (cfg.nz, cfg.ny, cfg.nx)
    h, psi, u1, u2, u3 = (_arr(a, shp) for a in (h, psi, u1, u2, u3))
    out = np.empty(shp)
    c = cfg.c()
    rc = lib.oracle_step(ctypes.byref(c), _ptr(h), _ptr(psi), _ptr(u1), _ptr(u2), _ptr(u3),
                         _ptr(out), None)
    if rc:
        raise ValueError("oracle_step rejected the configuration")
    return out


def stages(cfg: Config, h, psi, u1, u2, u3, lib=None) -> dict:
    """One step with every intermediate array returned."""
    lib = lib or load()
    shp = (cfg.nz, cfg.ny, cfg.nx)
    h, psi, u1, u2, u3 = (_arr(a, shp) for a in (h, psi, u1, u2, u3))
    names = ("psi1", "v1", "v2", "v3", "beta_up", "beta_dn", "vm1", "vm2", "vm3")
    bufs = {n: np.zeros(shp) for n in names}
    st = _Stages(*[b.ctypes.data for b in (bufs[n] for n in names)])
    out = np.empty(shp)
    c = cfg.c()
    rc = lib.oracle_step(ctypes.byref(c), _ptr(h), _ptr(psi), _ptr(u1), _ptr(u2), _ptr(u3),
                         _ptr(out), ctypes.byref(st))
    if rc:
        raise ValueError("oracle_step rejected the configuration")
    bufs["out"] = out
    return bufs


def run(cfg: Config, h, psi, u1, u2, u3, nsteps: int, lib=None) -> np.ndarray:
    """nsteps MPDATA steps; returns the final psi (float64)."""
    lib = lib or load()
    shp = (cfg.nz, cfg.ny, cfg.nx)
    h, u1, u2, u3 = (_arr(a, shp) for a in (h, u1, u2, u3))
    p = np.array(_arr(psi, shp), copy=True)
    c = cfg.c()
    rc = lib.oracle_run(ctypes.byref(c), _ptr(h), _ptr(p), _ptr(u1), _ptr(u2), _ptr(u3),
                        int(nsteps))
    if rc:
        raise ValueError("oracle_run rejected the configuration")
    return p


def mass(h, psi, lib=None) -> float:
    """Compensated sum of h*psi."""
    lib = lib or load()
    h = np.ascontiguousarray(h, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    assert h.shape == psi.shape
    return float(lib.oracle_mass(h.size, _ptr(h), _ptr(psi)))
