"""GB300-native (sm_103a) MPDATA advection: Python front end of libmpdata.

    import torch, paper_1507_01265_gb300 as mp
    s = mp.Solver(1024, 512, 64, periodic=(1, 1, 0))
    s.step(h, psi, u1, u2, u3, nsteps=50)        # CUDA tensors, in place on psi

Fields are contiguous [nz][ny][nx] tensors of the solver's dtype; u1[k][j][i]
is the Courant number on the x-face between cells i-1 and i (see
include/mpdata.h for the full contract).
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import MpdataError, check, version  # noqa: F401

_DTYPES = {"f32": _lib.MPDATA_F32, "f64": _lib.MPDATA_F64}
_PATHS = {"fused": _lib.MPDATA_PATH_FUSED, "stages": _lib.MPDATA_PATH_STAGES}


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One MPDATA problem size and option set (wraps an mpdata_t handle)."""

    def __init__(self, nx: int, ny: int, nz: int, *, periodic=(1, 1, 1), iterations: int = 2,
                 nonoscillatory: bool = True, dtype: str = "f32", path: str = "fused",
                 tile=None, eps: float = 1e-15):
        o = _lib.default_opts()
        o.iterations = int(iterations)
        o.nonoscillatory = int(bool(nonoscillatory))
        for d in range(3):
            o.periodic[d] = int(periodic[d])
        o.dtype = _DTYPES[dtype]
        o.path = _PATHS[path]
        if tile is not None:
            o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        o.eps = float(eps)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype_name = dtype
        self.opts = o
        self._h = ctypes.c_void_p()
        check(_lib.lib.mpdata_create(self.nx, self.ny, self.nz, ctypes.byref(o),
                                     ctypes.byref(self._h)), "mpdata_create")

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def torch_dtype(self):
        torch = _torch()
        return torch.float64 if self.dtype_name == "f64" else torch.float32

    def _dev(self, t, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype != self.torch_dtype() or not t.is_contiguous() or t.numel() != self.ncells:
            raise ValueError("%s must be a contiguous %s tensor of %d elements"
                             % (name, self.torch_dtype(), self.ncells))
        return ctypes.c_void_p(t.data_ptr())

    def step(self, h, psi, u1, u2, u3, nsteps: int, stream=None) -> None:
        """nsteps steps in place on psi (async on `stream`, default: current)."""
        args = [self._dev(t, n) for t, n in ((h, "h"), (psi, "psi"), (u1, "u1"), (u2, "u2"),
                                             (u3, "u3"))]
        check(_lib.lib.mpdata_step(self._h, *args, int(nsteps), _stream_handle(stream)),
              "mpdata_step")

    def solve_host(self, h, psi, u1, u2, u3, nsteps: int, stream=None) -> None:
        """nsteps steps on host arrays (numpy or CPU tensors); psi is updated
        in place.  Copies in, steps and copies back inside the call."""
        import numpy as np
        torch = _torch()
        ptrs = []
        want = np.float64 if self.dtype_name == "f64" else np.float32
        for a, n in ((h, "h"), (psi, "psi"), (u1, "u1"), (u2, "u2"), (u3, "u3")):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or not a.is_contiguous() or a.dtype != self.torch_dtype():
                    raise ValueError("%s must be a contiguous CPU tensor of %s" % (n, self.torch_dtype()))
                ptrs.append(ctypes.c_void_p(a.data_ptr()))
            else:
                if a.dtype != want or not a.flags.c_contiguous or a.size != self.ncells:
                    raise ValueError("%s must be a contiguous %s array of %d elements"
                                     % (n, np.dtype(want).name, self.ncells))
                ptrs.append(ctypes.c_void_p(a.ctypes.data))
        check(_lib.lib.mpdata_solve_host(self._h, *ptrs, int(nsteps), _stream_handle(stream)),
              "mpdata_solve_host")

    def mass(self, h, psi, out=None, stream=None):
        """(sum h*psi, min psi, max psi) as a float64 CUDA tensor of 3 (async)."""
        torch = _torch()
        if out is None:
            out = torch.empty(3, dtype=torch.float64, device=psi.device)
        check(_lib.lib.mpdata_mass(self._h, self._dev(h, "h"), self._dev(psi, "psi"),
                                   ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "mpdata_mass")
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib.mpdata_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
