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
_EXTREMA = {"both": _lib.MPDATA_EXTREMA_BOTH, "corrected": _lib.MPDATA_EXTREMA_CORRECTED}
_PRECISION = {"pure": _lib.MPDATA_PREC_PURE, "f64_beta": _lib.MPDATA_PREC_F64_BETA}


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def default_tile(nx: int, ny: int, nz: int, dtype: str = "f32", nsm: int = 152):
    """(tile_x, tile_y): the fused tile a default-tile solver of this grid
    runs on a device of nsm SMs.  Host only."""
    a, b = ctypes.c_int(), ctypes.c_int()
    check(_lib.lib.mpdata_default_tile(int(nx), int(ny), int(nz), _DTYPES[dtype], int(nsm), ctypes.byref(a),
                                       ctypes.byref(b)), "mpdata_default_tile")
    return (a.value, b.value)


def plan_bands(nx: int, ny: int, nz: int, periodic=(1, 1, 0), nsm: int = 152):
    """(n28, n24): the row bands a default-tile FP32 solver of this grid runs
    on a device of nsm SMs ((0, 0): one tile shape).  Host only."""
    per = (ctypes.c_int * 3)(*[int(p) for p in periodic])
    a, b = ctypes.c_int(), ctypes.c_int()
    check(_lib.lib.mpdata_plan_bands(int(nx), int(ny), int(nz), per, int(nsm), ctypes.byref(a), ctypes.byref(b)),
          "mpdata_plan_bands")
    return (a.value, b.value)


class Solver:
    """One MPDATA problem size and option set (wraps an mpdata_t handle)."""

    def __init__(self, nx: int, ny: int, nz: int, *, periodic=(1, 1, 1), iterations: int = 2,
                 nonoscillatory: bool = True, dtype: str = "f32", path: str = "fused",
                 tile=None, eps: float = 1e-15, extrema: str = "both", precision: str = "pure"):
        """extrema: "both" (psi^n and the corrected field) or "corrected";
        precision: "pure" or "f64_beta" (FP32 fields, FP64 limiter sums).
        iterations = 3, extrema = "corrected" and precision = "f64_beta" run
        on path = "stages"."""
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
        o.extrema = _EXTREMA[extrema]
        o.precision = _PRECISION[precision]
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype_name = dtype
        self.opts = o
        self._h = ctypes.c_void_p()
        self._inflight = {}  # ticket -> host arrays of a submit_host not yet waited for
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

    def _host_ptr(self, a, name):
        import numpy as np
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.is_cuda or not a.is_contiguous() or a.dtype != self.torch_dtype() or a.numel() != self.ncells:
                raise ValueError("%s must be a contiguous CPU tensor of %d %s elements"
                                 % (name, self.ncells, self.torch_dtype()))
            return ctypes.c_void_p(a.data_ptr())
        want = np.float64 if self.dtype_name == "f64" else np.float32
        if a.dtype != want or not a.flags.c_contiguous or a.size != self.ncells:
            raise ValueError("%s must be a contiguous %s array of %d elements"
                             % (name, np.dtype(want).name, self.ncells))
        return ctypes.c_void_p(a.ctypes.data)

    def solve_host(self, h, psi, u1, u2, u3, nsteps: int, stream=None) -> None:
        """nsteps steps on host arrays (numpy or CPU tensors); psi is updated
        in place.  Copies in, steps and copies back inside the call."""
        ptrs = [self._host_ptr(a, n) for a, n in ((h, "h"), (psi, "psi"), (u1, "u1"), (u2, "u2"), (u3, "u3"))]
        check(_lib.lib.mpdata_solve_host(self._h, *ptrs, int(nsteps), _stream_handle(stream)),
              "mpdata_solve_host")

    def submit_host(self, h, psi, u1, u2, u3, nsteps: int, psi_out=None, stream=None) -> int:
        """Enqueue one solve of nsteps steps on host arrays and return its
        ticket at once; the copies of consecutive solves overlap each other's
        steps (page-locked arrays, e.g. torch pin_memory(), are needed for
        that).  The result lands in psi_out (default: psi) once
        wait_host(ticket) has returned; until then the arrays must not be
        touched.  The solver keeps references to them until that wait."""
        out = psi if psi_out is None else psi_out
        arrays = (h, psi, u1, u2, u3, out)
        ptrs = [self._host_ptr(a, n) for a, n in zip(arrays, ("h", "psi", "u1", "u2", "u3", "psi_out"))]
        t = ctypes.c_ulonglong()
        check(_lib.lib.mpdata_host_submit(self._h, *ptrs[:5], int(nsteps), ptrs[5],
                                          _stream_handle(stream), ctypes.byref(t)), "mpdata_host_submit")
        self._inflight[t.value] = arrays
        return t.value

    def wait_host(self, ticket: int) -> None:
        """Block until solve `ticket` (and every earlier one) has written its psi_out."""
        check(_lib.lib.mpdata_host_wait(self._h, int(ticket)), "mpdata_host_wait")
        for k in [k for k in self._inflight if k <= ticket]:
            del self._inflight[k]

    @property
    def bands(self):
        """(n28, n24): rows in n28 bands of 32x28 tiles, then n24 bands of
        32x24 tiles, run concurrently; (0, 0) when one tile shape runs."""
        a, b = ctypes.c_int(), ctypes.c_int()
        check(_lib.lib.mpdata_get_bands(self._h, ctypes.byref(a), ctypes.byref(b)), "mpdata_get_bands")
        return (a.value, b.value)

    @property
    def tile(self):
        """(tile_x, tile_y) of the fused kernel this solver runs; (0, 0) on the stage path."""
        tx, ty = ctypes.c_int(), ctypes.c_int()
        check(_lib.lib.mpdata_get_tile(self._h, ctypes.byref(tx), ctypes.byref(ty)), "mpdata_get_tile")
        return (tx.value, ty.value)

    def mass(self, h, psi, out=None, stream=None):
        """(sum h*psi, min psi, max psi) as a float64 CUDA tensor of 3 (async)."""
        torch = _torch()
        if out is None:
            out = torch.empty(3, dtype=torch.float64, device=psi.device)
        check(_lib.lib.mpdata_mass(self._h, self._dev(h, "h"), self._dev(psi, "psi"),
                                   ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "mpdata_mass")
        return out

    def courant_max(self, h, u1, u2, u3, stream=None) -> float:
        """Largest outflow Courant number over all cells (the donor pass keeps
        psi >= 0 while it is <= 1); waits for the result."""
        torch = _torch()
        out = torch.empty(3, dtype=torch.float64, device=h.device)
        check(_lib.lib.mpdata_courant_max(self._h, self._dev(h, "h"), self._dev(u1, "u1"),
                                          self._dev(u2, "u2"), self._dev(u3, "u3"),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "mpdata_courant_max")
        return float(out[2].item())

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib.mpdata_destroy(self._h)  # waits for the pipelined host solves
            self._h = ctypes.c_void_p()
            self._inflight = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent FP32 grids advanced together by batched launches
    (mpdata_batch_*; one CTA per tile by default, largest tiles first).
    `grids` is a list of (nx, ny, nz) or (nx, ny, nz, (px, py, pz)); fields
    are attached per grid with set_fields."""

    # 0/1: two-column 32x24 (x/y periodic / a lid; nx % 4 != 0), 2/7: 32x24
    # with loader warps (periodic / lid; nx % 4 == 0), 3/4: two-column 32x16,
    # 5/6: two-column 32x28 (nx % 4 != 0), 8/9: 32x28 with loader warps
    # (nx % 4 == 0)
    VARIANTS = 10

    def __init__(self, grids, *, nonoscillatory: bool = True, tile=(32, 24), eps: float = 1e-15,
                 periodic=(1, 1, 1), tiles=None):
        """tile: the default tile; tiles: optional per-grid tile heights
        (16, 24, 28, or 0 for the default)."""
        o = _lib.default_opts()
        o.nonoscillatory = int(bool(nonoscillatory))
        o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        o.eps = float(eps)
        for d in range(3):
            o.periodic[d] = int(periodic[d])
        n = len(grids)
        dims = (ctypes.c_int * (3 * n))()
        per = (ctypes.c_int * (3 * n))()
        self.shapes = []
        for i, gdef in enumerate(grids):
            nx, ny, nz = (int(v) for v in gdef[:3])
            p = gdef[3] if len(gdef) > 3 else periodic
            dims[3 * i:3 * i + 3] = [nx, ny, nz]
            per[3 * i:3 * i + 3] = [int(v) for v in p]
            self.shapes.append((nz, ny, nx))
        self._h = ctypes.c_void_p()
        if tiles is None:
            check(_lib.lib.mpdata_batch_create(n, dims, per, ctypes.byref(o), ctypes.byref(self._h)),
                  "mpdata_batch_create")
        else:
            if len(tiles) != n:
                raise ValueError("tiles needs one tile height per grid")
            ty = (ctypes.c_int * n)(*[int(v) for v in tiles])
            check(_lib.lib.mpdata_batch_create_tiles(n, dims, per, ty, ctypes.byref(o),
                                                     ctypes.byref(self._h)),
                  "mpdata_batch_create_tiles")
        self._keep = {}

    def grid_variant(self, i) -> int:
        """Variant (work list) that runs grid i."""
        v = ctypes.c_int()
        check(_lib.lib.mpdata_batch_grid_variant(self._h, int(i), ctypes.byref(v)),
              "mpdata_batch_grid_variant")
        return v.value

    def set_fields(self, i, h, psi, u1, u2, u3) -> None:
        torch = _torch()
        ptrs = []
        for t, name in ((h, "h"), (psi, "psi"), (u1, "u1"), (u2, "u2"), (u3, "u3")):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 \
                    or not t.is_contiguous():
                raise ValueError("%s of grid %d must be a contiguous float32 CUDA tensor" % (name, i))
            if t.numel() != self.shapes[i][0] * self.shapes[i][1] * self.shapes[i][2]:
                raise ValueError("%s of grid %d has the wrong size" % (name, i))
            ptrs.append(ctypes.c_void_p(t.data_ptr()))
        self._keep[i] = (h, psi, u1, u2, u3)
        check(_lib.lib.mpdata_batch_set_fields(self._h, int(i), *ptrs), "mpdata_batch_set_fields")

    def work(self, variant):
        n, c = ctypes.c_int(), ctypes.c_int()
        check(_lib.lib.mpdata_batch_work(self._h, int(variant), ctypes.byref(n), ctypes.byref(c)),
              "mpdata_batch_work")
        return n.value, c.value

    def get_split(self, variant):
        _, ncta = self.work(variant)
        buf = (ctypes.c_int * (ncta + 1))()
        check(_lib.lib.mpdata_batch_get_split(self._h, int(variant), buf), "mpdata_batch_get_split")
        return list(buf)

    def set_split(self, variant, begin) -> None:
        begin = [int(v) for v in begin]
        buf = (ctypes.c_int * len(begin))(*begin)
        check(_lib.lib.mpdata_batch_set_split(self._h, int(variant), len(begin) - 1, buf),
              "mpdata_batch_set_split")

    def set_balanced_split(self, variant, ncta: int) -> None:
        """Persistent split: min(ncta, items) CTAs, contiguous ranges of
        nearly equal estimated cost (items are ordered largest first)."""
        check(_lib.lib.mpdata_batch_set_split(self._h, int(variant), int(ncta), None),
              "mpdata_batch_set_split")

    def step(self, nsteps: int, graph: bool = False, stream=None) -> None:
        check(_lib.lib.mpdata_batch_step(self._h, int(nsteps), int(bool(graph)),
                                         _stream_handle(stream)), "mpdata_batch_step")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib.mpdata_batch_destroy(self._h)
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


class Server:
    """Continuous-batching server (mpdata_server_*): submit FP32 host fields,
    get a ticket, wait for psi to be written back in place."""

    def __init__(self, hbm_budget_bytes: int = 8 << 30, *, max_active: int = 256,
                 max_queued: int = 1 << 20, chunk_steps: int = 8, tile_y: int = 24,
                 nonoscillatory: bool = True, inject_alloc_failure: int = 0, eps: float = 1e-15,
                 retain_finished: int = 1 << 16):
        o = _lib.ServerOpts()
        _lib.lib.mpdata_server_opts_default(ctypes.byref(o))
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        o.max_active, o.max_queued, o.chunk_steps = int(max_active), int(max_queued), int(chunk_steps)
        o.tile_y, o.nonoscillatory = int(tile_y), int(bool(nonoscillatory))
        o.inject_alloc_failure, o.eps = int(inject_alloc_failure), float(eps)
        o.retain_finished = int(retain_finished)
        self._h = ctypes.c_void_p()
        check(_lib.lib.mpdata_server_create(ctypes.byref(o), ctypes.byref(self._h)),
              "mpdata_server_create")
        self._keep = {}

    @staticmethod
    def _ptr(a, n, name):
        import numpy as np
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
                raise ValueError("%s must be a contiguous float32 CPU tensor of %d elements" % (name, n))
            return a.data_ptr()
        if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
            raise ValueError("%s must be a contiguous float32 array of %d elements" % (name, n))
        return a.ctypes.data

    def submit(self, h, psi, u1, u2, u3, nsteps: int, periodic=(1, 1, 1), shape=None) -> int:
        """Queue a solve; psi (host) receives the result.  shape = (nz, ny, nx)
        defaults to psi.shape."""
        nz, ny, nx = shape if shape is not None else tuple(psi.shape)
        n = nx * ny * nz
        r = _lib.Request()
        r.size = ctypes.sizeof(_lib.Request)
        r.nx, r.ny, r.nz, r.nsteps = int(nx), int(ny), int(nz), int(nsteps)
        for d in range(3):
            r.periodic[d] = int(periodic[d])
        r.h, r.u1, r.u2, r.u3 = (self._ptr(a, n, nm) for a, nm in ((h, "h"), (u1, "u1"), (u2, "u2"), (u3, "u3")))
        r.psi = self._ptr(psi, n, "psi")
        t = ctypes.c_uint64()
        check(_lib.lib.mpdata_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "mpdata_submit")
        self._keep[t.value] = (h, psi, u1, u2, u3)
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int()
        check(_lib.lib.mpdata_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(st)), "mpdata_poll")
        return st.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> None:
        rc = _lib.lib.mpdata_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms))
        if rc != _lib.MPDATA_ETIMEDOUT:  # finished (or unknown): the server is done with the buffers
            self._keep.pop(ticket, None)
        check(rc, "mpdata_wait")

    def cancel(self, ticket: int) -> None:
        check(_lib.lib.mpdata_cancel(self._h, ctypes.c_uint64(ticket)), "mpdata_cancel")

    def times(self, ticket: int):
        """(submit, admit, done) in seconds since the server started."""
        t = (ctypes.c_double * 3)()
        check(_lib.lib.mpdata_request_times(self._h, ctypes.c_uint64(ticket), t), "mpdata_request_times")
        return tuple(t)

    def release(self, ticket: int) -> None:
        """Forget a finished request (mpdata_release)."""
        check(_lib.lib.mpdata_release(self._h, ctypes.c_uint64(ticket)), "mpdata_release")
        self._keep.pop(ticket, None)

    def retained(self) -> int:
        """Requests the server still holds (mpdata_server_retained)."""
        n = ctypes.c_uint64()
        check(_lib.lib.mpdata_server_retained(self._h, ctypes.byref(n)), "mpdata_server_retained")
        return n.value

    def stats(self) -> dict:
        v = (ctypes.c_double * 6)()
        check(_lib.lib.mpdata_server_stats(self._h, v), "mpdata_server_stats")
        return {"completed": int(v[0]), "cell_steps": v[1], "admitted_bytes": int(v[2]),
                "queued": int(v[3]), "resident": int(v[4]), "uptime_s": v[5]}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib.mpdata_server_destroy(self._h)
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
