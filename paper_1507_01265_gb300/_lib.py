"""ctypes binding of libmpdata (include/mpdata.h).

Argument marshalling only: every step of the advection scheme runs in the
CUDA kernels of libmpdata.so.  There is no CPU fallback -- if the library is
missing, importing this module raises.  PyTorch is used for device memory
and streams (tensors are passed by data pointer, streams by handle).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpdata.so")

MPDATA_OK = 0
MPDATA_EINVAL = -1
MPDATA_ENOMEM = -2
MPDATA_ECUDA = -3
MPDATA_EBUSY = -4
MPDATA_ETIMEDOUT = -5
MPDATA_ENOENT = -6
MPDATA_ECANCELED = -7

MPDATA_F32 = 0
MPDATA_F64 = 1
MPDATA_PATH_FUSED = 0
MPDATA_PATH_STAGES = 1
MPDATA_EXTREMA_BOTH = 0
MPDATA_EXTREMA_CORRECTED = 1
MPDATA_PREC_PURE = 0
MPDATA_PREC_F64_BETA = 1


class Opts(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("iterations", ctypes.c_int32),
                ("nonoscillatory", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3),
                ("dtype", ctypes.c_int32), ("path", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("eps", ctypes.c_double),
                ("extrema", ctypes.c_int32), ("precision", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int32), ("max_queued", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("nonoscillatory", ctypes.c_int32), ("inject_alloc_failure", ctypes.c_int32),
                ("eps", ctypes.c_double), ("retain_finished", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3), ("nsteps", ctypes.c_int32),
                ("h", ctypes.c_void_p), ("u1", ctypes.c_void_p), ("u2", ctypes.c_void_p),
                ("u3", ctypes.c_void_p), ("psi", ctypes.c_void_p)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)


class MpdataError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s (%d): %s" % (what, strerror(code), code, last_error_message()))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmpdata.so is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I = ctypes.c_void_p, ctypes.c_int
    D = ctypes.c_double
    H = ctypes.c_void_p  # mpdata_t*
    sig = {
        "mpdata_opts_default": (None, [ctypes.POINTER(Opts)]),
        "mpdata_create": (I, [I, I, I, ctypes.POINTER(Opts), ctypes.POINTER(H)]),
        "mpdata_destroy": (I, [H]),
        "mpdata_get_tile": (I, [H, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mpdata_get_bands": (I, [H, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mpdata_plan_bands": (I, [I, I, I, ctypes.POINTER(I), I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mpdata_default_tile": (I, [I, I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mpdata_step": (I, [H, P, P, P, P, P, I, P]),
        "mpdata_solve_host": (I, [H, P, P, P, P, P, I, P]),
        "mpdata_host_submit": (I, [H, P, P, P, P, P, I, P, P, ctypes.POINTER(ctypes.c_ulonglong)]),
        "mpdata_host_wait": (I, [H, ctypes.c_ulonglong]),
        "mpdata_mass": (I, [H, P, P, P, P]),
        "mpdata_mass_noalloc": (I, [P, P, ctypes.c_longlong, I, P, P]),
        "mpdata_courant_max": (I, [H, P, P, P, P, P, P]),
        "mpdata_batch_create": (I, [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(Opts), ctypes.POINTER(H)]),
        "mpdata_batch_create_tiles": (I, [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(Opts), ctypes.POINTER(H)]),
        "mpdata_batch_grid_variant": (I, [H, I, ctypes.POINTER(I)]),
        "mpdata_batch_set_fields": (I, [H, I, P, P, P, P, P]),
        "mpdata_batch_work": (I, [H, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mpdata_batch_get_split": (I, [H, I, ctypes.POINTER(I)]),
        "mpdata_batch_set_split": (I, [H, I, I, ctypes.POINTER(I)]),
        "mpdata_batch_step": (I, [H, I, I, P]),
        "mpdata_batch_destroy": (I, [H]),
        "mpdata_server_opts_default": (None, [ctypes.POINTER(ServerOpts)]),
        "mpdata_server_create": (I, [ctypes.POINTER(ServerOpts), ctypes.POINTER(H)]),
        "mpdata_submit": (I, [H, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "mpdata_poll": (I, [H, ctypes.c_uint64, ctypes.POINTER(I)]),
        "mpdata_wait": (I, [H, ctypes.c_uint64, I]),
        "mpdata_cancel": (I, [H, ctypes.c_uint64]),
        "mpdata_request_times": (I, [H, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
        "mpdata_release": (I, [H, ctypes.c_uint64]),
        "mpdata_server_retained": (I, [H, ctypes.POINTER(ctypes.c_uint64)]),
        "mpdata_server_stats": (I, [H, ctypes.POINTER(ctypes.c_double)]),
        "mpdata_server_destroy": (I, [H]),
        "mpdata_fpm_algorithm1": (I, [D, I, D, P, P, I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "mpdata_fpm_partition": (I, [D, I, D, P, P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "mpdata_fpm_condition2": (I, [P, P, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "mpdata_strerror": (ctypes.c_char_p, [I]),
        "mpdata_last_error_message": (ctypes.c_char_p, []),
        "mpdata_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def strerror(code: int) -> str:
    return lib.mpdata_strerror(code).decode()


def last_error_message() -> str:
    return lib.mpdata_last_error_message().decode()


def version() -> str:
    return lib.mpdata_version().decode()


def check(code: int, what: str) -> None:
    if code != MPDATA_OK:
        raise MpdataError(code, what)


def default_opts() -> Opts:
    o = Opts()
    lib.mpdata_opts_default(ctypes.byref(o))
    return o
