"""Functional-performance-model partitioning (§2-§4 of the paper), calling
the library's C implementation (mpdata_fpm_*).

A speed function is given as measured points (sizes, speeds): speed in work
units per second of one processor running a workload of that size while all
processors run.  Execution time of x is x / s(x)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check


def _table(xs, ss):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ss = np.ascontiguousarray(ss, dtype=np.float64)
    if xs.shape != ss.shape or xs.ndim != 1:
        raise ValueError("sizes and speeds must be 1-D arrays of the same length")
    return xs, ss


def algorithm1(n, p, dx, xs, ss):
    """Algorithm 1 as printed (even p): returns (x_left, x_right, t_min)."""
    xs, ss = _table(xs, ss)
    xl, xr, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(_lib.lib.mpdata_fpm_algorithm1(float(n), int(p), float(dx), xs.ctypes.data, ss.ctypes.data,
                                         len(xs), ctypes.byref(xl), ctypes.byref(xr), ctypes.byref(t)),
          "mpdata_fpm_algorithm1")
    return xl.value, xr.value, t.value


def partition(n, p, dx, xs, ss):
    """Any p: returns (k_right, x_left, x_right, t_min); k_right processors take
    x_right, the others x_left (k_right = 0: balanced)."""
    xs, ss = _table(xs, ss)
    k = ctypes.c_int()
    xl, xr, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(_lib.lib.mpdata_fpm_partition(float(n), int(p), float(dx), xs.ctypes.data, ss.ctypes.data,
                                        len(xs), ctypes.byref(k), ctypes.byref(xl), ctypes.byref(xr),
                                        ctypes.byref(t)), "mpdata_fpm_partition")
    return k.value, xl.value, xr.value, t.value


def condition2(xs, ss):
    """(True, x, x') if condition (2) holds on the table (load imbalancing may
    pay), else (False, None, None)."""
    xs, ss = _table(xs, ss)
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = _lib.lib.mpdata_fpm_condition2(xs.ctypes.data, ss.ctypes.data, len(xs), ctypes.byref(a),
                                        ctypes.byref(b))
    if rc < 0:
        check(rc, "mpdata_fpm_condition2")
    return (True, a.value, b.value) if rc == 1 else (False, None, None)
