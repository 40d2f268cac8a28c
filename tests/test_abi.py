"""The C ABI library loads and exports what include/*.h declares; argument
checks that need no GPU return the documented codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g
    g.build()
    import paper_1507_01265_gb300 as mp
    return mp


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(mpdata_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("mpdata_create", "mpdata_step", "mpdata_destroy", "mpdata_mass"):
        assert n in names


def test_every_declared_symbol_is_exported(mp):
    lib = ctypes.CDLL(mp._lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults(mp):
    o = mp._lib.default_opts()
    assert o.size == ctypes.sizeof(mp._lib.Opts)
    assert (o.iterations, o.nonoscillatory, tuple(o.periodic), o.dtype, o.path) == (2, 1, (1, 1, 1), 0, 0)
    assert o.eps == 1e-15


def test_invalid_arguments_without_gpu(mp):
    L = mp._lib
    h = ctypes.c_void_p()
    o = L.default_opts()
    assert L.lib.mpdata_create(0, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    assert "dims" in L.last_error_message()
    o.iterations = 3
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    o = L.default_opts()
    o.eps = 0.0
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    o = L.default_opts()
    o.tile_x, o.tile_y = 7, 9
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    assert L.lib.mpdata_step(None, None, None, None, None, None, 1, None) == L.MPDATA_EINVAL
    assert L.lib.mpdata_destroy(None) == L.MPDATA_OK


def test_strerror(mp):
    L = mp._lib
    assert L.strerror(L.MPDATA_EINVAL) == "invalid argument"
    assert L.strerror(L.MPDATA_EBUSY).startswith("busy")
    assert "sm_103a" in L.version()
