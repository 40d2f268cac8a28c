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
    assert (o.extrema, o.precision) == (mp._lib.MPDATA_EXTREMA_BOTH, mp._lib.MPDATA_PREC_PURE)


def test_header_constants_match_binding(mp):
    """Every #define MPDATA_* of the header has the same value in the binding."""
    text = open(os.path.join(ROOT, "include", "mpdata.h")).read()
    defs = dict(re.findall(r"#define\s+(MPDATA_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    assert len(defs) >= 20
    for name, value in defs.items():
        bound = getattr(mp._lib, name, getattr(mp._lib, name[len("MPDATA_"):], None))
        assert bound == int(value), name


def test_invalid_arguments_without_gpu(mp):
    L = mp._lib
    h = ctypes.c_void_p()
    o = L.default_opts()
    assert L.lib.mpdata_create(0, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    assert "dims" in L.last_error_message()
    o.iterations = 4
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    # options the fused kernel lacks are refused on the fused path
    for field, value in (("iterations", 3), ("extrema", L.MPDATA_EXTREMA_CORRECTED),
                         ("precision", L.MPDATA_PREC_F64_BETA)):
        o = L.default_opts()
        setattr(o, field, value)
        assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
        assert "MPDATA_PATH_STAGES" in L.last_error_message()
    for field in ("extrema", "precision"):
        o = L.default_opts()
        o.path = L.MPDATA_PATH_STAGES
        setattr(o, field, 2)
        assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    o = L.default_opts()
    o.eps = 0.0
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    o = L.default_opts()
    o.tile_x, o.tile_y = 7, 9
    assert L.lib.mpdata_create(4, 4, 4, ctypes.byref(o), ctypes.byref(h)) == L.MPDATA_EINVAL
    assert L.lib.mpdata_step(None, None, None, None, None, None, 1, None) == L.MPDATA_EINVAL
    assert L.lib.mpdata_courant_max(None, None, None, None, None, None, None) == L.MPDATA_EINVAL
    assert L.lib.mpdata_destroy(None) == L.MPDATA_OK


def test_strerror(mp):
    L = mp._lib
    assert L.strerror(L.MPDATA_EINVAL) == "invalid argument"
    assert L.strerror(L.MPDATA_EBUSY).startswith("busy")
    assert "sm_103a" in L.version()
