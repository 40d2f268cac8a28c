"""mpdata_mass_noalloc: the diagnostics entry point that allocates nothing
(its reduction scratch is a static device array inside the library), for
callers whose device memory is owned by someone else.  It must give the same
result as mpdata_mass, call after call, although every call reuses the same
static scratch.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1507_01265_gb300 as mp
    return mp


def _noalloc(mp, h, psi, dtype_code):
    import torch
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=psi.device)
    rc = mp._lib.lib.mpdata_mass_noalloc(
        ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(psi.data_ptr()), psi.numel(), dtype_code,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    mp.check(rc, "mpdata_mass_noalloc")
    return out


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_mass_matches_handle_mass_two_calls(mp, dtype):
    import torch
    from gpu_helpers import rand_problem
    td = torch.float64 if dtype == "f64" else torch.float32
    code = mp._lib.MPDATA_F64 if dtype == "f64" else mp._lib.MPDATA_F32
    # two calls in a row on different grids: the second must not see the
    # first call's partials
    for shape, seed in (((16, 40, 70), 1), ((5, 9, 13), 2)):
        f = rand_problem(shape, seed)
        h = torch.from_numpy(f.h).to("cuda", td)
        psi = torch.from_numpy(f.psi).to("cuda", td)
        with mp.Solver(f.nx, f.ny, f.nz, dtype=dtype) as s:
            ref = s.mass(h, psi).cpu().numpy()
        got = _noalloc(mp, h, psi, code).cpu().numpy()
        torch.cuda.synchronize()
        # same kernels, same fixed reduction tree: the same bits
        assert np.array_equal(got, ref), (shape, got, ref)


def test_noalloc_rejects_sizes_outside_the_limit(mp):
    import torch
    t = torch.ones(16, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    L = mp._lib
    for n in (0, -1, 1 << 31):
        rc = L.lib.mpdata_mass_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                       n, L.MPDATA_F32, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == L.MPDATA_EINVAL
        assert "2^31" in L.last_error_message()
