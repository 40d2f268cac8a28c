"""The headline configuration checked cell by cell: the 1024x512x64
rotation-blob grid (periodic x/y, lids in z) run by the production launch --
the default tile, i.e. row bands of 32x28 and 32x24 tiles (both with loader
warps) as two concurrent launches -- for 10 steps against the FP64 oracle on every
cell (max |dpsi| <= 1e-5 max|psi|)."""
import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_rotation_blobs_every_cell_10_steps():
    import paper_1507_01265_gb300 as mp
    f = F.rotation_blobs()
    with mp.Solver(f.nx, f.ny, f.nz, periodic=f.periodic) as s:
        assert s.bands == (14, 5)
    got = run_gpu(f, 10)
    want = run_oracle(f, 10, omp=True)
    assert rel_err(got, want) <= 1e-5, rel_err(got, want)
    assert got.min() >= 0.0
