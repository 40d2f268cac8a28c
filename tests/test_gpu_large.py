"""A grid of more than 2^31 cells (4096 x 4096 x 136, 2.28 G cells, 55 GB of
FP32 fields on the device): plane offsets beyond the 32-bit range.  The
fields are integer formulas, so the host rebuilds any window of them bit for
bit and the oracle checks sampled cells of the top planes, whose element
offsets exceed 2^31."""
import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import oracle_at

pytestmark = pytest.mark.gpu

NX, NY, NZ = 4096, 4096, 136
COURANT = (0.2, -0.15, 0.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_grid_beyond_2_31_cells():
    import torch
    import paper_1507_01265_gb300 as mp
    free, _ = torch.cuda.mem_get_info()
    need = 7 * NX * NY * NZ * 4 + (4 << 30)
    if free < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    n = NX * NY * NZ
    assert n >= 2 ** 31
    dev = torch.device("cuda")
    fields = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(5)]
    h, psi, u1, u2, u3 = fields
    j = torch.arange(NY, device=dev, dtype=torch.int64)[:, None]
    i = torch.arange(NX, device=dev, dtype=torch.int64)[None, :]
    plane = NX * NY
    for k in range(NZ):
        sl = slice(k * plane, (k + 1) * plane)
        psi[sl] = (1.0 + ((i * 7 + j * 13 + k * 29) % 97).float() / 97.0).reshape(-1)
        h[sl] = (1.0 + ((i + 2 * j + 3 * k) % 5).float() / 10.0).reshape(-1)
    u1.fill_(COURANT[0])
    u2.fill_(COURANT[1])
    u3.fill_(COURANT[2])
    u3[:plane].zero_()  # lid face 0
    nsteps = 2
    with mp.Solver(NX, NY, NZ, periodic=(1, 1, 0)) as s:
        m0 = s.mass(h, psi).cpu().numpy()
        s.step(h, psi, u1, u2, u3, nsteps)
        m1 = s.mass(h, psi).cpu().numpy()
        torch.cuda.synchronize()
    assert abs(m1[0] / m0[0] - 1) <= 1e-6
    samples = [(NZ - 1, NY - 1, NX - 1), (NZ - 1, 0, 0), (NZ - 2, 2000, 3000), (NZ - 1, 17, 4095),
               (NZ // 2, 4095, 1), (0, 5, 7)]
    W = 3 * nsteps + 2
    for (k, jj, ii) in samples:
        assert (k * NY + jj) * NX + ii < n
        # a window around the cell (wrapped in x/y, clipped at the z lids)
        ks = np.arange(max(0, k - W), min(NZ, k + W + 1))
        js = np.arange(jj - W, jj + W + 1) % NY
        is_ = np.arange(ii - W, ii + W + 1) % NX
        K, J, I = np.meshgrid(ks, js, is_, indexing="ij")
        wpsi = (1.0 + ((I * 7 + J * 13 + K * 29) % 97).astype(np.float32) / np.float32(97.0)).astype(np.float32)
        wh = (1.0 + ((I + 2 * J + 3 * K) % 5).astype(np.float32) / np.float32(10.0)).astype(np.float32)
        shape = wpsi.shape
        wu = [np.full(shape, c, np.float32) for c in COURANT]
        if ks[0] == 0:
            wu[2][0] = 0.0
        f = F.Fields("window", shape[2], shape[1], shape[0], (0, 0, 0), wh, wpsi, wu[0], wu[1], wu[2],
                     nsteps, 0)
        want = oracle_at(f, [(k - ks[0], W, W)], nsteps)[0]
        got = float(psi[(k * NY + jj) * NX + ii].item())
        assert abs(got - want) <= 1e-5 * 2.0, ((k, jj, ii), got, want)
    del fields
    torch.cuda.empty_cache()
