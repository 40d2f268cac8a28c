"""The autotuner's measuring half on the GPU: speed functions taken with
every SM busy (§5.4's simultaneous measurement), the partitioner's split of
a real grid built from them (Algorithm 1 generalised, §4), and that split
installed on a batch -- whose result must stay the bits of the grid run
alone and match the oracle."""
import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1507_01265_gb300 as mp
    return mp


def test_speed_function_table(mp):
    from paper_1507_01265_gb300 import tune
    xs, ss = tune.speed_function((32, 16), xs=(1, 2, 3, 4), nz=8, steps=2)
    assert list(xs) == [1.0, 2.0, 3.0, 4.0]          # sizes strictly increasing
    assert np.all(np.isfinite(ss)) and np.all(ss > 0)
    # a CTA with more tiles is not faster per tile by more than a few per cent
    # than one with fewer, and not slower than half: a plausible, flat table
    per_tile = ss / xs
    assert np.all(per_tile > 0) and per_tile.max() / per_tile.min() < 4.0


def test_partitioned_split_runs_and_is_exact(mp):
    import torch
    from paper_1507_01265_gb300 import fpm, tune
    P = tune.num_sms()
    xs, ss = tune.speed_function((32, 16), xs=(1, 2, 3, 4), nz=8, steps=2)
    nx, ny, nz = 32 * 20, 16 * 19, 6              # 380 tiles of 32x16
    n = 20 * 19
    k, xl, xr, t_pred = fpm.partition(n, P, 1.0, xs, ss / (32 * 16 * 8))
    assert t_pred > 0 and 0 <= k <= P
    assert abs(k * xr + (P - k) * xl - n) < 1e-9 and xr >= n / P - 1e-9
    f = F.rotation_blobs(nx=nx, ny=ny, nz=nz, nblobs=3, seed=21)
    t = [torch.from_numpy(a).cuda() for a in (f.h, f.psi, f.u1, f.u2, f.u3)]
    with mp.Batch([(nx, ny, nz, f.periodic)], tile=(32, 16)) as b:
        b.set_fields(0, *t)
        v = b.grid_variant(0)
        items, ncta = b.work(v)
        assert items == n
        if k > 0:  # k CTAs take x_right tiles, the other P - k take x_left
            b.set_split(v, tune.split_for(n, P, k, xl, xr))
        else:
            b.set_balanced_split(v, P)
        split = b.get_split(v)
        assert split[0] == 0 and split[-1] == n
        b.step(4)
        torch.cuda.synchronize()
    got = t[1].double().cpu().numpy()
    assert np.array_equal(got, run_gpu(f, 4, tile=(32, 16)))
    assert rel_err(got, run_oracle(f, 4)) <= 1e-5


def test_tune_grid_report(mp):
    from paper_1507_01265_gb300 import tune
    rep = tune.tune_grid(32 * 20, 16 * 19, 8, steps=2, tiles=((32, 16),), xs_max=4)  # 380 tiles
    r = rep["shapes"]["32x16"]
    assert rep["chosen_tile"] == [32, 16] and r["tiles"] == 380
    for key in ("predicted_step_s", "balanced_step_s", "tuned_step_s", "per_tile_step_s"):
        assert r[key] > 0
    assert len(r["speed_x"]) == len(r["speed_cells_per_s"]) == 4
