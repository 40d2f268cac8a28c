"""Batched launches: every grid of a batch gives exactly (bit for bit) what
mpdata_step gives on that grid alone, whatever the mix of grids, the work
split between CTAs (one CTA per tile by default, balanced persistent, uneven),
odd or even step counts, or graph replay -- and matches the FP64 oracle
(max |dpsi| <= 1e-5 max|psi| for up to 10 steps)."""
import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import rand_problem, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1507_01265_gb300 as mp
    return mp


MIX = [  # (nx, ny, nz, periodic): x/y periodic or lids; nx % 4 == 0 (16-byte loads) or not
    (64, 40, 12, (1, 1, 1)), (36, 50, 7, (1, 1, 0)), (40, 30, 10, (0, 1, 1)),
    (37, 23, 11, (1, 1, 1)), (9, 40, 7, (0, 1, 0)), (96, 24, 4, (1, 0, 1)), (4, 3, 2, (1, 1, 1)),
]


def _fields(mp, fs):
    import torch
    return [[torch.from_numpy(a).cuda() for a in (f.h, f.psi, f.u1, f.u2, f.u3)] for f in fs]


def _batch(mp, fs, tile=(32, 24), nonosc=True):
    return mp.Batch([(f.nx, f.ny, f.nz, f.periodic) for f in fs], tile=tile, nonoscillatory=nonosc)


@pytest.mark.parametrize("nsteps", [1, 4, 5])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("nonosc", [True, False])
def test_batch_equals_alone(mp, nsteps, graph, nonosc):
    import torch
    fs = [rand_problem((nz, ny, nx), seed=i + 40, periodic=per) for i, (nx, ny, nz, per) in enumerate(MIX)]
    ts = _fields(mp, fs)
    with _batch(mp, fs, nonosc=nonosc) as b:
        for i, t in enumerate(ts):
            b.set_fields(i, *t)
        b.step(nsteps, graph=graph)
        b.step(nsteps, graph=graph)  # a second run reuses the cached graph
        torch.cuda.synchronize()
    for f, t in zip(fs, ts):
        got = t[1].double().cpu().numpy()
        alone = run_gpu(f, 2 * nsteps, nonosc=nonosc, tile=(32, 24))  # the batch tile
        assert np.array_equal(got, alone), f.name
        assert rel_err(got, run_oracle(f, 2 * nsteps, nonosc=nonosc, omp=True)) <= 1e-5, f.name


def test_uneven_and_degenerate_splits(mp):
    import torch
    fs = [F.tracer_grid(nx, ny, nz, c, seed=7 + i, nsteps=3)
          for i, (nx, ny, nz, c) in enumerate(F.tracer_batch_dims(count=12, seed=77))]
    ts = _fields(mp, fs)
    with _batch(mp, fs, tile=(32, 16)) as b:
        for i, t in enumerate(ts):
            b.set_fields(i, *t)
        for v in range(mp.Batch.VARIANTS):
            n, ncta = b.work(v)
            if n == 0:
                continue
            split = b.get_split(v)
            assert split[0] == 0 and split[-1] == n and all(a <= c for a, c in zip(split, split[1:]))
            # every item on CTA 0 except one item on the last CTA, the rest empty
            b.set_split(v, [0] + [n - 1] * (ncta - 1) + [n])
        b.step(3)
        torch.cuda.synchronize()
    for f, t in zip(fs, ts):
        got = t[1].double().cpu().numpy()
        assert np.array_equal(got, run_gpu(f, 3, tile=(32, 16))), f.name
        assert rel_err(got, run_oracle(f, 3, omp=True)) <= 1e-5, f.name


@pytest.mark.parametrize("graph", [False, True])
def test_default_and_balanced_splits(mp, graph):
    """The default split gives every work item its own CTA; the balanced
    persistent split runs min(ncta, items) CTAs over contiguous ranges.  Both
    give every grid the bits of its run alone."""
    import torch
    fs = [F.tracer_grid(nx, ny, nz, c, seed=90 + i, nsteps=3)
          for i, (nx, ny, nz, c) in enumerate(F.tracer_batch_dims(count=10, seed=78))]
    results = []
    for balanced in (False, True):
        ts = _fields(mp, fs)
        with _batch(mp, fs) as b:
            for i, t in enumerate(ts):
                b.set_fields(i, *t)
            for v in range(mp.Batch.VARIANTS):
                n, ncta = b.work(v)
                if n == 0:
                    assert ncta == 0
                    continue
                assert ncta == n and b.get_split(v) == list(range(n + 1))
                if balanced:
                    b.set_balanced_split(v, 5)
                    n2, ncta2 = b.work(v)
                    split = b.get_split(v)
                    assert n2 == n and ncta2 == min(5, n) and len(split) == ncta2 + 1
                    assert split[0] == 0 and split[-1] == n and all(a <= c for a, c in zip(split, split[1:]))
                    with pytest.raises(mp.MpdataError):
                        b.set_balanced_split(v, 0)
            b.step(3, graph=graph)
            torch.cuda.synchronize()
        results.append([t[1].double().cpu().numpy() for t in ts])
    for f, a, c in zip(fs, *results):
        alone = run_gpu(f, 3, tile=(32, 24))
        assert np.array_equal(a, alone) and np.array_equal(c, alone), f.name
        assert rel_err(a, run_oracle(f, 3, omp=True)) <= 1e-5, f.name


def test_bad_split_is_rejected(mp):
    fs = [rand_problem((4, 8, 32), seed=1)]
    with _batch(mp, fs) as b:
        n, ncta = b.work(0)
        with pytest.raises(mp.MpdataError):
            b.set_split(0, [0, n + 1])
        with pytest.raises(mp.MpdataError):
            b.set_split(0, [1, n])
        with pytest.raises(mp.MpdataError):
            b.step(1)  # fields not set


@pytest.mark.parametrize("graph", [False, True])
def test_per_grid_tiles(mp, graph):
    """Each grid runs with its own tile height; every result equals the
    single-grid run with that tile, and the grids land in the documented
    variants."""
    import torch
    tiles = [16, 24, 0, 28, 24, 16, 28]
    fs = [rand_problem((nz, ny, nx), seed=i + 80, periodic=per) for i, (nx, ny, nz, per) in enumerate(MIX)]
    ts = _fields(mp, fs)
    with mp.Batch([(f.nx, f.ny, f.nz, f.periodic) for f in fs], tiles=tiles) as b:
        want = []
        for i, (f, ty) in enumerate(zip(fs, tiles)):
            lid = not (f.periodic[0] and f.periodic[1])
            if (ty or 24) == 24 and f.nx % 4 == 0:  # 32x24 with loader warps
                want.append(7 if lid else 2)
            elif ty == 28 and f.nx % 4 == 0:  # 32x28 with loader warps
                want.append(9 if lid else 8)
            else:
                want.append({24: 0, 16: 3, 28: 5}[ty or 24] + int(lid))
        assert [b.grid_variant(i) for i in range(len(fs))] == want
        for i, t in enumerate(ts):
            b.set_fields(i, *t)
        b.step(3, graph=graph)
        torch.cuda.synchronize()
    for f, t, ty in zip(fs, ts, tiles):
        got = t[1].double().cpu().numpy()
        assert np.array_equal(got, run_gpu(f, 3, tile=(32, ty or 24))), (f.name, ty)
        assert rel_err(got, run_oracle(f, 3, omp=True)) <= 1e-5, (f.name, ty)


def test_bad_tile_heights_are_rejected(mp):
    fs = [rand_problem((4, 8, 32), seed=1), rand_problem((4, 8, 32), seed=2)]
    with pytest.raises(mp.MpdataError):
        mp.Batch([(f.nx, f.ny, f.nz, f.periodic) for f in fs], tiles=[16, 8])
    with pytest.raises(ValueError):
        mp.Batch([(f.nx, f.ny, f.nz, f.periodic) for f in fs], tiles=[16])
