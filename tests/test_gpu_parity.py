"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP32 state, max|dpsi| <= 1e-5 max|psi| after 10 steps and
<= 1e-4 max|psi| after 100 steps; FP64 GPU path <= 1e-12 relative.  Exact
cases (shift at Courant 1, constant fields) are compared bit for bit."""
import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import oracle_at, rand_problem, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


# ---- the 64x32x16 parity configuration --------------------------------------------------

@pytest.mark.parametrize("path", ["fused", "stages"])
def test_gaussian_constant_f32_10_steps(path):
    f = F.gaussian_constant()
    got = run_gpu(f, 10, path=path)
    want = run_oracle(f, 10)
    assert rel_err(got, want) <= 1e-5


@pytest.mark.parametrize("path", ["fused", "stages"])
def test_gaussian_constant_f32_100_steps(path):
    f = F.gaussian_constant()
    got = run_gpu(f, 100, path=path)
    want = run_oracle(f, 100)
    assert rel_err(got, want) <= 1e-4


@pytest.mark.parametrize("path", ["fused", "stages"])
def test_gaussian_constant_f64(path):
    f = F.gaussian_constant()
    got = run_gpu(f, 10, dtype="f64", path=path)
    want = run_oracle(f, 10)
    assert rel_err(got, want) <= 1e-12


# ---- edge shapes: ragged tiles, tiny grids, lids on every axis --------------------------

EDGE = [
    (37, 23, 11, (1, 1, 1)), (5, 3, 2, (1, 1, 1)), (1, 1, 1, (1, 1, 1)), (1, 1, 1, (0, 0, 0)),
    (9, 40, 7, (0, 1, 0)), (70, 5, 3, (1, 0, 0)), (33, 17, 20, (1, 1, 0)), (64, 32, 16, (0, 0, 0)),
    (32, 16, 4, (1, 1, 1)), (31, 15, 6, (0, 1, 1)), (65, 33, 3, (1, 0, 1)), (2, 70, 2, (0, 0, 1)),
    # nx % 4 == 0: 16-byte loads in the two-column kernel (others: 4-byte loads)
    (40, 30, 10, (0, 1, 1)), (36, 50, 5, (1, 0, 1)), (8, 8, 8, (0, 0, 0)), (4, 3, 2, (1, 1, 1)),
    (100, 26, 9, (1, 1, 0)), (64, 49, 6, (1, 0, 0)), (96, 24, 4, (1, 1, 1)), (4, 1, 1, (0, 1, 0)),
]


@pytest.mark.parametrize("nx,ny,nz,per", EDGE)
@pytest.mark.parametrize("nonosc", [True, False])
def test_edge_shapes_f64(nx, ny, nz, per, nonosc):
    f = rand_problem((nz, ny, nx), seed=nx * 131 + ny * 7 + nz, periodic=per)
    want = run_oracle(f, 3, nonosc=nonosc)
    for path in ("fused", "stages"):
        got = run_gpu(f, 3, dtype="f64", path=path, nonosc=nonosc)
        assert rel_err(got, want) <= 1e-12, path


@pytest.mark.parametrize("nx,ny,nz,per", EDGE)
@pytest.mark.parametrize("tile", [None, (24, 24), (16, 16), (32, 12), (32, 16), (32, 24), (32, 28)])
def test_edge_shapes_f32(nx, ny, nz, per, tile):
    f = rand_problem((nz, ny, nx), seed=nx * 17 + ny * 5 + nz, periodic=per)
    want = run_oracle(f, 3)
    got = run_gpu(f, 3, tile=tile)
    assert rel_err(got, want) <= 1e-5


@pytest.mark.parametrize("per", [(1, 1, 0), (0, 0, 1)])
@pytest.mark.parametrize("nx", [64, 63, 66, 33])
def test_pair_kernel_matches_single_column_kernel(per, nx):
    f = rand_problem((12, 40, nx), seed=21, periodic=per)
    a = run_gpu(f, 6, tile=(32, 24))   # two columns per thread
    a28 = run_gpu(f, 6, tile=(32, 28))
    assert np.array_equal(a, a28)      # same arithmetic whatever the tile
    b = run_gpu(f, 6, tile=(24, 24))   # one column per thread
    assert rel_err(a, b) <= 1e-6


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_donor_only(dtype):
    f = rand_problem((9, 14, 33), seed=3, periodic=(1, 0, 1))
    got = run_gpu(f, 4, dtype=dtype, iterations=1)
    want = run_oracle(f, 4, iterations=1)
    assert rel_err(got, want) <= (1e-5 if dtype == "f32" else 1e-12)


# ---- stage-path options: three passes, extrema set, FP64 limiter sums -------------------

OPTION_SHAPES = [(37, 23, 11, (1, 1, 1)), (9, 40, 7, (0, 1, 0)), (64, 32, 16, (0, 0, 0)),
                 (5, 3, 2, (1, 1, 1)), (33, 17, 20, (1, 1, 0))]
OPTIONS = [(3, "both"), (3, "corrected"), (2, "corrected")]


@pytest.mark.parametrize("nx,ny,nz,per", OPTION_SHAPES)
@pytest.mark.parametrize("iterations,extrema", OPTIONS)
@pytest.mark.parametrize("nonosc", [True, False])
def test_stage_options_f64(nx, ny, nz, per, iterations, extrema, nonosc):
    f = rand_problem((nz, ny, nx), seed=nx * 7 + ny * 3 + nz, periodic=per)
    want = run_oracle(f, 3, iterations=iterations, nonosc=nonosc, extrema=extrema)
    got = run_gpu(f, 3, dtype="f64", path="stages", iterations=iterations, nonosc=nonosc,
                  extrema=extrema)
    assert rel_err(got, want) <= 1e-12


@pytest.mark.parametrize("nx,ny,nz,per", OPTION_SHAPES)
@pytest.mark.parametrize("iterations,extrema", OPTIONS)
@pytest.mark.parametrize("precision", ["pure", "f64_beta"])
def test_stage_options_f32(nx, ny, nz, per, iterations, extrema, precision):
    f = rand_problem((nz, ny, nx), seed=nx * 11 + ny * 5 + nz, periodic=per)
    want = run_oracle(f, 3, iterations=iterations, extrema=extrema)
    got = run_gpu(f, 3, path="stages", iterations=iterations, extrema=extrema, precision=precision)
    assert rel_err(got, want) <= 1e-5


@pytest.mark.parametrize("iterations", [2, 3])
def test_f64_beta_gaussian_constant_100_steps(iterations):
    f = F.gaussian_constant()
    got = run_gpu(f, 100, path="stages", iterations=iterations, precision="f64_beta")
    want = run_oracle(f, 100, iterations=iterations)
    assert rel_err(got, want) <= 1e-4


def test_f64_beta_is_a_no_op_for_f64():
    f = rand_problem((6, 20, 24), seed=41, periodic=(1, 1, 0))
    a = run_gpu(f, 3, dtype="f64", path="stages", precision="f64_beta")
    b = run_gpu(f, 3, dtype="f64", path="stages")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_three_passes_shift_exact(dtype):
    shape = (5, 12, 17)
    r = np.random.default_rng(12)
    psi = r.integers(1, 2 ** 20, size=shape).astype(np.float32)
    for axis in range(3):
        u = [np.zeros(shape, np.float32) for _ in range(3)]
        u[axis][:] = -1.0
        f = F.Fields("shift3", shape[2], shape[1], shape[0], (1, 1, 1),
                     np.ones(shape, np.float32), psi, u[0], u[1], u[2], 2, 0)
        for extrema in ("both", "corrected"):
            got = run_gpu(f, 2, dtype=dtype, path="stages", iterations=3, extrema=extrema)
            assert np.array_equal(got, np.roll(psi.astype(np.float64), -2, axis=2 - axis))


# ---- exact cases ------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("path", ["fused", "stages"])
def test_shift_at_courant_one_is_exact(dtype, path):
    shape = (6, 20, 37)
    r = np.random.default_rng(11)
    psi = r.integers(1, 2 ** 20, size=shape).astype(np.float32)
    for axis in range(3):
        for sign in (1.0, -1.0):
            u = [np.zeros(shape, np.float32) for _ in range(3)]
            u[axis][:] = sign
            f = F.Fields("shift", shape[2], shape[1], shape[0], (1, 1, 1),
                         np.ones(shape, np.float32), psi, u[0], u[1], u[2], 3, 0)
            got = run_gpu(f, 3, dtype=dtype, path=path)
            assert np.array_equal(got, np.roll(psi.astype(np.float64), int(sign) * 3, axis=2 - axis))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_constant_is_preserved_exactly(dtype):
    nx, ny, nz = 70, 41, 9
    u1, u2, u3 = F.rotation_courant(nx, ny, nz, 0.5)
    h = F.sine_density(nx, ny, nz)
    psi = np.full((nz, ny, nx), 3.25, np.float32)
    f = F.Fields("const", nx, ny, nz, (1, 1, 0), h, psi, u1, u2, u3, 5, 0)
    got = run_gpu(f, 5, dtype=dtype)
    assert np.all(got == 3.25)


# ---- conservation and diagnostics -------------------------------------------------------

def test_mass_conservation_and_diagnostics():
    import torch
    import oracle
    import paper_1507_01265_gb300 as mp
    f = rand_problem((12, 30, 45), seed=5, periodic=(1, 1, 0))
    dev = torch.device("cuda")
    for dtype, tol in (("f64", 1e-12), ("f32", 1e-5)):
        td = torch.float64 if dtype == "f64" else torch.float32
        t = [torch.from_numpy(a).to(dev, td) for a in (f.h, f.psi, f.u1, f.u2, f.u3)]
        with mp.Solver(f.nx, f.ny, f.nz, periodic=f.periodic, dtype=dtype) as s:
            m0 = s.mass(t[0], t[1]).cpu().numpy()
            ref = oracle.mass(t[0].double().cpu().numpy(), t[1].double().cpu().numpy())
            assert abs(m0[0] / ref - 1) <= 1e-14
            assert m0[1] == t[1].min().item() and m0[2] == t[1].max().item()
            s.step(*t, 10)
            m1 = s.mass(t[0], t[1]).cpu().numpy()
            assert abs(m1[0] / m0[0] - 1) <= tol, dtype
            again = s.mass(t[0], t[1]).cpu().numpy()
            assert np.array_equal(m1, again)  # bit-reproducible


def test_solve_host_and_odd_steps_match_step():
    import torch
    import paper_1507_01265_gb300 as mp
    f = rand_problem((8, 19, 27), seed=9)
    a = run_gpu(f, 5)
    b = run_gpu(f, 2)
    b = run_gpu(f, 3, psi=b.astype(np.float32))
    assert np.array_equal(a, b)
    psi = f.psi.copy()
    with mp.Solver(f.nx, f.ny, f.nz) as s:
        s.solve_host(f.h, psi, f.u1, f.u2, f.u3, 5)
        s.solve_host(f.h, psi, f.u1, f.u2, f.u3, 0)
    assert np.array_equal(psi.astype(np.float64), a)
    torch.cuda.synchronize()


def test_fused_matches_stage_per_kernel():
    f = F.rotation_blobs(nx=96, ny=64, nz=24, nsteps=6)
    a = run_gpu(f, 6, path="fused")
    b = run_gpu(f, 6, path="stages")
    assert rel_err(a, b) <= 1e-6


def test_bad_pointers_are_rejected():
    import torch
    import paper_1507_01265_gb300 as mp
    with mp.Solver(8, 8, 8) as s:
        t = torch.zeros(8 * 8 * 8 + 1, device="cuda")
        view = t[1:]  # 4-byte offset: not 16-byte aligned
        with pytest.raises(mp.MpdataError) as e:
            s.step(view, view, view, view, view, 1)
        assert e.value.code == -1


# ---- the 1024x512x64 roofline configuration, in the launch configuration bench.py times ---

@pytest.mark.parametrize("nsteps", [1, 2])
def test_rotation_blobs_full_size_sampled(nsteps):
    f = F.rotation_blobs()  # 1024 x 512 x 64, periodic x/y, lids in z
    got = run_gpu(f, nsteps)
    r = np.random.default_rng(100 + nsteps)
    samples = [(int(r.integers(f.nz)), int(r.integers(f.ny)), int(r.integers(f.nx)))
               for _ in range(120)]
    samples += [(0, 0, 0), (f.nz - 1, f.ny - 1, f.nx - 1), (0, f.ny - 1, 5), (f.nz - 1, 3, f.nx - 1)]
    want = oracle_at(f, samples, nsteps)
    vals = np.array([got[s] for s in samples])
    scale = float(np.abs(f.psi).max())
    assert np.abs(vals - want).max() <= 1e-5 * scale


@pytest.mark.parametrize("nx,ny,per,tile", [
    (1021, 509, (1, 1, 0), (32, 24)),   # odd nx: 4-byte loads, ghost column wraps
    (1022, 510, (0, 1, 0), (32, 28)),   # nx % 4 == 2 with an x lid
    (1021, 512, (1, 0, 0), None),       # odd nx with a y lid, default tile
])
def test_ragged_full_size_sampled(nx, ny, per, tile):
    """Full-size grids whose nx is not a multiple of 4 (the 4-byte load path
    and the per-column stores), sampled against the oracle, with the cells
    next to the x edges always among the samples."""
    f = F.rotation_blobs(nx=nx, ny=ny, nz=64, periodic=per, nsteps=2)
    got = run_gpu(f, 2, tile=tile)
    r = np.random.default_rng(nx + ny)
    samples = [(int(r.integers(f.nz)), int(r.integers(f.ny)), int(r.integers(f.nx)))
               for _ in range(80)]
    for i in (0, 1, 2, nx - 3, nx - 2, nx - 1):
        samples.append((int(r.integers(f.nz)), int(r.integers(f.ny)), i))
    samples += [(0, 0, 0), (f.nz - 1, f.ny - 1, f.nx - 1)]
    want = oracle_at(f, samples, 2)
    vals = np.array([got[s] for s in samples])
    assert np.abs(vals - want).max() <= 1e-5 * float(np.abs(f.psi).max())


def test_rotation_blobs_full_size_invariants():
    import torch
    import paper_1507_01265_gb300 as mp
    f = F.rotation_blobs()
    dev = torch.device("cuda")
    t = [torch.from_numpy(a).to(dev) for a in (f.h, f.psi, f.u1, f.u2, f.u3)]
    with mp.Solver(f.nx, f.ny, f.nz, periodic=f.periodic) as s:
        m0 = s.mass(t[0], t[1]).cpu().numpy()
        s.step(*t, 20)
        m1 = s.mass(t[0], t[1]).cpu().numpy()
    assert abs(m1[0] / m0[0] - 1) <= 1e-5
    assert m1[1] >= m0[1] - 1e-6 * m0[2] and m1[2] <= m0[2] * (1 + 1e-6)


# ---- stability diagnostic ----------------------------------------------------------------

def _outflow_courant_max(f, periodic):
    """max_c sum_d ([U_d(c + e_d)]+ - [U_d(c)]-) / h_c written out with numpy;
    lid faces (index 0 and n on a lid axis) carry no velocity."""
    out = np.zeros((f.nz, f.ny, f.nx))
    for d, u in enumerate((f.u1, f.u2, f.u3)):
        a = 2 - d
        u = u.astype(np.float64)
        lower, upper = u.copy(), np.roll(u, -1, axis=a)
        if not periodic[d]:
            n = u.shape[a]
            lower[tuple(slice(0, 1) if x == a else slice(None) for x in range(3))] = 0.0
            upper[tuple(slice(n - 1, n) if x == a else slice(None) for x in range(3))] = 0.0
        out += np.maximum(upper, 0.0) - np.minimum(lower, 0.0)
    return float((out / f.h.astype(np.float64)).max())


@pytest.mark.parametrize("per", [(1, 1, 1), (1, 1, 0), (0, 1, 1), (0, 0, 0)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_courant_max(per, dtype):
    import torch
    import paper_1507_01265_gb300 as mp
    f = rand_problem((7, 19, 33), seed=61, umax=0.3, periodic=per)
    td = torch.float64 if dtype == "f64" else torch.float32
    t = [torch.from_numpy(a).to("cuda", td) for a in (f.h, f.u1, f.u2, f.u3)]
    with mp.Solver(f.nx, f.ny, f.nz, periodic=per, dtype=dtype) as s:
        got = s.courant_max(*t)
    assert got == pytest.approx(_outflow_courant_max(f, per), rel=1e-15, abs=0)


def test_courant_max_closed_forms():
    import torch
    import paper_1507_01265_gb300 as mp
    # constant Courant vector, h = 1: every cell moves sum_d |C_d| out
    nx, ny, nz = 24, 10, 6
    u = F.constant_courant(nx, ny, nz, (0.25, -0.125, 0.5))
    h = np.ones((nz, ny, nx), np.float32)
    t = [torch.from_numpy(a).cuda() for a in (h,) + u]
    with mp.Solver(nx, ny, nz) as s:
        assert s.courant_max(*t) == 0.875
    # with lids on z, the top cells have no upper z-face: still 0.875 elsewhere,
    # and a field whose only velocity sits on the lid faces gives 0
    uz = [np.zeros((nz, ny, nx), np.float32) for _ in range(3)]
    uz[2][0] = 0.7
    t = [torch.from_numpy(a).cuda() for a in [h] + uz]
    with mp.Solver(nx, ny, nz, periodic=(1, 1, 0)) as s:
        assert s.courant_max(*t) == 0.0


def test_default_tile_choice():
    """The default tile follows the predicted step time: the two-column
    kernel with 32x28 tiles for the 1024x512 grid (608 tiles, four full
    waves on 152 SMs, against five of 32x24) and for 4096x2048 (63 waves of
    1.91 us per plane against 73 of 1.67: 32x24 is not the 2 % better that
    displaces the first candidate), the fastest single-CTA plane for a grid
    too small to fill the GPU (32x12 with its loader warp, 1.11 us, when
    nx % 4 == 0; else 32x16 or 16x16 at 1.45 each), 16x16 for FP64."""
    import torch
    import paper_1507_01265_gb300 as mp
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    with mp.Solver(40, 24, 12) as s:
        assert s.tile == (32, 12)
    with mp.Solver(42, 24, 12) as s:
        assert s.tile in ((16, 16), (32, 16))
    with mp.Solver(64, 64, 8, dtype="f64") as s:
        assert s.tile == (16, 16)
    with mp.Solver(64, 64, 8, path="stages") as s:
        assert s.tile == (0, 0)
    for nx, ny, nz in ((40, 24, 12), (42, 24, 12), (512, 256, 16), (1024, 512, 8), (300, 40, 4)):
        with mp.Solver(nx, ny, nz, periodic=(1, 1, 0)) as s:
            assert s.tile == mp.default_tile(nx, ny, nz, nsm=nsm), (nx, ny, nz)
    if nsm == 152:
        with mp.Solver(1024, 512, 64, periodic=(1, 1, 0)) as s:
            assert s.tile == (32, 28)
        with mp.Solver(4096, 2048, 32, periodic=(1, 1, 0)) as s:
            assert s.tile == (32, 28)


@pytest.mark.parametrize("nonosc", [True, False])
@pytest.mark.parametrize("nx,ny,nz,bands,per", [(1024, 512, 4, (14, 5), (1, 1, 0)), (2048, 1024, 2, (28, 10), (1, 1, 0)),
                                                (1024, 512, 3, (14, 5), (1, 0, 1)), (1024, 512, 3, (14, 5), (0, 1, 0))])
def test_row_bands(nx, ny, nz, bands, per, nonosc):
    """With the default tile a large x/y-periodic grid runs in rows of 32x28
    and 32x24 bands, two concurrent launches per step.  Every cell is computed
    by the same arithmetic as with one tile shape: the banded result equals
    both single-shape results bit for bit."""
    import torch
    import paper_1507_01265_gb300 as mp
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("band plans are tuned for 152 SMs")
    f = rand_problem((nz, ny, nx), seed=ny + nz, periodic=per)
    with mp.Solver(nx, ny, nz, periodic=per) as s:
        assert s.bands == bands
    banded = run_gpu(f, 3, nonosc=nonosc)
    for tile in ((32, 28), (32, 24)):
        with mp.Solver(nx, ny, nz, periodic=per, tile=tile) as s:
            assert s.bands == (0, 0)
        assert np.array_equal(banded, run_gpu(f, 3, tile=tile, nonosc=nonosc)), tile


def test_row_bands_in_a_cuda_graph():
    """A banded step forks onto the handle's stream and joins back; captured
    into a CUDA graph by the caller it replays to the eager result."""
    import torch
    import paper_1507_01265_gb300 as mp
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("band plans are tuned for 152 SMs")
    nx, ny, nz = 1024, 512, 3
    f = rand_problem((nz, ny, nx), seed=5, periodic=(1, 1, 0))
    eager = run_gpu(f, 4)
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.h, f.psi, f.u1, f.u2, f.u3)]
    with mp.Solver(nx, ny, nz, periodic=(1, 1, 0)) as s:
        assert s.bands != (0, 0)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            s.step(*t, 2, stream=side)  # warm up outside the capture (kernel attributes)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        t[1].copy_(torch.from_numpy(np.ascontiguousarray(f.psi)))
        with torch.cuda.graph(g):
            s.step(*t, 2, stream=torch.cuda.current_stream())
        g.replay()
        g.replay()
        torch.cuda.synchronize()
    assert np.array_equal(t[1].double().cpu().numpy(), eager)


@pytest.mark.parametrize("ty", [12, 24, 28])
@pytest.mark.parametrize("nonosc", [True, False])
@pytest.mark.parametrize("nx,ny,nz,per", [
    (96, 50, 9, (1, 1, 0)), (128, 61, 7, (1, 1, 1)), (64, 24, 33, (1, 1, 0)), (32, 5, 4, (1, 1, 1)),
    (96, 50, 9, (0, 1, 0)), (128, 61, 7, (1, 0, 1)), (64, 57, 12, (0, 0, 0)), (40, 30, 10, (0, 1, 1)),
    (4, 3, 2, (0, 0, 0)), (8, 52, 5, (1, 0, 0)),
])
def test_loader_warp_tile(nx, ny, nz, per, nonosc, ty):
    """32x12, 32x24 and 32x28 tiles of grids with nx % 4 == 0 (lids on x or
    y included) run the two-column kernel with loader warps (the compute
    warps issue no loads; the 32x24 tile's last compute warp carries 8 idle
    threads; the 32x12 tile has one loader warp and two CTAs per SM).  It
    matches the oracle and, bit for bit, the 32x28 tile and the batch's
    persistent kernel, whose CTAs run several tiles each and whose loader
    warps therefore cross from tile to tile (24 and 28 rows)."""
    import torch
    import paper_1507_01265_gb300 as mp
    f = rand_problem((nz, ny, nx), seed=nx + ny + nz, periodic=per)
    got = run_gpu(f, 10, tile=(32, ty), nonosc=nonosc)
    assert rel_err(got, run_oracle(f, 10, nonosc=nonosc)) <= 1e-5
    if ty == 12:
        assert np.array_equal(got, run_gpu(f, 10, tile=(32, 28), nonosc=nonosc))
        return
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.h, f.psi, f.u1, f.u2, f.u3)]
    with mp.Batch([(nx, ny, nz, per)], tile=(32, ty), nonoscillatory=nonosc) as b:
        v = b.grid_variant(0)
        lid = not (per[0] and per[1])
        assert v == {(24, False): 2, (24, True): 7, (28, False): 8, (28, True): 9}[(ty, lid)]
        n, _ = b.work(v)
        b.set_balanced_split(v, max(1, n // 3))
        b.set_fields(0, *t)
        b.step(10)
        torch.cuda.synchronize()
    assert np.array_equal(t[1].double().cpu().numpy(), got)


@pytest.mark.parametrize("nx,ny,nz,per", [
    (8192, 2, 3, (1, 1, 0)),    # a thin slab: the y halo wraps several times
    (2, 4000, 5, (0, 1, 1)),    # a narrow column: every pair straddles the x lid
    (4, 4, 3000, (1, 1, 0)),    # a long z-march
    (3, 1, 2000, (1, 1, 1)),
])
def test_extreme_aspect_ratios(nx, ny, nz, per):
    f = rand_problem((nz, ny, nx), seed=nx + 7 * ny + 3 * nz, periodic=per)
    want = run_oracle(f, 2)
    for tile in (None, (32, 28)):
        assert rel_err(run_gpu(f, 2, tile=tile), want) <= 1e-5, tile
    assert rel_err(run_gpu(f, 2, dtype="f64"), want) <= 1e-12
