"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the
same seeded inputs."""
from __future__ import annotations

import numpy as np

import gen.fields as F
import oracle


def rand_problem(shape, seed, umax=0.12, periodic=(1, 1, 1), hvar=True):
    """Random positive psi, random h in [0.8, 1.25] (or 1), random Courant
    numbers in [-umax, umax] (stable: 6 * umax < 0.8); float32-rounded."""
    r = np.random.default_rng(seed)
    nz, ny, nx = shape
    psi = r.uniform(0.5, 2.0, size=shape)
    h = r.uniform(0.8, 1.25, size=shape) if hvar else np.ones(shape)
    u = [r.uniform(-umax, umax, size=shape) for _ in range(3)]
    for d in range(3):
        if not periodic[d]:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            u[d][tuple(sl)] = 0.0
    f32 = lambda a: np.ascontiguousarray(a.astype(np.float32))
    return F.Fields("random_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, tuple(periodic), f32(h),
                    f32(psi), f32(u[0]), f32(u[1]), f32(u[2]), 3, seed)


def run_gpu(f: F.Fields, nsteps, dtype="f32", path="fused", iterations=2, nonosc=True,
            tile=None, psi=None, extrema="both", precision="pure"):
    import torch
    import paper_1507_01265_gb300 as mp
    td = torch.float64 if dtype == "f64" else torch.float32
    dev = torch.device("cuda")
    arrs = [f.h, f.psi if psi is None else psi, f.u1, f.u2, f.u3]
    t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev, td) for a in arrs]
    with mp.Solver(f.nx, f.ny, f.nz, periodic=f.periodic, iterations=iterations,
                   nonoscillatory=nonosc, dtype=dtype, path=path, tile=tile, extrema=extrema,
                   precision=precision) as s:
        s.step(t[0], t[1], t[2], t[3], t[4], nsteps)
        torch.cuda.synchronize()
    return t[1].double().cpu().numpy()


def oracle_lib(omp=True):
    """The oracle's OpenMP build (same bits as the serial one, all host
    cores) when it loads, else the serial build."""
    if omp:
        try:
            return oracle.load(omp=True)
        except Exception:  # noqa: BLE001  (no OpenMP on this host)
            pass
    return oracle.load()


def run_oracle(f: F.Fields, nsteps, iterations=2, nonosc=True, extrema="both", omp=False):
    cfg = oracle.Config(f.nx, f.ny, f.nz, tuple(f.periodic), iterations, int(nonosc), 1e-15,
                        {"both": 0, "corrected": 1}[extrema])
    return oracle.run(cfg, *f.as_f64(), nsteps=nsteps, lib=oracle_lib() if omp else None)


def rel_err(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


def oracle_at(f: F.Fields, samples, nsteps, nonosc=True):
    """Oracle value of psi after nsteps at each sampled cell (k, j, i),
    computed on a window around the cell.  The step's domain of dependence
    has radius 3, so a window of radius 3*nsteps + 2 gives the exact value at
    its centre whatever ghost rule its cut faces use; a window reaching a lid
    is clipped there, so the real lid is used."""
    W = 3 * nsteps + 2
    h, psi, u1, u2, u3 = f.as_f64()
    dims = (f.nz, f.ny, f.nx)
    per = (f.periodic[2], f.periodic[1], f.periodic[0])  # array axis order
    out = []
    for (k, j, i) in samples:
        idx = []
        win_per = []
        centre = []
        for ax, c in enumerate((k, j, i)):
            n = dims[ax]
            if per[ax] and 2 * W + 1 >= n:
                ids = np.arange(n)
                win_per.append(1)
                centre.append(c)
            elif per[ax]:
                ids = np.arange(c - W, c + W + 1) % n
                win_per.append(0)
                centre.append(W)
            else:
                lo, hi = max(0, c - W), min(n - 1, c + W)
                ids = np.arange(lo, hi + 1)
                win_per.append(0)
                centre.append(c - lo)
            idx.append(ids)
        sub = lambda a: np.ascontiguousarray(a[np.ix_(*idx)])
        wh, wp, w1, w2, w3 = (sub(a) for a in (h, psi, u1, u2, u3))
        wz, wy, wx = wp.shape
        cfg = oracle.Config(wx, wy, wz, (win_per[2], win_per[1], win_per[0]), 2, int(nonosc))
        res = oracle.run(cfg, wh, wp, w1, w2, w3, nsteps=nsteps)
        out.append(res[tuple(centre)])
    return np.array(out)
