"""Pins of the FP64 oracle: facts fixed by the mathematics of the MPDATA
scheme, none of them a restatement of the oracle's own formulas.

Each pin takes an oracle library handle (so the same pins can be run against
mutated copies of the oracle) and raises AssertionError when the oracle
breaks it.  Together they are meant to catch a plausible mistake anywhere in
the step: a flipped sign, a dropped term, a wrong face index, a transposed
axis, h in the wrong place, a limiter that does nothing.

  shift            Courant number exactly +-1 along one axis: the step is a
                   pure shift (donor flux = upwind value, antidiffusive
                   coefficient |U| - U^2/h = 0), bit-exact for integers.
  constant         psi = const stays const bit-exactly for fields whose face
                   values do not vary along their own axis.
  mass             sum h psi is conserved (flux form), also with lids.
  positivity       psi >= 0 stays >= 0 under the Courant bound.
  monotone         with the limiter no new global extrema appear on a square
                   wave; without it they do.
  binomial         iterations = 1 in 1D is the binomial closed form of the
                   donor-cell scheme.
  convergence_1d   second order on a smooth Gaussian (h = 1 and h varying).
  convergence_2d   second order for diagonal flow in each coordinate plane
                   (only true with correct cross terms).
  scale            (h, U) -> (2h, 2U) leaves the equation unchanged.
  mirror           reflecting an axis (u on that axis negated, faces
                   re-staggered) reflects the result.
  permute          cycling the axes cycles the result.
  lid_face         the stored face-0 value on a lid axis is not read.
  lid_wall         a lid is a reflecting wall: a lid domain of n cells gives
                   the first half of the periodic domain of 2n cells that
                   holds the mirror-extended problem.
  local_bounds     the limiter's defining property: each corrected value lies
                   within the extrema of its 7-point stencil over the chosen
                   set (psi^n and the corrected field, or the corrected field
                   alone), for any h > 0 and any flow, with 2 or 3 passes.
  extrema_set      the two sets differ where they should: with psi^n in the
                   set a corrective pass may rebuild a peak that the donor
                   pass flattened; without it, it may not.
  iterations3      a second corrective pass lowers the error of a smooth
                   solution and keeps the second order.

Shift, constant and mass also run with three passes.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


def _run(lib, shape, h, psi, u, nsteps, periodic=(1, 1, 1), iterations=2, nonosc=1, eps=1e-15,
         extrema=0):
    nz, ny, nx = shape
    cfg = O.Config(nx, ny, nz, tuple(periodic), iterations, nonosc, eps, extrema)
    return O.run(cfg, h, psi, u[0], u[1], u[2], nsteps, lib=lib)


def _axis_shape(axis, n):
    shp = [1, 1, 1]
    shp[2 - axis] = n
    return tuple(shp)


def pin_shift(lib, steps=3):
    r = _rng(1)
    shape = (4, 5, 6)
    psi = r.integers(1, 2 ** 20, size=shape).astype(np.float64)
    h = np.ones(shape)
    for axis in range(3):
        for sign in (1.0, -1.0):
            for nonosc, iterations in ((0, 2), (1, 2), (1, 3)):
                u = [np.zeros(shape) for _ in range(3)]
                u[axis][:] = sign
                out = _run(lib, shape, h, psi, u, steps, nonosc=nonosc, iterations=iterations)
                want = np.roll(psi, int(sign) * steps, axis=2 - axis)
                assert np.array_equal(out, want), ("shift", axis, sign, nonosc, iterations)


def pin_constant(lib, steps=3):
    import gen.fields as F
    r = _rng(2)
    shape = (5, 6, 7)
    c = 3.25
    psi = np.full(shape, c)
    h = r.uniform(0.5, 2.0, size=shape)
    u = [np.full(shape, v) for v in (0.3, -0.2, 0.1)]
    for iterations, extrema in ((2, 0), (3, 0), (3, 1)):
        out = _run(lib, shape, h, psi, u, steps, iterations=iterations, extrema=extrema)
        assert np.array_equal(out, psi), ("constant: constant U, random h", iterations, extrema)
    nz, ny, nx = 6, 10, 12
    u1, u2, u3 = F.rotation_courant(nx, ny, nz, 0.5)
    h = F.sine_density(nx, ny, nz)
    psi = np.full((nz, ny, nx), c)
    out = _run(lib, (nz, ny, nx), h, psi, [u1, u2, u3], steps, periodic=(1, 1, 0))
    assert np.array_equal(out, psi), "constant: rotation, lid z"


def _random_problem(seed, shape, umax=0.12, lid=None):
    r = _rng(seed)
    psi = r.uniform(1.0, 2.0, size=shape)
    h = r.uniform(0.8, 1.25, size=shape)
    u = [r.uniform(-umax, umax, size=shape) for _ in range(3)]
    if lid is not None:
        # lid faces carry no velocity; zero the stored face-0 values too
        sl = [slice(None)] * 3
        sl[2 - lid] = 0
        u[lid][tuple(sl)] = 0.0
    return h, psi, u


def pin_mass(lib, steps=5):
    shape = (6, 7, 8)
    for periodic, lid in (((1, 1, 1), None), ((1, 1, 0), 2), ((0, 1, 1), 0), ((1, 0, 0), 1)):
        h, psi, u = _random_problem(3, shape, lid=lid)
        for d in range(3):
            if not periodic[d]:
                sl = [slice(None)] * 3
                sl[2 - d] = 0
                u[d][tuple(sl)] = 0.0
        m0 = O.mass(h, psi, lib=lib)
        for nonosc, iterations in ((0, 2), (1, 2), (1, 3)):
            out = _run(lib, shape, h, psi, u, steps, periodic=periodic, nonosc=nonosc,
                       iterations=iterations)
            m1 = O.mass(h, out, lib=lib)
            assert abs(m1 / m0 - 1.0) <= 1e-12, ("mass", periodic, nonosc, iterations, m1 / m0 - 1.0)


def pin_positivity(lib, steps=10):
    shape = (8, 9, 10)
    h, _, u = _random_problem(4, shape, umax=0.12)
    z, y, x = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    r2 = (x - 5) ** 2 + (y - 4.5) ** 2 + (z - 4) ** 2
    psi = np.maximum(0.0, np.exp(-r2 / 6.0) - 0.2)  # exact zeros outside a ball
    for nonosc in (0, 1):
        out = _run(lib, shape, h, psi, u, steps, nonosc=nonosc)
        assert out.min() >= 0.0, ("positivity", nonosc, out.min())


def pin_monotone(lib, steps=20):
    shape = (8, 10, 12)
    psi = np.ones(shape)
    psi[2:6, 3:7, 3:8] = 3.0
    h = np.ones(shape)
    for uvec in ((0.2, -0.15, 0.1), (-0.1, 0.25, -0.2)):
        u = [np.full(shape, v) for v in uvec]
        out = _run(lib, shape, h, psi, u, steps, nonosc=1)
        assert out.max() <= 3.0 + 1e-12 and out.min() >= 1.0 - 1e-12, ("monotone", uvec)
        out0 = _run(lib, shape, h, psi, u, steps, nonosc=0)
        assert out0.max() > 3.0 + 1e-3 or out0.min() < 1.0 - 1e-3, ("limiter-off overshoot", uvec)


def pin_binomial(lib, steps=9, n=37):
    r = _rng(5)
    for axis in range(3):
        shp = _axis_shape(axis, n)
        psi = r.uniform(0.0, 1.0, size=shp)
        p0 = psi.reshape(-1)
        for C in (0.3, -0.3):
            u = [np.zeros(shp) for _ in range(3)]
            u[axis][:] = C
            out = _run(lib, shp, np.ones(shp), psi, u, steps, iterations=1).reshape(-1)
            a = abs(C)
            want = np.zeros(n)
            for kk in range(steps + 1):
                w = math.comb(steps, kk) * a ** kk * (1 - a) ** (steps - kk)
                want += w * np.roll(p0, kk if C > 0 else -kk)
            assert np.allclose(out, want, rtol=1e-13, atol=0), ("binomial", axis, C)


def _gauss_1d(n, sigma):
    x = np.arange(n) + 0.5
    return 1.0 + np.exp(-(x - n / 2) ** 2 / (2 * sigma ** 2))


def convergence_1d(lib, axis, C, hvar, nonosc, sizes=(64, 128, 256)):
    errs = []
    for n in sizes:
        shp = _axis_shape(axis, n)
        psi = _gauss_1d(n, n / 16).reshape(shp)
        x = np.arange(n) + 0.5
        h = (1.0 + hvar * np.sin(2 * np.pi * x / n)).reshape(shp)
        u = [np.zeros(shp) for _ in range(3)]
        u[axis][:] = C
        # one transit: the characteristic speed U/h has mean U over a period
        out = _run(lib, shp, h, psi, u, int(round(n / abs(C))), nonosc=nonosc)
        errs.append(math.sqrt(np.mean((out - psi) ** 2)))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def pin_convergence_1d(lib):
    for axis, C, hvar in ((0, 0.25, 0.0), (1, -0.25, 0.0), (2, -0.25, 0.2), (0, 0.25, 0.2)):
        for nonosc in (0, 1):
            orders = convergence_1d(lib, axis, C, hvar, nonosc)
            assert min(orders) >= 1.75, ("convergence_1d", axis, C, hvar, nonosc, orders)


def convergence_2d(lib, axes, sizes, nonosc=0, c=(0.2, 0.1)):
    errs = []
    for n in sizes:
        shp = [1, 1, 1]
        for a in axes:
            shp[2 - a] = n
        shp = tuple(shp)
        g = np.exp(-(np.arange(n) + 0.5 - n / 2) ** 2 / (2 * (n / 8) ** 2))
        psi = (1.0 + 2.0 * np.outer(g, g)).reshape(shp)
        u = [np.zeros(shp) for _ in range(3)]
        u[axes[0]][:] = c[0]
        u[axes[1]][:] = c[1]
        steps = int(round(n / min(abs(c[0]), abs(c[1]))))  # whole transits on both axes
        out = _run(lib, shp, np.ones(shp), psi, u, steps, nonosc=nonosc)
        errs.append(math.sqrt(np.mean((out - psi) ** 2)))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def pin_convergence_2d(lib, sizes=(16, 32, 64), threshold=1.75):
    for axes in ((0, 1), (1, 2), (2, 0)):
        orders = convergence_2d(lib, axes, sizes)
        assert orders[-1] >= threshold, ("convergence_2d", axes, orders)


def pin_scale(lib, steps=3):
    shape = (5, 6, 7)
    for periodic in ((1, 1, 1), (1, 1, 0)):
        h, psi, u = _random_problem(6, shape, lid=None if periodic[2] else 2)
        for nonosc in (0, 1):
            a = _run(lib, shape, h, psi, u, steps, periodic=periodic, nonosc=nonosc)
            b = _run(lib, shape, 2 * h, psi, [2 * v for v in u], steps, periodic=periodic,
                     nonosc=nonosc)
            assert np.allclose(a, b, rtol=1e-12, atol=0), ("scale", periodic, nonosc)


def _mirror(axis, h, psi, u):
    """Reflect the problem along one axis.  A face field on that axis is
    re-staggered (face f -> face n - f) and negated."""
    ax = 2 - axis
    fl = lambda a: np.flip(a, axis=ax)
    uu = []
    for d in range(3):
        if d == axis:
            # face f of the mirrored grid is face n - f of the original
            uu.append(-np.roll(fl(u[d]), 1, axis=ax))
        else:
            uu.append(fl(u[d]))
    return fl(h), fl(psi), uu


def pin_mirror(lib, steps=3):
    shape = (5, 6, 7)
    h, psi, u = _random_problem(7, shape)
    for nonosc in (0, 1):
        base = _run(lib, shape, h, psi, u, steps, nonosc=nonosc)
        for axis in range(3):
            mh, mp, mu = _mirror(axis, h, psi, u)
            out = _run(lib, shape, mh, mp, mu, steps, nonosc=nonosc)
            assert np.allclose(np.flip(out, axis=2 - axis), base, rtol=1e-13, atol=0), \
                ("mirror", axis, nonosc)


def pin_permute(lib, steps=3):
    shape = (5, 6, 7)  # (nz, ny, nx)
    h, psi, u = _random_problem(8, shape)
    # new axes: x' = y, y' = z, z' = x  -> array [z'][y'][x'] = [x][z][y]
    perm = lambda a: np.ascontiguousarray(np.transpose(a, (2, 0, 1)))
    for nonosc in (0, 1):
        base = _run(lib, shape, h, psi, u, steps, nonosc=nonosc)
        out = _run(lib, perm(psi).shape, perm(h), perm(psi), [perm(u[1]), perm(u[2]), perm(u[0])],
                   steps, nonosc=nonosc)
        assert np.allclose(out, perm(base), rtol=1e-13, atol=0), ("permute", nonosc)


def pin_lid_face(lib, steps=3):
    shape = (5, 6, 7)
    for lid in range(3):
        periodic = [1, 1, 1]
        periodic[lid] = 0
        h, psi, u = _random_problem(9, shape, lid=lid)
        a = _run(lib, shape, h, psi, u, steps, periodic=periodic)
        u2 = [v.copy() for v in u]
        sl = [slice(None)] * 3
        sl[2 - lid] = 0
        u2[lid][tuple(sl)] = 0.37
        b = _run(lib, shape, h, psi, u2, steps, periodic=periodic)
        assert np.array_equal(a, b), ("lid_face", lid)


def _wall_extend(axis, n, h, psi, u):
    """Mirror-extend a lid problem along `axis` into a periodic one of 2n
    cells: cell fields are reflected; the normal velocity is reflected about
    the wall faces 0 and n (which carry zero velocity) and negated."""
    ax = 2 - axis
    ext = lambda a: np.concatenate([a, np.flip(a, axis=ax)], axis=ax)
    uu = []
    for d in range(3):
        if d != axis:
            uu.append(ext(u[d]))
            continue
        faces = np.moveaxis(u[d], ax, 0).copy()
        faces[0] = 0.0  # wall face
        full = np.concatenate([faces, np.zeros_like(faces[:1]), -np.flip(faces[1:], axis=0)],
                              axis=0)
        uu.append(np.ascontiguousarray(np.moveaxis(full, 0, ax)))
    return ext(h), ext(psi), uu


def pin_lid_wall(lib, steps=3):
    shape = (6, 7, 8)
    for lid in range(3):
        for nonosc in (0, 1):
            periodic = [1, 1, 1]
            periodic[lid] = 0
            h, psi, u = _random_problem(10 + lid, shape, lid=lid)
            a = _run(lib, shape, h, psi, u, steps, periodic=periodic, nonosc=nonosc)
            n = shape[2 - lid]
            eh, ep, eu = _wall_extend(lid, n, h, psi, u)
            b = _run(lib, ep.shape, eh, ep, eu, steps, periodic=(1, 1, 1), nonosc=nonosc)
            b = np.take(b, np.arange(n), axis=2 - lid)
            assert np.allclose(a, b, rtol=1e-13, atol=0), ("lid_wall", lid, nonosc)


def _stencil(f, periodic):
    """f and its six face neighbours (c - e_d, c + e_d for each axis d):
    wrapped on a periodic axis, an edge copy beyond a lid."""
    out = [f]
    for d in range(3):
        a = 2 - d
        pad = [(0, 0)] * 3
        pad[a] = (1, 1)
        g = np.pad(f, pad, mode="wrap" if periodic[d] else "edge")
        n = f.shape[a]
        out.append(np.take(g, np.arange(0, n), axis=a))
        out.append(np.take(g, np.arange(2, n + 2), axis=a))
    return out


def _bounds(fields, periodic):
    vals = [v for f in fields for v in _stencil(f, periodic)]
    return np.maximum.reduce(vals), np.minimum.reduce(vals)


def _spiky_problem(seed, shape, umax, lid):
    h, _, u = _random_problem(seed, shape, umax=umax, lid=lid)
    r = _rng(seed + 100)
    psi = 0.01 + 10.0 * r.uniform(0.0, 1.0, size=shape) ** 6  # rough, strictly positive
    return h, psi, u


def pin_local_bounds(lib):
    """Corrected value within the stencil extrema of the bounding set.  From
    the limiter's definition: the limited inflow of a cell is at most
    beta_up * IN, so the pass adds at most (psi_max - p) h IN / (IN + eps) / h
    to p; likewise for the outflow and psi_min (requires psi >= 0)."""
    shape = (6, 7, 8)
    for seed, periodic, lid in ((20, (1, 1, 1), None), (21, (1, 1, 0), 2), (22, (0, 1, 1), 0)):
        h, psi, u = _spiky_problem(seed, shape, 0.15, lid)
        tol = 1e-12 * psi.max()
        for iterations in (2, 3):
            for extrema in (0, 1):
                if iterations == 2:
                    nz, ny, nx = shape
                    cfg = O.Config(nx, ny, nz, periodic, 1, 1, 1e-15)
                    prev = O.step(cfg, h, psi, u[0], u[1], u[2], lib=lib)
                else:
                    prev = _run(lib, shape, h, psi, u, 1, periodic=periodic, iterations=2,
                                extrema=extrema)
                mx, mn = _bounds([psi, prev] if extrema == 0 else [prev], periodic)
                out = _run(lib, shape, h, psi, u, 1, periodic=periodic, iterations=iterations,
                           extrema=extrema)
                assert np.all(out <= mx + tol) and np.all(out >= mn - tol), \
                    ("local_bounds", periodic, iterations, extrema,
                     float((out - mx).max()), float((mn - out).max()))


def pin_extrema_set(lib):
    """A one-cell spike moving at C = 0.3: the donor pass lowers it to 0.7 of
    its height; with psi^n in the bounding set the corrective pass raises it
    above that again, with the corrected field alone it stays at or below."""
    n = 24
    shp = _axis_shape(0, n)
    psi = np.full(shp, 0.1)
    psi.reshape(-1)[10] = 1.0
    u = [np.zeros(shp) for _ in range(3)]
    u[0][:] = 0.3
    h = np.ones(shp)
    cfg = O.Config(n, 1, 1, (1, 1, 1), 1, 1, 1e-15)
    psi1 = O.step(cfg, h, psi, u[0], u[1], u[2], lib=lib)
    mx1, _ = _bounds([psi1], (1, 1, 1))
    both = _run(lib, shp, h, psi, u, 1, extrema=0)
    only = _run(lib, shp, h, psi, u, 1, extrema=1)
    assert np.all(only <= mx1 + 1e-14), ("extrema_set: corrected-field-only bound", float((only - mx1).max()))
    assert (both - mx1).max() > 1e-3, ("extrema_set: psi^n not in the default set", float((both - mx1).max()))


def _err_1d(lib, axis, n, C, hvar, nonosc, iterations):
    shp = _axis_shape(axis, n)
    psi = _gauss_1d(n, n / 16).reshape(shp)
    x = np.arange(n) + 0.5
    h = (1.0 + hvar * np.sin(2 * np.pi * x / n)).reshape(shp)
    u = [np.zeros(shp) for _ in range(3)]
    u[axis][:] = C
    out = _run(lib, shp, h, psi, u, int(round(n / abs(C))), nonosc=nonosc, iterations=iterations)
    return math.sqrt(np.mean((out - psi) ** 2))


def pin_iterations3(lib, sizes=(64, 128, 256)):
    """Each corrective pass estimates and removes the leading error of the
    pass before (Smolarkiewicz 1984): a second one must lower the error of a
    smooth transit and keep second-order convergence."""
    for axis, C, hvar in ((0, 0.25, 0.0), (2, -0.5, 0.2), (1, 0.5, 0.0)):
        for nonosc in (0, 1):
            e2 = _err_1d(lib, axis, sizes[1], C, hvar, nonosc, 2)
            e3 = [_err_1d(lib, axis, n, C, hvar, nonosc, 3) for n in sizes]
            assert e3[1] <= 0.9 * e2, ("iterations3: no gain", axis, C, hvar, nonosc, e3[1] / e2)
            orders = [math.log2(e3[i] / e3[i + 1]) for i in range(len(e3) - 1)]
            assert min(orders) >= 1.75, ("iterations3: order", axis, C, hvar, nonosc, orders)


FAST_PINS = [pin_shift, pin_constant, pin_lid_face, pin_lid_wall, pin_mass, pin_scale, pin_mirror,
             pin_permute, pin_positivity, pin_monotone, pin_binomial, pin_local_bounds,
             pin_extrema_set, pin_iterations3]
