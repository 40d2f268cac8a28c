"""Seeded synthetic MPDATA inputs: psi, h and the staggered Courant fields.

This module holds input generation only -- no step of the advection scheme.
Both the FP64 oracle and the CUDA path are fed from it: fields are generated
in float64, rounded to float32 (the GPU state type), and the oracle runs on
the float32-rounded values promoted back to float64, so both sides see
identical inputs.

Random draws come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a counter-based generator,
draw n = mix(seed + (n+1) * 0x9E3779B97F4A7C15); a double in [0, 1) is
(x >> 11) * 2^-53.

Layout: every array is [nz][ny][nx] (x fastest).  u1[k][j][i] is the
Courant number on the x-face between cells i-1 and i; u2, u3 likewise for
y and z.  Cell centres sit at i + 0.5.

Workloads (the paper's own runs are synthetic MPDATA domains of
240x240x128 and 480x480x128, §6; these recipes stand in for them):
  * ``gaussian_constant``: one Gaussian (sigma 4) on background 1 plus
    U[0, 0.01) noise, constant Courant vector, h = 1, all axes periodic
    (the 64x32x16 parity case);
  * ``rotation_blobs``: solid-body rotation about z scaled to max |C|,
    h = 1 + 0.1 sin(2 pi (i + 0.5) / nx), a sum of seeded Gaussian blobs
    (sigma U[8, 32], amplitude U[1, 4], centre uniform) on a background,
    periodic x/y and rigid lids in z (the 1024x512x64 roofline case and the
    2048x1024x64 precision case);
  * ``tracer_batch``: independent grids with log-uniform sizes and
    per-grid constant Courant vectors (the batched-launch case);
  * ``near_zero_blobs`` / ``truncated_blobs``: narrower blobs on a 1e-6
    background, or on exact zeros with a jump at a cutoff (the psi -> 0
    regime of the limiter).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Draws start .. start+n-1 of the SplitMix64 stream with this seed."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential uniform draws from one SplitMix64 seed."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def uniform(self, n: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        x = splitmix64(self.seed, self.pos, n)
        self.pos += n
        u = (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def scalar(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return float(self.uniform(1, lo, hi)[0])

    def log_uniform_int(self, lo: int, hi: int) -> int:
        v = math.exp(self.scalar(math.log(lo), math.log(hi)))
        return int(min(hi, max(lo, round(v))))


@dataclasses.dataclass
class Fields:
    """One MPDATA problem: float32 arrays [nz][ny][nx] plus its options."""

    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple
    h: np.ndarray
    psi: np.ndarray
    u1: np.ndarray
    u2: np.ndarray
    u3: np.ndarray
    nsteps: int
    seed: int

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def as_f64(self):
        """The float32-rounded inputs promoted to float64 (the oracle's view)."""
        return tuple(np.ascontiguousarray(a, dtype=np.float64)
                     for a in (self.h, self.psi, self.u1, self.u2, self.u3))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _axis_offsets(n: int, centre: float, periodic: bool) -> np.ndarray:
    d = np.arange(n, dtype=np.float64) + 0.5 - centre
    if periodic:
        d = d - n * np.round(d / n)  # minimum-image distance
    return d


def gaussian_sum(shape, periodic, background, blobs) -> np.ndarray:
    """background + sum_b A_b exp(-|x - c_b|^2 / (2 sigma_b^2)) in float64.

    Each blob is separable, exp(-dx^2/2s^2) exp(-dy^2/2s^2) exp(-dz^2/2s^2),
    so it is built as an outer product."""
    nz, ny, nx = shape
    out = np.full(shape, float(background), dtype=np.float64)
    for amp, cx, cy, cz, sig in blobs:
        s2 = 2.0 * sig * sig
        ex = np.exp(-_axis_offsets(nx, cx, periodic[0]) ** 2 / s2)
        ey = np.exp(-_axis_offsets(ny, cy, periodic[1]) ** 2 / s2)
        ez = np.exp(-_axis_offsets(nz, cz, periodic[2]) ** 2 / s2)
        out += amp * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return out


def draw_blobs(st: Stream, nblobs, nx, ny, nz, sigma=(8.0, 32.0), amp=(1.0, 4.0)):
    blobs = []
    for _ in range(nblobs):
        a = st.scalar(*amp)
        cx = st.scalar(0.0, nx)
        cy = st.scalar(0.0, ny)
        cz = st.scalar(0.0, nz)
        s = st.scalar(*sigma)
        blobs.append((a, cx, cy, cz, s))
    return blobs


def rotation_courant(nx, ny, nz, max_c):
    """Solid-body rotation about the z axis in Courant units:
    u1 = -w (j + 0.5 - ny/2) on x-faces, u2 = w (i + 0.5 - nx/2) on y-faces,
    u3 = 0, w = max_c / max((nx-1)/2, (ny-1)/2).  u1 does not vary along x
    and u2 does not vary along y, so the field is discretely divergence
    free."""
    w = max_c / max((nx - 1) / 2.0, (ny - 1) / 2.0, 1e-300)
    jj = np.arange(ny, dtype=np.float64) + 0.5 - ny / 2.0
    ii = np.arange(nx, dtype=np.float64) + 0.5 - nx / 2.0
    u1 = np.broadcast_to((-w * jj)[None, :, None], (nz, ny, nx))
    u2 = np.broadcast_to((w * ii)[None, None, :], (nz, ny, nx))
    u3 = np.zeros((nz, ny, nx))
    return _f32(u1), _f32(u2), _f32(u3)


def constant_courant(nx, ny, nz, c):
    shp = (nz, ny, nx)
    return (_f32(np.full(shp, c[0])), _f32(np.full(shp, c[1])), _f32(np.full(shp, c[2])))


def sine_density(nx, ny, nz, amp=0.1):
    i = np.arange(nx, dtype=np.float64) + 0.5
    row = 1.0 + amp * np.sin(2.0 * math.pi * i / nx)
    return _f32(np.broadcast_to(row[None, None, :], (nz, ny, nx)))


def gaussian_constant(nx=64, ny=32, nz=16, courant=(0.3, -0.2, 0.1), nsteps=10,
                      seed=1508) -> Fields:
    """Single Gaussian, sigma 4, about the grid centre on background 1, plus
    U[0, 0.01) noise from the seed; h = 1; all axes periodic."""
    st = Stream(seed)
    shape = (nz, ny, nx)
    psi = gaussian_sum(shape, (True, True, True), 1.0,
                       [(4.0, nx / 2.0, ny / 2.0, nz / 2.0, 4.0)])
    psi += st.uniform(psi.size, 0.0, 0.01).reshape(shape)
    u1, u2, u3 = constant_courant(nx, ny, nz, courant)
    return Fields("gaussian_constant_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, (1, 1, 1),
                  _f32(np.ones(shape)), _f32(psi), u1, u2, u3, nsteps, seed)


def rotation_blobs(nx=1024, ny=512, nz=64, max_c=0.5, nblobs=8, background=1.0,
                   nsteps=50, seed=1509, periodic=(1, 1, 0)) -> Fields:
    """Rotation field, sine density and seeded Gaussian blobs (see module doc)."""
    st = Stream(seed)
    shape = (nz, ny, nx)
    blobs = draw_blobs(st, nblobs, nx, ny, nz)
    per = tuple(bool(p) for p in periodic)
    psi = gaussian_sum(shape, per, background, blobs)
    u1, u2, u3 = rotation_courant(nx, ny, nz, max_c)
    return Fields("rotation_blobs_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, tuple(periodic),
                  sine_density(nx, ny, nz), _f32(psi), u1, u2, u3, nsteps, seed)


def tracer_batch_dims(count=64, seed=1510, lo=32, hi=512, zlo=16, zhi=64):
    """Per-grid (nx, ny, nz, courant) of the batched-tracer workload.  Each
    Courant component is U[-0.5, 0.5]; when sum |C| > 1 the vector is
    rescaled to sum |C| = 0.95 so that the donor-cell pass stays stable."""
    st = Stream(seed)
    out = []
    for _ in range(count):
        nx = st.log_uniform_int(lo, hi)
        ny = st.log_uniform_int(lo, hi)
        nz = st.log_uniform_int(zlo, zhi)
        c = st.uniform(3, -0.5, 0.5)
        s = float(np.abs(c).sum())
        if s > 1.0:
            c = c * (0.95 / s)
        out.append((nx, ny, nz, tuple(float(v) for v in c)))
    return out


def tracer_grid(nx, ny, nz, courant, seed, nsteps=20) -> Fields:
    st = Stream(seed)
    shape = (nz, ny, nx)
    blobs = draw_blobs(st, 4, nx, ny, nz, sigma=(max(2.0, min(nx, ny, nz) / 8.0),
                                                  max(3.0, min(nx, ny, nz) / 3.0)))
    psi = gaussian_sum(shape, (True, True, True), 1.0, blobs)
    u1, u2, u3 = constant_courant(nx, ny, nz, courant)
    return Fields("tracer_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, (1, 1, 1),
                  _f32(np.ones(shape)), _f32(psi), u1, u2, u3, nsteps, seed)


def precision_grid(nx=2048, ny=1024, nz=64, nsteps=100, seed=1512) -> Fields:
    """The precision-study grid: rotation_blobs with the blobs on a 1e-6
    background, so that values span six decades."""
    f = rotation_blobs(nx=nx, ny=ny, nz=nz, background=1e-6, nsteps=nsteps, seed=seed)
    return dataclasses.replace(f, name="precision_%dx%dx%d" % (nx, ny, nz))


def near_zero_blobs(nx, ny, nz, background=1e-6, nblobs=4, sigma=(2.0, 6.0), max_c=0.5,
                    nsteps=10, seed=1513, periodic=(1, 1, 0)) -> Fields:
    """The psi -> 0 regime of the limiter: rotation field, sine density and
    seeded Gaussian blobs (sigma U[2, 6], amplitude U[1, 4]) on a 1e-6
    background, so that values span six decades and the limiter's
    denominators are dominated by eps over most of the grid."""
    st = Stream(seed)
    shape = (nz, ny, nx)
    blobs = draw_blobs(st, nblobs, nx, ny, nz, sigma=sigma)
    psi = gaussian_sum(shape, tuple(bool(p) for p in periodic), background, blobs)
    u1, u2, u3 = rotation_courant(nx, ny, nz, max_c)
    return Fields("near_zero_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, tuple(periodic),
                  sine_density(nx, ny, nz), _f32(psi), u1, u2, u3, nsteps, seed)


def truncated_blobs(nx, ny, nz, cutoff=1e-3, nblobs=4, sigma=(2.0, 6.0), max_c=0.5,
                    nsteps=10, seed=1514, periodic=(1, 1, 0)) -> Fields:
    """Exact zeros: the blobs of near_zero_blobs on background 0 with every
    value below `cutoff` set to exactly 0, so that most of the grid is zero
    and every blob ends in a jump of about `cutoff`."""
    f = near_zero_blobs(nx, ny, nz, background=0.0, nblobs=nblobs, sigma=sigma, max_c=max_c,
                        nsteps=nsteps, seed=seed, periodic=periodic)
    psi = np.where(f.psi.astype(np.float64) < cutoff, 0.0, f.psi.astype(np.float64))
    return dataclasses.replace(f, name="truncated_%dx%dx%d" % (nx, ny, nz), psi=_f32(psi))


def subsample(f: Fields, every=8, max_c=0.5) -> Fields:
    """A copy of f every `every`-th cell in x and y (psi and h sampled from
    f's initial fields, all of z kept) with the rotation field regenerated
    at the smaller size and the same max |C|."""
    psi = np.ascontiguousarray(f.psi[:, ::every, ::every])
    h = np.ascontiguousarray(f.h[:, ::every, ::every])
    nz, ny, nx = psi.shape
    u1, u2, u3 = rotation_courant(nx, ny, nz, max_c)
    return Fields("%s_every%d" % (f.name, every), nx, ny, nz, f.periodic, h, psi, u1, u2, u3,
                  f.nsteps, f.seed)
