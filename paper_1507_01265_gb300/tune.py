"""Speed-function autotuner for the batched launch (§5.4, §4).

The paper builds speed functions of its core teams by timing every team at
once on equal workloads (so contention is included, §5.4), then feeds them
to Algorithm 1 to pick a possibly uneven partition.  The GPU analogue here:

  * a "processor" is one persistent CTA (one per SM) and its workload x is
    the number of tiles it marches;
  * s(x) is measured with all CTAs busy: a synthetic grid of exactly P*x
    tiles (P = number of SMs), so the balanced split gives every CTA x tiles;
    s(x) = x * (tile cells) / (time of one step), cells per second per CTA;
  * for a workload of n tiles the partitioner (mpdata_fpm_partition) returns
    k CTAs with x_right tiles and P - k with x_left, or the balanced split;
  * the speed functions of the available tile shapes are compared and the
    shape with the shortest predicted step is chosen;
  * `tune_grid` also times the library's default split, one CTA per tile
    handed out by the hardware (largest first), against the balanced and
    the partitioner's persistent splits;
  * in a batch of uneven grids each grid may get its own shape
    (`choose_tiles`): a tile of shape ty costs 32*ty*(nz+3) cell-planes over
    the per-SM rate of that shape (measured whole-GPU rate / P); the tiles
    of one shape form one launch of one CTA per tile, whose time is that of
    handing the tiles out largest first to the SM that frees first, plus a
    launch.  Starting from the best of the uniform choices and the per-grid
    cheapest shapes, grids switch shape while the predicted batch time
    drops.

  * `tile_times` measures the step time of single-grid launches per tile
    shape (the data behind the library's default-tile model: waves of tiles
    x per-plane time of one CTA).

Usage:  python -m paper_1507_01265_gb300.tune --grid 1024 512 64
        python -m paper_1507_01265_gb300.tune --tile-probe 40
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import Batch, fpm

def _device_fields(nx, ny, nz, seed=11, periodic=(1, 1, 0)):
    import torch
    import gen.fields as F
    f = F.rotation_blobs(nx=nx, ny=ny, nz=nz, nblobs=2, seed=seed, periodic=periodic)
    return f, [torch.from_numpy(a).cuda() for a in (f.h, f.psi, f.u1, f.u2, f.u3)]


def _time_batch(b, steps, warmup=2):
    import torch
    for _ in range(warmup):
        b.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / steps


def num_sms():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def speed_function(tile=(32, 24), xs=(1, 2, 3, 4, 5, 6, 7, 8), nz=64, steps=6):
    """Measured s(x) in cells/s per CTA for x tiles per CTA, all SMs busy."""
    P = num_sms()
    tx, ty = tile
    speeds = []
    for x in xs:
        nx, ny = tx * P, ty * x  # P*x tiles: every CTA of the balanced split gets x
        f, t = _device_fields(nx, ny, nz)
        with Batch([(nx, ny, nz, (1, 1, 0))], tile=tile) as b:
            b.set_fields(0, *t)
            b.set_balanced_split(b.grid_variant(0), P)  # P persistent CTAs, x tiles each
            n, ncta = b.work(b.grid_variant(0))
            assert n == P * x and ncta == P
            dt = _time_batch(b, steps)
        speeds.append(x * tx * ty * nz / dt)
        del t
    return np.array(xs, dtype=float), np.array(speeds)


def split_for(n_items, ncta, k, xl, xr):
    """begin[] of a split where the first k CTAs take xr items, the rest xl."""
    sizes = [int(round(xr))] * k + [int(round(xl))] * (ncta - k)
    if sum(sizes) != n_items:
        raise ValueError("split does not cover the work list")
    return list(np.concatenate([[0], np.cumsum(sizes)]).astype(int))


def list_time(costs, nsm):
    """Time of one launch of one CTA per item: items handed out largest
    first, each to the SM that frees first."""
    import heapq
    if not costs:
        return 0.0
    free = [0.0] * min(nsm, len(costs))
    for c in sorted(costs, reverse=True):
        heapq.heapreplace(free, free[0] + c)
    return max(free)


def batch_time(dims, tiles, rates, nsm, launch_s=50e-6, tx=32):
    """Predicted time of one batched step: one launch per tile shape in use
    (the library's default split, one CTA per tile), a tile of shape ty
    costing tx*ty*(nz+3) cell-planes at rates[ty] / nsm per SM, plus
    launch_s per launch (a launch's fill and drain: a second shape's launch
    measured about 60 us per step on the tracer batch)."""
    items = {}
    for (nx, ny, nz), ty in zip(dims, tiles):
        tile_s = tx * ty * (nz + 3) / (rates[ty] / nsm)
        items.setdefault(ty, []).extend([tile_s] * (math.ceil(nx / tx) * math.ceil(ny / ty)))
    return sum(list_time(c, nsm) + launch_s for c in items.values())


def choose_tiles(dims, rates, nsm, launch_s=50e-6):
    """Per-grid tile heights (keys of `rates`, e.g. {24: r24, 16: r16}) for
    the grids dims = [(nx, ny, nz), ...]: the best of the uniform choices and
    of every grid taking its own cheapest shape, then single-grid switches
    (largest predicted gain first) while the predicted batch time drops."""
    shapes = list(rates)

    def own_cost(nx, ny, nz, ty):
        return math.ceil(nx / 32) * math.ceil(ny / ty) * 32 * ty * (nz + 3) / rates[ty]

    starts = [[ty] * len(dims) for ty in shapes]
    starts.append([min(shapes, key=lambda ty: own_cost(nx, ny, nz, ty)) for nx, ny, nz in dims])
    best = min(starts, key=lambda t: batch_time(dims, t, rates, nsm, launch_s))
    t_best = batch_time(dims, best, rates, nsm, launch_s)
    improved = True
    while improved:
        improved = False
        cands = []
        for i in range(len(dims)):
            for ty in shapes:
                if ty != best[i]:
                    trial = best[:i] + [ty] + best[i + 1:]
                    cands.append((batch_time(dims, trial, rates, nsm, launch_s), i, ty))
        if cands:
            t, i, ty = min(cands)
            if t < t_best * (1 - 1e-9):
                best[i], t_best, improved = ty, t, True
    return best


def tune_grid(nx, ny, nz, periodic=(1, 1, 0), steps=10, tiles=((32, 28), (32, 24), (32, 16)), xs_max=10):
    """Speed functions per tile shape, the partitioner's choice, and measured
    step times of the balanced and the chosen split on this grid."""
    P = num_sms()
    report = {"grid": [nx, ny, nz], "sms": P, "shapes": {}}
    f, t = _device_fields(nx, ny, nz, periodic=periodic)
    best = None
    for tile in tiles:
        tx, ty = tile
        ntiles = math.ceil(nx / tx) * math.ceil(ny / ty)
        xs, ss = speed_function(tile, xs=tuple(range(1, xs_max + 1)), nz=nz)
        cond2, x_at, x_more = fpm.condition2(xs, ss)
        k, xl, xr, t_pred = fpm.partition(ntiles, P, 1.0, xs, ss / (tx * ty * nz))
        with Batch([(nx, ny, nz, periodic)], tile=tile) as b:
            b.set_fields(0, *t)
            variant = b.grid_variant(0)
            t_tile = _time_batch(b, steps)  # default: one CTA per tile
            b.set_balanced_split(variant, P)
            n, ncta = b.work(variant)
            t_bal = _time_batch(b, steps)
            chosen = b.get_split(variant)
            if k > 0:
                chosen = split_for(n, ncta, k, xl, xr)
                b.set_split(variant, chosen)
            t_tuned = _time_batch(b, steps)
        rec = {"tiles": ntiles, "speed_x": xs.tolist(), "speed_cells_per_s": ss.tolist(),
               "condition2": bool(cond2), "condition2_sizes": [x_at, x_more],
               "k_right": k, "x_left": xl, "x_right": xr, "predicted_step_s": t_pred,
               "balanced_step_s": t_bal, "tuned_step_s": t_tuned, "per_tile_step_s": t_tile,
               "gcell_steps_per_s_per_tile": nx * ny * nz / t_tile / 1e9,
               "gcell_steps_per_s_balanced": nx * ny * nz / t_bal / 1e9,
               "gcell_steps_per_s_tuned": nx * ny * nz / t_tuned / 1e9}
        report["shapes"]["%dx%d" % tile] = rec
        if best is None or t_pred < best[1]:
            best = (tile, t_pred)
    report["chosen_tile"] = list(best[0])
    return report


PROBE_TILES = ((32, 28), (32, 24), (32, 16), (32, 12), (24, 24), (24, 16), (16, 16))


def probe_grids(count=40, seed=1511):
    """Grid sizes of the serving workload's request templates: nx, ny, nz
    log-uniform in [32, 512] x [32, 256] x [32, 64] (drawn as in bench.py)."""
    import gen.fields as F
    st = F.Stream(seed)
    out = []
    for _ in range(count):
        nx = st.log_uniform_int(32, 512)
        ny = st.log_uniform_int(32, 256)
        nz = st.log_uniform_int(32, 64)
        st.scalar(0.1, 0.5)
        out.append((nx, ny, nz))
    return out


def tile_times(grids, tiles=PROBE_TILES, steps=20):
    """Microseconds per step of one mpdata_step launch per tile shape, for
    each (nx, ny, nz) (x/y periodic, lid z), plus the default tile the
    library picks."""
    import torch
    from . import Solver
    rows = []
    for nx, ny, nz in grids:
        f, t = _device_fields(nx, ny, nz)
        us = {}
        for tile in tiles:
            with Solver(nx, ny, nz, periodic=(1, 1, 0), tile=tile) as s:
                p = t[1].clone()
                s.step(t[0], p, t[2], t[3], t[4], 2)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.step(t[0], p, t[2], t[3], t[4], steps)
                e1.record()
                torch.cuda.synchronize()
                us["%dx%d" % tile] = e0.elapsed_time(e1) / steps * 1e3
        with Solver(nx, ny, nz, periodic=(1, 1, 0)) as s:
            default = "%dx%d" % s.tile
        rows.append({"grid": [nx, ny, nz], "us": us, "best": min(us, key=us.get), "default": default})
        del t
    return rows


def per_plane_medians(rows, nsm):
    """The default-tile model's table: per tile shape, the median of step
    time / (nz + 6) over the grids that need at most one tile per SM, for
    nx % 4 == 0 and for other nx."""
    import statistics
    out = {}
    for tile in rows[0]["us"]:
        tx, ty = (int(v) for v in tile.split("x"))
        for aligned in (True, False):
            v = [r["us"][tile] / (r["grid"][2] + 6) for r in rows
                 if (r["grid"][0] % 4 == 0) == aligned
                 and math.ceil(r["grid"][0] / tx) * math.ceil(r["grid"][1] / ty) <= nsm]
            if v:
                out["%s %s" % (tile, "nx%4==0" if aligned else "other nx")] = statistics.median(v)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[1024, 512, 64])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--xs-max", type=int, default=8)
    ap.add_argument("--tile-probe", type=int, default=0, metavar="N",
                    help="time every tile shape on N serving-size grids instead")
    a = ap.parse_args()
    if a.tile_probe:
        rows = tile_times(probe_grids(a.tile_probe))
        for r in rows:
            print(json.dumps(r))
        best = sum(min(r["us"].values()) for r in rows)
        dflt = sum(r["us"][r["default"]] for r in rows)
        print(json.dumps({"sum_us_best": best, "sum_us_default": dflt,
                          "sum_us_by_tile": {k: sum(r["us"][k] for r in rows) for k in rows[0]["us"]},
                          "per_plane_us": per_plane_medians(rows, num_sms())}))
        return
    rep = tune_grid(*a.grid, steps=a.steps, xs_max=a.xs_max)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
