"""The FPM partitioner (Algorithm 1 of §4 and its generalisation) on the
paper's worked example (§5.4, Table 1) and against brute force."""
import itertools
import math

import numpy as np
import pytest

FRAME = 120 * 128  # cells per frame of a 120 x m x 128 sub-domain (§5.4)


@pytest.fixture(scope="module")
def fpm():
    import __graft_entry__ as g
    g.build()
    from paper_1507_01265_gb300 import fpm
    return fpm


def _worked_example_table():
    """Speeds (cells/s) at m = 108..132 frames, step 4.  s(112) and s(128) are
    the two values printed in §5.4; the others are set so that the times the
    table implies match the theoretical column of Table 1 for dm = 0, 4, 12
    (1.486 s, 1.470 s, 1.402 s: the larger workload x_right is the slower
    one), while the smaller workloads finish earlier."""
    m = np.array([108, 112, 116, 120, 124, 128, 132], dtype=float)
    t = {120: 1.486, 124: 1.470, 132: 1.402}
    s = {}
    for x, tt in t.items():
        s[x] = FRAME * x / tt  # cells per second giving time tt
    s[128] = 1418579.0
    s[112] = 1436742.0
    s[116] = FRAME * 116 / 1.30   # finishes before its x_right partner
    s[108] = FRAME * 108 / 1.15
    return m, np.array([s[int(x)] if int(x) in s else 0 for x in m])


def test_worked_example_time(fpm):
    # t = max(120*128*128/1418579, 120*112*128/1436742) = 1.386 s (§5.4)
    t = max(120 * 128 * 128 / 1418579, 120 * 112 * 128 / 1436742)
    assert round(t, 3) == 1.386


def test_algorithm1_reproduces_worked_example(fpm):
    m, s = _worked_example_table()
    speeds = s / FRAME  # frames per second; the unit does not matter (§4)
    xl, xr, t = fpm.algorithm1(480, 4, 4, m, speeds)
    assert (xl, xr) == (112, 128)
    assert round(t * 1.0, 3) == 1.386
    # scale invariance: a * s(x) gives the same split (§4)
    xl2, xr2, t2 = fpm.algorithm1(480, 4, 4, m, speeds * 1000.0)
    assert (xl2, xr2) == (xl, xr) and math.isclose(t2 * 1000.0, t)
    # the general form agrees for even p
    k, gl, gr, gt = fpm.partition(480, 4, 4, m, speeds)
    assert (k, gl, gr) == (2, 112, 128) and math.isclose(gt, t)


def _brute_force(n, p, dx, xs, ss, two_sizes):
    f = lambda x: x / np.interp(x, xs, ss)
    units = int(round(n / dx))
    best = math.inf
    lo, hi = xs[0], xs[-1]
    for parts in itertools.combinations_with_replacement(range(1, units + 1), p):
        if sum(parts) != units:
            continue
        sizes = [q * dx for q in parts]
        if min(sizes) < lo - 1e-9 or max(sizes) > hi + 1e-9:
            continue
        if two_sizes and len(set(sizes)) > 2:
            continue
        best = min(best, max(f(x) for x in sizes))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_partition_matches_brute_force_over_two_size_splits(fpm, seed):
    r = np.random.default_rng(seed)
    p = int(r.integers(2, 6))
    dx = 1.0
    n = float(p * int(r.integers(3, 7)))
    xs = np.arange(1.0, n + 1.0)
    ss = r.uniform(0.5, 2.0, size=xs.size) * xs ** r.uniform(0.2, 1.2)
    k, xl, xr, t = fpm.partition(n, p, dx, xs, ss)
    assert k * xr + (p - k) * xl == pytest.approx(n) or k == 0
    assert t == pytest.approx(_brute_force(n, p, dx, xs, ss, two_sizes=True), rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_theorem1_balanced_is_optimal_when_condition1_holds(fpm, seed):
    # s(x)/x non-increasing (condition (1)): e.g. s(x) = a x / (b + x)
    r = np.random.default_rng(seed)
    p = 4
    n = float(p * int(r.integers(2, 5)))
    xs = np.arange(1.0, n + 1.0)
    ss = r.uniform(1, 3) * xs / (r.uniform(0.5, 4) + xs)
    ok, _, _ = fpm.condition2(xs, ss)
    assert not ok
    k, xl, xr, t = fpm.partition(n, p, 1.0, xs, ss)
    assert k == 0 and xl == xr == n / p
    assert t == pytest.approx(_brute_force(n, p, 1.0, xs, ss, two_sizes=False), rel=1e-12)


def test_condition2_detects_a_profile_that_rewards_imbalance(fpm):
    xs = np.array([1.0, 2.0, 3.0, 4.0])
    ss = np.array([1.0, 1.0, 4.0, 4.0])  # 3 units run as fast as 1
    ok, x, x2 = fpm.condition2(xs, ss)
    assert ok and x < x2
    k, xl, xr, t = fpm.partition(8, 4, 1.0, xs, ss)  # balanced: 2 each, time 2
    assert t < 2.0 and k > 0


def test_bad_tables_are_rejected(fpm):
    from paper_1507_01265_gb300 import MpdataError
    with pytest.raises(MpdataError):
        fpm.algorithm1(480, 3, 4, [1.0, 2.0], [1.0, 1.0])  # odd p
    with pytest.raises(MpdataError):
        fpm.partition(10, 2, 1.0, [2.0, 1.0], [1.0, 1.0])   # sizes not increasing
    with pytest.raises(MpdataError):
        fpm.partition(10, 2, 1.0, [1.0, 2.0], [1.0, -1.0])  # negative speed


def test_tile_choice_model():
    """Per-grid tile heights: the better uniform choice unless a mix lowers
    the predicted batch time; a mix is chosen where each shape fits its own
    grids exactly and both launches fill the GPU."""
    import itertools
    from paper_1507_01265_gb300 import tune
    rates = {24: 1e10, 16: 1e10}
    # ny = 72 fits 32x24 exactly (3 rows; 32x16 needs 5 = 80 rows), ny = 32 fits
    # 32x16 exactly (2 rows; 32x24 needs 2 = 48 rows)
    dims = [(1024, 72, 64)] * 20 + [(1024, 32, 64)] * 20
    t = tune.choose_tiles(dims, rates, nsm=152)
    got = tune.batch_time(dims, t, rates, 152)
    clean = tune.batch_time(dims, [24] * 20 + [16] * 20, rates, 152)
    assert got <= clean < min(tune.batch_time(dims, [ty] * 40, rates, 152) for ty in (24, 16))
    assert sum(ty == 16 for ty in t[20:]) > 10 and sum(ty == 24 for ty in t[:20]) > 10
    # a few small grids: a second launch would not fill the GPU, stay uniform
    small = [(64, 40, 16), (64, 32, 16), (96, 16, 20)]
    t = tune.choose_tiles(small, rates, nsm=152)
    assert len(set(t)) == 1
    # never worse than brute force by more than the greedy's step, never worse than uniform
    dims = [(256, 40, 32), (128, 56, 16), (512, 16, 64), (64, 88, 24), (320, 72, 48)]
    t = tune.choose_tiles(dims, {24: 1.1e10, 16: 0.9e10}, nsm=8)
    got = tune.batch_time(dims, t, {24: 1.1e10, 16: 0.9e10}, 8)
    brute = min(tune.batch_time(dims, list(a), {24: 1.1e10, 16: 0.9e10}, 8)
                for a in itertools.product((24, 16), repeat=len(dims)))
    assert brute <= got <= min(tune.batch_time(dims, [ty] * 5, {24: 1.1e10, 16: 0.9e10}, 8) for ty in (24, 16))
    assert got <= brute * 1.05
