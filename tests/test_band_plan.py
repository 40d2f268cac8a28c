"""The row-band planner (host logic, no GPU): its choices equal a plain
restatement of its model -- tiles handed out largest first, each to the SM
that frees first -- and it only takes plans that the model says pay."""
import math

import pytest

T28, T24 = 1.91, 1.67  # us per plane of one CTA: 32x28 and 32x24, two-column with loader warps


def handout(costs, nsm):
    """Finish time of the tiles handed out largest first to the least-loaded SM."""
    import heapq
    free = [0.0] * nsm
    for c in sorted(costs, reverse=True):
        heapq.heapreplace(free, free[0] + c)
    return max(free)


def model(nx, ny, nsm):
    ntx = (nx + 31) // 32
    w24 = math.ceil(ntx * math.ceil(ny / 24) / nsm)
    w28 = math.ceil(ntx * math.ceil(ny / 28) / nsm)
    single = min(w24 * T24, w28 * T28)
    if min(w24, w28) > 48:
        return (0, 0)
    best = None
    for n28 in range(1, ny):
        if 28 * n28 >= ny:
            break
        n24 = math.ceil((ny - 28 * n28) / 24)
        t = handout([T28] * (ntx * n28) + [T24] * (ntx * n24), nsm) + 0.02 * T28
        if best is None or t < best[0]:
            best = (t, n28, n24)
    return (best[1], best[2]) if best and best[0] < 0.99 * single else (0, 0)


@pytest.fixture(scope="module")
def mp():
    import paper_1507_01265_gb300 as mp
    return mp


def test_known_plans(mp):
    assert mp.plan_bands(1024, 512, 64) == (14, 5)      # 14*28 + 5*24 = 512 rows, 608 tiles
    assert mp.plan_bands(2048, 1024, 64) == (28, 10)
    assert mp.plan_bands(4096, 2048, 32) == (0, 0)      # below the 1 % bar
    assert mp.plan_bands(512, 512, 64) == (0, 0)        # two waves of 32x28 tiles already fit
    assert mp.plan_bands(1024, 512, 64, (0, 1, 0)) == (14, 5)  # lids on x or y band the same way
    assert mp.plan_bands(1026, 512, 64) == (0, 0)       # nx % 4 != 0
    assert mp.plan_bands(1024, 512, 64, nsm=0) == (0, 0)
    assert mp.plan_bands(1024, 65535, 8) == (0, 0)      # beyond 48 waves


@pytest.mark.parametrize("nsm", [152, 132, 8])
def test_plans_follow_the_model(mp, nsm):
    grids = [(1024, 512), (2048, 1024), (1024, 1024), (768, 512), (640, 640), (1536, 512),
             (2048, 2048), (256, 1024), (96, 300), (4096, 512), (512, 100), (1024, 60)]
    for nx, ny in grids:
        got = mp.plan_bands(nx, ny, 16, nsm=nsm)
        assert got == model(nx, ny, nsm), (nx, ny, nsm)
        if got != (0, 0):
            n28, n24 = got
            assert n28 >= 1 and n24 >= 1
            assert ny <= 28 * n28 + 24 * n24 < ny + 24   # rows covered, the last band not wasted


def test_planner_is_fast(mp):
    import time
    t0 = time.perf_counter()
    for ny in (65535, 40000, 9999):
        mp.plan_bands(32, ny, 8)
        mp.plan_bands(4096, ny // 8, 8)
    assert time.perf_counter() - t0 < 1.0


def test_bad_arguments(mp):
    with pytest.raises(mp.MpdataError):
        mp.plan_bands(0, 512, 64)
    with pytest.raises(mp.MpdataError):
        mp.plan_bands(1024, 512, 64, nsm=-1)
