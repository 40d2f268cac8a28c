"""The default-tile model (host logic, no GPU): mpdata_default_tile equals a
plain restatement of its rule -- waves of tiles times the per-plane time of
a wave, the one-wave time while the tiles do not outnumber the SMs, 32x28
first and a later candidate taken only when 2 % faster -- and the choices
the measurements behind the table call for."""
import math

import pytest

# (tx, ty, CTAs per SM, us per plane per wave: nx % 4 == 0, other nx,
#  us per plane while tiles <= SMs: nx % 4 == 0, other nx)
TABLE = [
    (32, 28, 1, 1.91, 2.38, 1.91, 2.38),
    (32, 24, 1, 1.67, 1.91, 1.67, 1.91),
    (32, 16, 1, 1.39, 1.45, 1.39, 1.45),
    (32, 12, 2, 1.78, 2.25, 1.11, 1.76),
    (24, 16, 1, 1.76, 1.76, 1.76, 1.76),
    (16, 16, 1, 1.44, 1.45, 1.44, 1.45),
]


def model(nx, ny, nsm):
    sms = nsm if nsm > 0 else 1 << 28
    a16 = nx % 4 == 0
    best, pick = None, None
    for tx, ty, per_sm, ua, uo, u1a, u1o in TABLE:
        tiles = math.ceil(nx / tx) * math.ceil(ny / ty)
        if tiles <= sms:
            t = u1a if a16 else u1o
        else:
            t = math.ceil(tiles / (sms * per_sm)) * (ua if a16 else uo)
        if best is None or t < best * 0.98:
            best, pick = t, (tx, ty)
    return pick


@pytest.fixture(scope="module")
def mp():
    import paper_1507_01265_gb300 as mp
    return mp


def test_known_choices(mp):
    assert mp.default_tile(1024, 512, 64) == (32, 28)    # 608 tiles: four full waves
    assert mp.default_tile(4096, 2048, 32) == (32, 28)   # 63 waves of 1.91 vs 73 of 1.67
    assert mp.default_tile(40, 24, 12) == (32, 12)       # one wave, 32x12 alone on its SM
    assert mp.default_tile(42, 24, 12) == (32, 16)       # nx % 4 != 0: no loader warp
    assert mp.default_tile(512, 256, 64) == (32, 16)     # 256 tiles: two waves of 32x16
    assert mp.default_tile(64, 64, 8, dtype="f64") == (16, 16)
    assert mp.default_tile(1024, 512, 64, nsm=0) == (32, 12)  # unknown device: one wave


@pytest.mark.parametrize("nsm", [152, 132, 8, 0])
def test_choices_follow_the_model(mp, nsm):
    grids = [(1024, 512), (2048, 1024), (4096, 2048), (40, 24), (42, 24), (512, 256), (128, 128),
             (256, 128), (1022, 510), (33, 33), (1, 1), (600, 300), (200, 900), (96, 2000), (8192, 2)]
    for nx, ny in grids:
        assert mp.default_tile(nx, ny, 16, nsm=nsm) == model(nx, ny, nsm), (nx, ny, nsm)


def test_small_aligned_grids_take_the_two_cta_tile(mp):
    """Every grid with nx % 4 == 0 whose 32x12 tiles fit one per SM takes
    32x12 (1.11 us per plane, the fastest one-wave plane)."""
    for nx in range(4, 129, 4):
        for ny in (1, 12, 13, 60, 100):
            if math.ceil(nx / 32) * math.ceil(ny / 12) <= 152:
                assert mp.default_tile(nx, ny, 32) == (32, 12), (nx, ny)


def test_bad_arguments(mp):
    with pytest.raises(mp.MpdataError):
        mp.default_tile(0, 16, 16)
    with pytest.raises(mp.MpdataError):
        mp.default_tile(16, 16, 16, nsm=-1)
