"""The FP64 oracle against facts the MPDATA scheme fixes (see tests/pins.py).

These run on the CPU only; the oracle is the reference the CUDA path is
checked against, so it is pinned to the mathematics first."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.FAST_PINS, ids=lambda p: p.__name__)
def test_pin(oracle_lib, pin):
    pin(oracle_lib)


def test_convergence_1d(oracle_lib):
    pins.pin_convergence_1d(oracle_lib)


def test_convergence_2d_cross_terms(oracle_lib):
    pins.pin_convergence_2d(oracle_lib)


def test_mass_compensated_sum(oracle_lib):
    import numpy as np
    import oracle
    # 1 + many tiny terms: a naive running sum loses them, the compensated one does not
    h = np.ones(1 + 100000)
    psi = np.full(h.size, 1e-17)
    psi[0] = 1.0
    assert oracle.mass(h, psi) == pytest.approx(1.0 + 1e-12, rel=0, abs=1e-27)


def test_openmp_build_matches_serial(oracle_lib):
    """The all-core build of the oracle computes every cell with the serial
    expression, so it must return identical bits."""
    import numpy as np
    from oracle import oracle as O
    try:
        omp = O.load(omp=True)
    except Exception as e:  # noqa: BLE001
        pytest.skip("no OpenMP build: %s" % e)
    h, psi, u = pins._spiky_problem(30, (9, 10, 11), 0.15, 2)
    for iterations, extrema in ((2, 0), (3, 1)):
        cfg = O.Config(11, 10, 9, (1, 1, 0), iterations, 1, 1e-15, extrema)
        a = O.run(cfg, h, psi, *u, nsteps=3, lib=oracle_lib)
        b = O.run(cfg, h, psi, *u, nsteps=3, lib=omp)
        assert np.array_equal(a, b)
    assert O.threads(omp) >= 1 and O.threads(oracle_lib) == 1
