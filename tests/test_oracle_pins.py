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
