"""Plant each mistake of tests/mutants.py in a copy of the oracle and check
that the pins notice it.  This is the evidence that the pins constrain every
part of the step (a pin suite that passes any oracle would prove nothing)."""
import os

import pytest

import mutants
import pins
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpdata_oracle.c")


def _small_conv2d(lib):
    pins.pin_convergence_2d(lib, sizes=(16, 32), threshold=1.3)


_small_conv2d.__name__ = "pin_convergence_2d_small"

ORDERED = pins.FAST_PINS + [_small_conv2d, pins.pin_convergence_1d]


def test_small_conv2d_passes_on_oracle(oracle_lib):
    _small_conv2d(oracle_lib)


@pytest.mark.parametrize("name,old,new", mutants.MUTANTS, ids=[m[0] for m in mutants.MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    path = tmp_path / ("mut_%s.c" % name)
    path.write_text(src.replace(old, new))
    lib = O.load(O.build(force=True, src=str(path), out=str(tmp_path / ("mut_%s.so" % name))))
    for pin in ORDERED:
        try:
            pin(lib)
        except AssertionError:
            return  # caught
    pytest.fail("no pin caught the planted mistake " + name)
