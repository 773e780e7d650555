"""The FP64 oracle against closed forms, published kernel values, numpy.pad,
torch's float64 interpolate, an exact-rational brute force and invariants."""
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=[p.__name__ for p in pins.ALL_PINS])
def test_pin(o, pin):
    pin(o)
