"""The FP64 oracle against facts outside itself (closed forms, scipy, hand-worked cases)."""
import pytest

import oracle as O

from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_pin(pin):
    pin(O.load())
