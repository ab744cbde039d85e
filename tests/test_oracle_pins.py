"""The CPU oracle against its pins (worked examples of the paper, brute force,
ground truth of the generator, invariants, Graham's LPT bound)."""
import pytest

import oracle
from tests import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.default())
