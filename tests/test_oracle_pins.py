"""The CPU oracle against its pins (no GPU)."""
import pytest

import oracle
from tests import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    oracle.use_library(None)
    pin(oracle)
