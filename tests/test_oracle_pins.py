"""The FP64 oracle against closed forms, textbook values, scipy and brute force."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(0)
