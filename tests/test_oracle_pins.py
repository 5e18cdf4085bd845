"""The FP64 oracle against its pins (CPU only)."""
import pytest

import pins
from oracle import ptycho_oracle as orc


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(orc)
