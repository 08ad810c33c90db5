"""The FP64 oracle against its pins (no GPU)."""
import pytest

import oracle_pins as P
from oracle import Oracle


def _make(ix, dim):
    return Oracle(ix, dim=dim)


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, oracle_lib):
    pin(_make)
