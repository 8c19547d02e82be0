"""The FP64 oracle against its pins (hand-derived fixtures, closed forms,
invariants, brute force).  CPU only."""

import pytest

import oracle.gsvd_music as O
from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(O)
