"""Pins of the oracle's void volume fraction and void-opening flux modifier
(tests/pins_void.py holds the checks; CPU only)."""
import pytest

import pins_void as P


@pytest.mark.parametrize("name", list(P.CHECKS))
def test_pin(name):
    P.CHECKS[name](None)
