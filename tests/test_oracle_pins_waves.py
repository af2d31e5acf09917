"""Pins of the oracle's HLLD shear-wave branch, reflective walls, 3D sweeps
and totals (tests/pins_waves.py holds the checks; CPU only)."""
import pytest

import pins_waves as P


@pytest.mark.parametrize("name", list(P.CHECKS))
def test_pin(name):
    P.CHECKS[name](None)
