"""The CPU oracle against independent statements of the physics (see tests/pins.py)."""
import pytest

from pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_oracle_pin(pin, oracle_mod):
    pin(oracle_mod.simulate)
