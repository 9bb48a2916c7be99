"""The CPU oracle against facts that do not come from itself (see tests/oracle_pins.py for what pins what)."""
import pytest

from tests import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(orc, check):
    check(orc)
