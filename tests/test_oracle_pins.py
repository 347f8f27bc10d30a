"""The CPU oracle checked against mathematics and independent libraries
(Gram-Schmidt by brute force, Cholesky, LAPACK, closed forms, invariants)."""

import pytest

from tests import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)
