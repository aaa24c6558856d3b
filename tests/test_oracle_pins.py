"""The CPU oracle against its pins (exact arithmetic, closed forms, invariants,
the paper's worked example).  CPU only."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(orc, pin):
    results = pin(orc)
    assert results
    failed = [(name, detail) for name, ok, detail in results if not ok]
    assert not failed, failed
