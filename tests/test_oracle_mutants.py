"""Every planted mistake in the oracle (a dropped 1/2, a flipped Pdot sign, an
inverted log ratio, a transposed marginal, round instead of floor, a wrong
magnitude scale, a wrong normaliser, a wrong epoch sign, a missing 1/P, one
normalisation for all filters, the mean for the median) must
make at least one pin fail.  The mistakes are compiled into separate copies of
the oracle on the CPU; the real oracle is untouched."""
import pytest

import oracle
import oracle_pins

MUTANTS = {
    1: "Pdot term without the 1/2",
    2: "Pdot term with the wrong sign",
    3: "log ratio inverted",
    4: "magnitude marginal used instead of the phase marginal",
    5: "phase bin rounded instead of floored",
    6: "magnitude range scaled by n_mag - 1",
    7: "probabilities normalised by n_phase instead of N",
    9: "epoch added instead of subtracted",
    10: "Pdot term missing one factor 1/P",
    11: "one set of filter statistics for the whole curve",
    12: "filter mean subtracted instead of its median",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda k: MUTANTS[k])
def test_mutant_is_caught(mutant):
    orc = oracle.Oracle(mutant)
    failed = []
    for pin in oracle_pins.ALL_PINS:
        failed += [name for name, ok, _ in pin(orc) if not ok]
        if failed:
            break
    assert failed, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
