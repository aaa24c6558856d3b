"""Every planted mistake in the oracle (a dropped 1/2, a flipped Pdot sign, an
inverted log ratio, a transposed marginal, round instead of floor, a wrong
magnitude scale, a wrong normaliser, a wrong epoch sign, a missing 1/P, one
normalisation for all filters, the mean for the median, an overlapping bin
dropped or not wrapped around the phase circle, the edge distance in the
wrong unit, a sampled cell read from the wrong curve) must
make at least one pin fail.  The mistakes are compiled into separate copies of
the oracle on the CPU; the real oracle is untouched."""
import numpy as np
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
    13: "overlapping bins: the second bin of each point dropped",
    14: "overlapping bins: no wrap-around from the first phase bin to the last",
    15: "edge distance reported in phase bins instead of cycles",
    16: "sampled cells read from the previous curve's first point",
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


def _topk_larger_index_first(grid, k):
    flat = grid.reshape(grid.shape[0], -1)
    rev = flat[:, ::-1]
    idx = flat.shape[1] - 1 - np.argsort(rev, axis=1, kind="stable")[:, :k]
    return np.take_along_axis(flat, idx, axis=1), idx.astype(np.int64)


def _significance_sample_std(grid):
    flat = grid.reshape(grid.shape[0], -1)
    mu, sd = flat.mean(axis=1), flat.std(axis=1, ddof=1)
    return mu, sd, np.where(sd > 0, (mu - flat.min(axis=1)) / np.where(sd > 0, sd, 1.0), 0.0)


def _significance_max_for_min(grid):
    flat = grid.reshape(grid.shape[0], -1)
    mu, sd = flat.mean(axis=1), flat.std(axis=1)
    return mu, sd, np.where(sd > 0, (flat.max(axis=1) - mu) / np.where(sd > 0, sd, 1.0), 0.0)


PY_MUTANTS = {
    "top-k ties to the larger flat index": ("oracle_topk", _topk_larger_index_first),
    "Eq. 5 with the sample standard deviation": ("oracle_significance", _significance_sample_std),
    "Eq. 5 measured from the grid maximum": ("oracle_significance", _significance_max_for_min),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_is_caught(name, monkeypatch):
    """Planted mistakes in the oracle's Python selection step, swapped in for the
    duration of one test only."""
    attr, fn = PY_MUTANTS[name]
    monkeypatch.setattr(oracle, attr, fn)
    orc = oracle.Oracle()
    failed = [n for pin in (oracle_pins.pin_selection, oracle_pins.pin_significance)
              for n, ok, _ in pin(orc) if not ok]
    assert failed, f"{name} passed every pin"
