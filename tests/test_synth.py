"""The seeded input generator: determinism, workload shapes, the paper's
production grid size, cadences and the injected phase law.  CPU only."""
import json
import os

import numpy as np
import pytest

import synth
from synth.grids import DAY

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_numbers.json")


def test_paper_production_grid_count():
    g = json.load(open(GOLDEN))["production_grid"]
    f = synth.paper_frequency_grid(as_periods_seconds=False)
    assert f.shape[0] == g["n_periods"]
    assert abs(f[-1] - g["f_max_per_day"]) < 1e-9
    assert abs(f[0] - 2.0 / 3600.0) < 1e-15
    assert np.allclose(np.diff(f), 1.0 / (3 * 3600.0))
    for n in g["pdot_sizes"]:
        pd = synth.paper_pdot_grid(n)
        assert pd.shape[0] == n and np.isclose(pd[0], -g["pdot_lo"]) and np.isclose(pd[-1], -g["pdot_hi"])


@pytest.mark.parametrize("k", [0, 1, 2, 4])
def test_workload_deterministic(k):
    a = synth.make_config(k)
    b = synth.make_config(k)
    assert a.digest() == b.digest()


def test_workload_shapes():
    expect = {0: (1, 100, 1000, 1, 15), 1: (1000, 1_000_000, 100_000, 1, 15),
              2: (100, 50_000, 10_000, 256, 15)}
    for k, (nc, npts, npd, nq, nphi) in expect.items():
        b = synth.make_config(k)
        assert (b.n_curves, int(b.offsets[-1]), b.periods.size, b.pdots.size, b.n_phase) == \
            (nc, npts, npd, nq, nphi)
        assert b.n_mag == 10
        assert np.all(np.diff(b.offsets) > 0)
    b = synth.make_config(4)
    assert b.n_curves == 1000 and b.n_obs.min() >= 200 and b.n_obs.max() <= 1000
    assert b.periods.size == 100_000 and b.pdots.size == 64 and b.n_phase == 20
    assert np.all(b.pdots < 0)


def test_ragged_lengths():
    b = synth.make_config(3)
    n = b.n_obs
    assert b.n_curves == 10_000 and n.min() >= 50 and n.max() <= 2000
    # log-uniform lengths: median near sqrt(50 * 2000) = 316
    assert 250 < np.median(n) < 400
    assert set(np.unique(b.truth_class)) == {0, 1, 2}


def test_nightly_cadence_respects_seasons():
    rng = np.random.default_rng(0)
    t = synth.nightly_cadence(rng, 1000)
    day = np.floor(t / DAY)
    assert np.all(day % 365 < 240)
    assert np.all(np.diff(t) >= 0)
    assert np.all(t - day * DAY < 8 * 3600.0)
    assert t.max() < 3 * 365 * DAY


def test_sparse_cadence_second_visits():
    rng = np.random.default_rng(1)
    t = synth.sparse_cadence(rng, 1000)
    day = np.floor(t / DAY)
    assert np.all(day % 365 < 240) and np.all((day % 365) % 3 == 0)
    assert t.max() < 10 * 365 * DAY
    # 200 nights carry a second visit 15 min - 2 h after the first
    _, counts = np.unique(day, return_counts=True)
    assert counts.max() == 2 and (counts == 2).sum() == 1000 - counts.size


def test_chirp_phase_law():
    """The injected phase is the exact integral of Eq. 2; Eq. 3's fold is its
    first-order expansion, off by Pdot^2 tau^3 / (3 P^3) cycles."""
    tau = np.linspace(0, 3.2e8, 1001)
    for p0, pdot in [(180.0, -1e-10), (420.0, -2.14e-11), (3600.0, 1e-12)]:
        exact = synth.lightcurves.chirp_cycles(tau, p0, pdot)
        first = tau / p0 - 0.5 * pdot * tau ** 2 / p0 ** 2
        bound = pdot ** 2 * tau ** 3 / (3 * p0 ** 3) * 1.01 + 1e-6
        assert np.all(np.abs(exact - first) <= bound)
    assert np.array_equal(synth.lightcurves.chirp_cycles(tau, 300.0, 0.0), tau / 300.0)


def test_paper_workload():
    """Workload 5: Sec. 3's production grid with Sec. 2.2's ~weekly 10-yr sampling."""
    b = synth.make_config(5, periods=np.array([600.0, 700.0]))
    assert b.n_curves == 100 and b.pdots.size == 32
    assert 480 < b.n_obs.mean() < 560 and b.times.max() < 10 * 365.25 * DAY
    assert np.all(b.truth_p0 >= 240) and np.all(b.truth_p0 <= 38 * 60)
    assert np.all(b.truth_pdot < 0)
    gaps = np.diff(b.curve(0)[0]) / DAY
    assert 6.5 < gaps.mean() < 7.5


def test_multiband_generator():
    """Multi-filter stand-in: one filter index per visit, each filter present, the
    same seed gives the same bytes, and the filters of a curve differ by their
    colour offsets (so normalising each filter on its own matters)."""
    b, bands = synth.make_multiband(5, n_curves=6, n_obs=400, n_bands=3)
    b2, bands2 = synth.make_multiband(5, n_curves=6, n_obs=400, n_bands=3)
    assert np.array_equal(b.times, b2.times) and np.array_equal(bands, bands2)
    assert bands.dtype == np.uint8 and bands.shape == b.times.shape and bands.max() < 3
    spread = []
    for c in range(b.n_curves):
        lo, hi = b.offsets[c], b.offsets[c + 1]
        assert hi - lo >= 300
        assert np.all(np.diff(b.times[lo:hi]) >= 0)
        meds = [np.median(b.mags[lo:hi][bands[lo:hi] == k]) for k in range(3)]
        spread.append(max(meds) - min(meds))
    assert np.median(spread) > 0.1
