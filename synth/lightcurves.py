"""Seeded survey-shaped light curves for the five benchmark workloads.

Workloads (sizes, cadences and signal families as the benchmark configurations
state them; every random draw comes from numpy's PCG64 with seed
20200611 + workload index, in the order: per-curve N, times, signal class and
parameters, noise):

  0 "plain"     1 curve x 100 times U(0, 365 d) sorted; 15 + 0.3 sin(2 pi t/P0)
                + N(0, 0.02), P0 = 20 min; 1000 periods linear in frequency over
                3-60 min; Pdot = 0; 15 phase x 10 mag bins.
  1 "batch"     1000 curves x 1000 obs, nightly cadence (3 yr, 240-night
                seasons, 1-3 visits per night in an 8-h window); detached
                eclipsing binary (two Gaussian dips, depth U(0.1, 1) mag, width
                U(0.02, 0.08) of phase, secondary at half depth), N(0, 0.02);
                P0 log-U(5 min, 1 d); 1e5 log-spaced periods over the same range;
                Pdot = 0; 15 x 10 bins.
  2 "pdot"      100 curves x 500 obs, 3-yr nightly cadence; chirping eclipses,
                P0 log-U(3, 15 min), Pdot = -10^U(-12, -10); 1e4 log-spaced
                periods on 3-15 min x 256 Pdot linear in [-1e-10, 0]; 15 x 10.
  3 "ragged"    10,000 curves, N = round(exp U(ln 50, ln 2000)); 3-yr nightly
                cadence (denser nights for the longest curves); 1/3 each sinusoid (amplitude U(0.05, 0.5)), eclipse,
                pure noise; sigma U(0.01, 0.1); P0 log-U(3 min, 1 d); 5e4
                log-spaced periods over 3 min-1 d; Pdot = 0; 15 x 10; top-5.
  4 "longbase"  1000 curves, N ~ U{200..1000}; 10-yr baseline, 240-night
                seasons, every third in-season night, second same-night visits
                (15 min-2 h later) once N exceeds the ~800 nights; chirping
                eclipses, P0 log-U(3, 60 min), Pdot = -10^U(-13, -10); 1e5
                log-spaced periods on 3-60 min x 64 Pdot log-spaced
                -[1e-13, 1e-10]; 20 phase x 10 mag bins; top-5.

  5 "paper"     the production search of Sec. 3: 100 curves, 10-yr baseline
                with Gaussian spacing of mean 7 d (Sec. 2.2's VRO-like sampling,
                n ~ 520); chirping eclipses of a Burdge-like set (Sec. 2.1): P0
                U(4, 38) min, Pdot log-U over -[1.22e-12, 5.44e-11] (Sec. 3);
                5,183,995 periods linear in frequency (2/B .. 480 per day, step
                1/(3B), B = 3600 d) x 32 log-spaced Pdot in -[1e-12, 1e-10];
                15 x 10 bins; top-5.

Times are float64 seconds from the survey start (t0 = 0).  The paper's own
catalogs (Sec. 2.1) and its ellc light curves (Sec. 2.2) are not available;
these draws stand in for them with the shapes above.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

from .grids import DAY, linear_frequency_periods, log_periods

SEED_BASE = 20200611
CONFIG_NAMES = ("plain", "batch", "pdot", "ragged", "longbase", "paper")
YEAR_NIGHTS = 365
SEASON_NIGHTS = 240
NIGHT_WINDOW = 8 * 3600.0


@dataclasses.dataclass
class LightCurveBatch:
    """A ragged batch of light curves plus its trial grid.

    times, mags: float64[sum N]; offsets: int64[n_curves + 1] (curve c owns
    [offsets[c], offsets[c+1])); periods: float64[n_P]; pdots: float64[n_Pd].
    truth: per-curve injected parameters (P0, Pdot, class code: 0 sinusoid,
    1 eclipse, 2 pure noise)."""
    name: str
    times: np.ndarray
    mags: np.ndarray
    offsets: np.ndarray
    periods: np.ndarray
    pdots: np.ndarray
    n_phase: int
    n_mag: int
    truth_p0: np.ndarray
    truth_pdot: np.ndarray
    truth_class: np.ndarray
    t0: float = 0.0
    topk: int = 0

    @property
    def n_curves(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_obs(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def point_trials(self) -> int:
        return int(self.offsets[-1]) * int(self.periods.shape[0]) * int(self.pdots.shape[0])

    def curve(self, c: int):
        lo, hi = int(self.offsets[c]), int(self.offsets[c + 1])
        return self.times[lo:hi], self.mags[lo:hi]

    def subset(self, curves, periods=None, pdots=None) -> "LightCurveBatch":
        """A batch made of the listed curves (and optionally a sub-grid)."""
        curves = np.asarray(curves, dtype=np.int64)
        parts_t, parts_m, offs = [], [], [0]
        for c in curves:
            t, m = self.curve(int(c))
            parts_t.append(t)
            parts_m.append(m)
            offs.append(offs[-1] + t.shape[0])
        return LightCurveBatch(
            name=self.name + "-subset",
            times=np.concatenate(parts_t) if parts_t else np.zeros(0),
            mags=np.concatenate(parts_m) if parts_m else np.zeros(0),
            offsets=np.asarray(offs, dtype=np.int64),
            periods=self.periods if periods is None else np.asarray(periods, dtype=np.float64),
            pdots=self.pdots if pdots is None else np.asarray(pdots, dtype=np.float64),
            n_phase=self.n_phase, n_mag=self.n_mag,
            truth_p0=self.truth_p0[curves], truth_pdot=self.truth_pdot[curves],
            truth_class=self.truth_class[curves], t0=self.t0, topk=self.topk)

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.times, self.mags, self.offsets, self.periods, self.pdots):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


# ------------------------------------------------------------------ cadences

def uniform_cadence(rng, n: int, span: float) -> np.ndarray:
    """n times uniform on [0, span), sorted."""
    return np.sort(rng.uniform(0.0, span, size=n))


def _season_nights(years: float, every: int) -> np.ndarray:
    """Observed nights (days since the survey start): the first 240 nights of
    every 365, every `every`-th one, within the baseline."""
    n_years = int(np.ceil(years))
    d = np.arange(0, SEASON_NIGHTS, every, dtype=np.float64)
    nights = (np.arange(n_years, dtype=np.float64)[:, None] * YEAR_NIGHTS + d[None, :]).ravel()
    return nights[nights < years * YEAR_NIGHTS]


def _night_slots(rng, years: float, every: int, visits_lo: int, visits_hi: int):
    """Candidate visit times: visits_lo..visits_hi visits per observed night at
    uniform times inside an 8-hour window."""
    nights = _season_nights(years, every)
    n_visits = rng.integers(visits_lo, visits_hi + 1, size=nights.shape[0])
    base = np.repeat(nights * DAY, n_visits)
    return base + rng.uniform(0.0, NIGHT_WINDOW, size=base.shape[0])


def nightly_cadence(rng, n: int, years: float = 3.0) -> np.ndarray:
    """ZTF-like nightly cadence: n visits drawn without replacement from the
    season/night/visit slots, sorted.  Nights get 1-3 visits; a curve denser than
    that allows (n above about 1.25x the expected slot count) gets a higher
    per-night cap, the smallest that leaves that margin."""
    n_nights = _season_nights(years, 1).shape[0]
    hi = 3
    while 0.5 * (1 + hi) * n_nights < 1.25 * n:
        hi += 1
    while True:
        slots = _night_slots(rng, years, 1, 1, hi)
        if slots.shape[0] >= n:
            return np.sort(rng.choice(slots, size=n, replace=False))
        hi += 1


def sparse_cadence(rng, n: int, years: float = 10.0, every: int = 3) -> np.ndarray:
    """VRO-like sparse cadence over a long baseline: one visit on every third
    in-season night (about 800 nights in 10 years); when n exceeds the number of
    nights, second same-night visits 15 min to 2 h after the first are added."""
    nights = _season_nights(years, every)
    first = nights * DAY + rng.uniform(0.0, NIGHT_WINDOW - 2 * 3600.0, size=nights.shape[0])
    second = first + rng.uniform(15 * 60.0, 2 * 3600.0, size=nights.shape[0])
    if n <= nights.shape[0]:
        pick = rng.choice(nights.shape[0], size=n, replace=False)
        return np.sort(first[pick])
    extra = rng.choice(nights.shape[0], size=n - nights.shape[0], replace=False)
    return np.sort(np.concatenate([first, second[extra]]))


# ------------------------------------------------------------------ signals

def chirp_cycles(tau, p0: float, pdot: float) -> np.ndarray:
    """Cycles elapsed since tau = 0 for P(t) = P0 + Pdot t (Eq. 2): the exact
    integral of dt / P(t)."""
    tau = np.asarray(tau, dtype=np.float64)
    if pdot == 0.0:
        return tau / p0
    return np.log1p(pdot * tau / p0) / pdot


def _wrapped_distance(x):
    d = np.mod(x, 1.0)
    return np.minimum(d, 1.0 - d)


def eclipse_signal(cycles, depth: float, width: float, phase0: float) -> np.ndarray:
    """Detached eclipsing binary: primary Gaussian dip of the given depth (mag)
    and width (phase sigma) at phase0, secondary dip of half that depth half a
    cycle later (the secondary-to-primary surface-brightness ratio 0.5 of
    Sec. 2.2).  Fainter means a larger magnitude."""
    d1 = _wrapped_distance(cycles - phase0)
    d2 = _wrapped_distance(cycles - phase0 - 0.5)
    g1 = np.exp(-0.5 * (d1 / width) ** 2)
    g2 = np.exp(-0.5 * (d2 / width) ** 2)
    return depth * g1 + 0.5 * depth * g2


def sinusoid_signal(cycles, amp: float, phase0: float) -> np.ndarray:
    return amp * np.sin(2.0 * np.pi * (cycles - phase0))


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


# ------------------------------------------------------------------ workloads

def _assemble(name, times_list, mags_list, periods, pdots, n_phase, n_mag, p0, pdot, cls,
              topk=0):
    offsets = np.zeros(len(times_list) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([t.shape[0] for t in times_list])
    return LightCurveBatch(
        name=name, times=np.concatenate(times_list).astype(np.float64),
        mags=np.concatenate(mags_list).astype(np.float64), offsets=offsets,
        periods=np.asarray(periods, dtype=np.float64), pdots=np.asarray(pdots, dtype=np.float64),
        n_phase=n_phase, n_mag=n_mag, truth_p0=np.asarray(p0, dtype=np.float64),
        truth_pdot=np.asarray(pdot, dtype=np.float64), truth_class=np.asarray(cls, dtype=np.int32),
        topk=topk)


def _make_plain(rng):
    p0 = 20 * 60.0
    t = uniform_cadence(rng, 100, 365 * DAY)
    m = 15.0 + 0.3 * np.sin(2 * np.pi * t / p0) + rng.normal(0.0, 0.02, size=t.shape[0])
    periods = linear_frequency_periods(3 * 60.0, 60 * 60.0, 1000)
    return _assemble("plain", [t], [m], periods, [0.0], 15, 10, [p0], [0.0], [0])


def _eclipse_curve(rng, t, p0, pdot, sigma):
    depth = rng.uniform(0.1, 1.0)
    width = rng.uniform(0.02, 0.08)
    phase0 = rng.uniform(0.0, 1.0)
    m = 15.0 + eclipse_signal(chirp_cycles(t, p0, pdot), depth, width, phase0)
    return m + rng.normal(0.0, sigma, size=t.shape[0])


def _make_batch(rng, n_curves=1000, n_obs=1000, n_periods=100_000):
    ns = np.full(n_curves, n_obs)
    ts = [nightly_cadence(rng, int(n)) for n in ns]
    p0 = _loguniform(rng, 300.0, 86400.0, size=n_curves)
    ms = [_eclipse_curve(rng, t, p, 0.0, 0.02) for t, p in zip(ts, p0)]
    periods = log_periods(300.0, 86400.0, n_periods)
    return _assemble("batch", ts, ms, periods, [0.0], 15, 10, p0, np.zeros(n_curves),
                     np.ones(n_curves), topk=5)


def _make_pdot(rng, n_curves=100, n_obs=500, n_periods=10_000, n_pdots=256):
    ns = np.full(n_curves, n_obs)
    ts = [nightly_cadence(rng, int(n)) for n in ns]
    p0 = _loguniform(rng, 180.0, 900.0, size=n_curves)
    pd = -10.0 ** rng.uniform(-12.0, -10.0, size=n_curves)
    ms = [_eclipse_curve(rng, t, p, d, 0.02) for t, p, d in zip(ts, p0, pd)]
    periods = log_periods(180.0, 900.0, n_periods)
    pdots = np.linspace(-1e-10, 0.0, n_pdots)
    return _assemble("pdot", ts, ms, periods, pdots, 15, 10, p0, pd, np.ones(n_curves), topk=5)


def _make_ragged(rng, n_curves=10_000, n_periods=50_000):
    ns = np.rint(np.exp(rng.uniform(np.log(50.0), np.log(2000.0), size=n_curves))).astype(np.int64)
    ts = [nightly_cadence(rng, int(n)) for n in ns]
    cls = rng.integers(0, 3, size=n_curves)
    p0 = _loguniform(rng, 180.0, 86400.0, size=n_curves)
    sig = rng.uniform(0.01, 0.1, size=n_curves)
    ms = []
    for t, c, p, s in zip(ts, cls, p0, sig):
        if c == 0:
            amp = rng.uniform(0.05, 0.5)
            m = 15.0 + sinusoid_signal(chirp_cycles(t, p, 0.0), amp, rng.uniform(0.0, 1.0))
            m = m + rng.normal(0.0, s, size=t.shape[0])
        elif c == 1:
            m = _eclipse_curve(rng, t, p, 0.0, s)
        else:
            m = 15.0 + rng.normal(0.0, s, size=t.shape[0])
        ms.append(m)
    periods = log_periods(180.0, 86400.0, n_periods)
    return _assemble("ragged", ts, ms, periods, [0.0], 15, 10, p0, np.zeros(n_curves), cls,
                     topk=5)


def _make_longbase(rng, n_curves=1000, n_periods=100_000, n_pdots=64):
    ns = rng.integers(200, 1001, size=n_curves)
    ts = [sparse_cadence(rng, int(n)) for n in ns]
    p0 = _loguniform(rng, 180.0, 3600.0, size=n_curves)
    pd = -10.0 ** rng.uniform(-13.0, -10.0, size=n_curves)
    ms = [_eclipse_curve(rng, t, p, d, 0.02) for t, p, d in zip(ts, p0, pd)]
    periods = log_periods(180.0, 3600.0, n_periods)
    pdots = -np.geomspace(1e-13, 1e-10, n_pdots)
    return _assemble("longbase", ts, ms, periods, pdots, 20, 10, p0, pd, np.ones(n_curves),
                     topk=5)


def gaussian_cadence(rng, years: float = 10.0, mean_days: float = 7.0, sd_days: float = 1.0):
    """Sec. 2.2: gaps between observations drawn from a Gaussian of mean mean_days
    (sd sd_days, truncated at 0.1 d), until the baseline is covered."""
    span = years * 365.25 * DAY
    gaps = np.maximum(rng.normal(mean_days, sd_days, int(span / (mean_days * DAY) * 1.2) + 10),
                      0.1) * DAY
    t = np.cumsum(gaps)
    return t[t < span] - 0.0


def _make_paper(rng, n_curves=100, n_pdots=32, periods=None):
    from .grids import paper_frequency_grid, paper_pdot_grid
    ts = [gaussian_cadence(rng) for _ in range(n_curves)]
    p0 = rng.uniform(4.0, 38.0, size=n_curves) * 60.0
    pd = -np.exp(rng.uniform(np.log(1.22e-12), np.log(5.44e-11), size=n_curves))
    ms = [_eclipse_curve(rng, t, p, d, 0.02) for t, p, d in zip(ts, p0, pd)]
    per = paper_frequency_grid() if periods is None else periods
    return _assemble("paper", ts, ms, per, paper_pdot_grid(n_pdots), 15, 10, p0, pd,
                     np.ones(n_curves), topk=5)


_MAKERS = (_make_plain, _make_batch, _make_pdot, _make_ragged, _make_longbase, _make_paper)


def make_config(index: int, **overrides) -> LightCurveBatch:
    """Workload `index` (0..5, see the module docstring), drawn with seed
    20200611 + index.  Keyword overrides shrink the workload (n_curves, n_obs,
    n_periods, n_pdots where the workload has them) for tests; the draw order
    is unchanged, so a shrunken workload is a prefix-consistent relative of the
    full one only in its seed, not its values."""
    rng = np.random.default_rng(SEED_BASE + int(index))
    return _MAKERS[int(index)](rng, **overrides)


def make_multiband(seed: int, n_curves: int = 40, n_obs: int = 600, n_bands: int = 2,
                   n_periods: int = 2000, pdots=(0.0,)):
    """Multi-filter light curves (the filter combination of Sec. 2.3): every visit of
    a 3-year nightly cadence is in one of n_bands filters, drawn uniformly.  Filter
    b of a curve shifts its magnitudes by a colour offset U(-0.5, 0.5) mag, scales
    the eclipse depth by U(0.6, 1.2) and has its own noise sigma U(0.01, 0.05).
    Eclipsing binaries with P0 log-U(300 s, 3000 s) over log-spaced periods
    300-3000 s.  Returns (batch, bands uint8[sum N])."""
    rng = np.random.default_rng(int(seed))
    ts, ms, bs, p0s = [], [], [], []
    for _ in range(n_curves):
        t = nightly_cadence(rng, n_obs)
        b = rng.integers(0, n_bands, size=t.shape[0])
        p0 = float(_loguniform(rng, 300.0, 3000.0))
        depth, width, phase0 = rng.uniform(0.2, 1.0), rng.uniform(0.02, 0.06), rng.uniform(0, 1)
        colour = rng.uniform(-0.5, 0.5, size=n_bands)
        gain = rng.uniform(0.6, 1.2, size=n_bands)
        sigma = rng.uniform(0.01, 0.05, size=n_bands)
        base = eclipse_signal(chirp_cycles(t, p0, 0.0), depth, width, phase0)
        m = 15.0 + colour[b] + gain[b] * base + rng.normal(0.0, 1.0, size=t.shape[0]) * sigma[b]
        ts.append(t)
        ms.append(m)
        bs.append(b.astype(np.uint8))
        p0s.append(p0)
    batch = _assemble("multiband", ts, ms, log_periods(300.0, 3000.0, n_periods), list(pdots),
                      15, 10, np.array(p0s), np.zeros(n_curves), np.ones(n_curves), topk=5)
    return batch, np.concatenate(bs)


def make_onegrid_injection(seed: int, n_curves: int, n_obs: int, periods, pdots,
                           kind: str = "eclipse", years: float = 3.0, noise: float = 0.0):
    """Noiseless (or lightly noisy) signals whose (P0, Pdot) sit exactly on the given
    grid: curve c takes periods[pi[c]] and pdots[qi[c]] for random grid indices.
    Returns (batch, pi, qi)."""
    rng = np.random.default_rng(int(seed))
    periods = np.asarray(periods, dtype=np.float64)
    pdots = np.asarray(pdots, dtype=np.float64)
    pi = rng.integers(0, periods.shape[0], size=n_curves)
    qi = rng.integers(0, pdots.shape[0], size=n_curves)
    ts, ms = [], []
    for c in range(n_curves):
        t = nightly_cadence(rng, n_obs, years=years)
        cyc = chirp_cycles(t, periods[pi[c]], pdots[qi[c]])
        if kind == "eclipse":
            m = 15.0 + eclipse_signal(cyc, rng.uniform(0.3, 1.0), rng.uniform(0.03, 0.06),
                                      rng.uniform(0.0, 1.0))
        else:
            m = 15.0 + sinusoid_signal(cyc, rng.uniform(0.2, 0.5), rng.uniform(0.0, 1.0))
        if noise > 0:
            m = m + rng.normal(0.0, noise, size=t.shape[0])
        ts.append(t)
        ms.append(m)
    batch = _assemble("injection", ts, ms, periods, pdots, 15, 10, periods[pi], pdots[qi],
                      np.ones(n_curves))
    return batch, pi, qi
