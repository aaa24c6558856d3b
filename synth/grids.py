"""Trial grids over period P and period derivative Pdot.

Sec. 3 of arXiv:2006.06866 builds its production grid in frequency: from twice
the inverse baseline up to 1/(3 min) = 480 per day, in steps of 1/(3 B).  The
paper prints 5,183,995 trial periods for it; that count comes out exactly with
B = 3600 days and both end points included (the printed f_min = 5.47e-4 and
df = 9.13e-5 per day correspond to B = 3650 d instead, so the text is not
self-consistent; the count is the number this helper reproduces).  Its Pdot axis
is log-spaced from -1e-12 to -1e-10 with 32, 128 or 512 values.
"""
from __future__ import annotations

import numpy as np

DAY = 86400.0


def linear_frequency_periods(p_min: float, p_max: float, n: int) -> np.ndarray:
    """n periods whose frequencies are evenly spaced on [1/p_max, 1/p_min],
    both ends included; returned in increasing frequency (decreasing period)."""
    f = np.linspace(1.0 / p_max, 1.0 / p_min, int(n))
    return 1.0 / f


def log_periods(p_min: float, p_max: float, n: int) -> np.ndarray:
    """n log-spaced periods on [p_min, p_max], both ends included."""
    return np.geomspace(float(p_min), float(p_max), int(n))


def paper_frequency_grid(baseline_days: float = 3600.0, f_max_per_day: float = 480.0,
                         oversample: int = 3, as_periods_seconds: bool = True) -> np.ndarray:
    """The production period grid of Sec. 3: f from 2/B to f_max inclusive in steps
    of 1/(oversample B).  With the defaults it has 5,183,995 points.

    The count is taken in integer arithmetic: with df = 1/(k B) the number of steps
    from 2/B to f_max is f_max k B - 2 k."""
    k = int(oversample)
    steps = f_max_per_day * k * baseline_days - 2 * k
    n = int(np.floor(steps + 1e-9)) + 1
    f = (2.0 * k + np.arange(n, dtype=np.float64)) / (k * baseline_days)  # per day
    if as_periods_seconds:
        return DAY / f
    return f


def paper_pdot_grid(n: int, lo: float = 1e-12, hi: float = 1e-10) -> np.ndarray:
    """Sec. 3's period-derivative axis: n values log-spaced from -lo to -hi."""
    return -np.geomspace(lo, hi, int(n))
