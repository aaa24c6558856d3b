"""Seeded synthetic light curves and trial grids for the CE (P, Pdot) search.

This package only draws inputs: observation times, magnitudes, trial periods and
period derivatives.  It holds none of the search's arithmetic (no fold, no
binning, no entropy), so the CPU oracle and the GPU path can both be fed from it
without sharing any of the method.

Injected signals follow the period law of Eq. 2 (P(t) = P0 + Pdot t) through its
exact phase integral, cycles(tau) = ln(1 + Pdot tau / P0) / Pdot (tau / P0 when
Pdot = 0).  That is the physical model the paper injects (Sec. 2.2 stitches
light curves whose period changes with time); the search's Eq. 3 is its
first-order expansion, and the two differ by Pdot^2 tau^3 / (3 P0^3) cycles
(below 6e-4 cycles for every configuration here).
"""
from .grids import (linear_frequency_periods, log_periods, paper_frequency_grid,
                    paper_pdot_grid)
from .lightcurves import (CONFIG_NAMES, LightCurveBatch, make_config, make_multiband,
                          make_onegrid_injection,
                          nightly_cadence, sparse_cadence, uniform_cadence)

__all__ = [
    "CONFIG_NAMES", "LightCurveBatch", "make_config", "make_multiband", "make_onegrid_injection",
    "nightly_cadence", "sparse_cadence", "uniform_cadence", "linear_frequency_periods",
    "log_periods", "paper_frequency_grid", "paper_pdot_grid",
]
