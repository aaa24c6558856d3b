"""Partition of a ragged light-curve batch across ranks.

Curves are independent (every (curve, trial) cell is), so a multi-GPU run gives
each rank a disjoint set of curves and needs no collective on the data path.
The work of a curve is its point count times the (shared) trial count, so curves
are assigned longest first to the rank with the least work so far (greedy LPT).
"""
from __future__ import annotations

import numpy as np


def shard_curves(n_obs, world: int):
    """Curve indices per rank (each sorted ascending), balanced by points."""
    n_obs = np.asarray(n_obs, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-n_obs, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(n_obs.shape[0], dtype=np.int64)
    for c in order:
        r = int(np.argmin(load))
        owner[c] = r
        load[r] += n_obs[c]
    return [np.flatnonzero(owner == r) for r in range(world)]


def shard_arrays(times, mags, offsets, curves):
    """(times, mags, offsets) of the listed curves, concatenated in that order."""
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = [np.arange(offsets[c], offsets[c + 1]) for c in curves]
    sel = np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)
    n = np.array([offsets[c + 1] - offsets[c] for c in curves], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    return np.asarray(times)[sel], np.asarray(mags)[sel], offs
