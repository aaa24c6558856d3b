"""Helpers shared by the GPU parity tests: moving a synthetic batch to the
device, running the library through its C ABI, and comparing against the CPU
oracle with the tolerances of the parity contract.

Tolerances (written here once, used by every GPU test):
  FP64 fold:    histogram counts bit-exact; |dH| <= 1e-6 on every cell.
  SPLIT32/FIXED32: |dH| <= 1e-4 on every cell whose points all lie farther than
                4 eps from a phase-bin edge (the oracle's dmin); cells closer
                than that may legitimately differ by a point's bin and are only
                counted.  eps is each fold's phase-error bound in cycles.
"""
from __future__ import annotations

import numpy as np
import torch

import paper_2006_06866_gb300 as g

TOL_H = {"fp64": 1e-6, "split32": 1e-4, "fixed32": 1e-4}
# Phase-error bounds of the two reduced-precision folds, in cycles (see DESIGN
# notes for the derivation); near-edge cells are those with dmin <= 4 eps.
EPS_PHASE = {"fp64": 0.0, "split32": 2.5e-7, "fixed32": 4e-9}


def dev_args(batch, pdots=None, periods=None, device="cuda:0"):
    d = torch.device(device)
    per = batch.periods if periods is None else periods
    pdt = batch.pdots if pdots is None else pdots
    return dict(times=torch.tensor(batch.times, device=d), mags=torch.tensor(batch.mags, device=d),
                offsets=np.asarray(batch.offsets, dtype=np.int64),
                periods=torch.tensor(np.asarray(per, dtype=np.float64), device=d),
                pdots=torch.tensor(np.asarray(pdt, dtype=np.float64), device=d))


def gpu_grid(h, args, mode, n_phase=15, n_mag=10, t0=0.0, use_graph=True):
    cfg = g.Config(n_phase, n_mag, mode, t0=t0, use_graph=use_graph)
    out = g.gce_ce_grid(h, cfg=cfg, **args)
    st = g.gce_stream_status(h)
    assert st == g.GCE_OK, st
    return out.cpu().numpy().astype(np.float64)


def compare_grid(mode, got, ref, dmin):
    """Returns a dict of statistics; asserts the parity contract."""
    err = np.abs(got - ref)
    stats = {"cells": int(err.size), "max_err": float(err.max()) if err.size else 0.0}
    if mode == "fp64":
        assert err.max() <= TOL_H["fp64"], f"fp64 max |dH| {err.max():.3g}"
        return stats
    far = dmin > 4 * EPS_PHASE[mode]
    stats["near_edge"] = int((~far).sum())
    stats["near_edge_frac"] = float((~far).mean())
    stats["max_err_far"] = float(err[far].max()) if far.any() else 0.0
    stats["max_err_near"] = float(err[~far].max()) if (~far).any() else 0.0
    assert stats["max_err_far"] <= TOL_H[mode], (mode, stats)
    return stats


def sample_cells(rng, n_curves, n_trials, n):
    cc = rng.integers(0, n_curves, size=n)
    ct = rng.integers(0, n_trials, size=n)
    return cc.astype(np.int64), ct.astype(np.int64)
