"""CPU oracle for the conditional-entropy (P, Pdot) search.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow CPU statement of
what the GPU path computes (Eq. 3 fold, Sec. 2.3 histogram, Eq. 4 entropy of
arXiv:2006.06866).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import it.  The GPU library never
imports it, and it imports nothing from the GPU library.

The arithmetic lives in ``ce_oracle.c`` (binary64, pinned operation order,
built with ``-ffp-contract=off``); this module only compiles it with gcc and
marshals numpy arrays through ctypes.  Top-k selection is a stable numpy sort
of the oracle grid by (H, flat trial index), as the ``oracle_topk`` helper
states.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ce_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or one planted-mistake variant) with gcc."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    if mutant:
        cmd.insert(1, f"-DORACLE_MUTANT={int(mutant)}")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


def _bind(lib):
    lib.oracle_mag_bins.argtypes = [_D, ctypes.c_int64, ctypes.c_int32, _I32]
    lib.oracle_mag_bins.restype = None
    lib.oracle_trial_constants.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
    lib.oracle_trial_constants.restype = None
    lib.oracle_phase_bin.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int32, _D]
    lib.oracle_phase_bin.restype = ctypes.c_int32
    lib.oracle_entropy.argtypes = [_I64, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_entropy.restype = ctypes.c_double
    lib.oracle_cell.argtypes = [_D, _D, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                _I64, _D]
    lib.oracle_cell.restype = ctypes.c_double
    lib.oracle_ce_grid.argtypes = [_D, _D, _I64, ctypes.c_int32, _D, ctypes.c_int32, _D,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_int32, _D, _D, ctypes.c_int32]
    lib.oracle_ce_grid.restype = ctypes.c_int
    lib.oracle_ce_cells.argtypes = [_D, _D, _I64, _D, ctypes.c_int32, _D, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_int64, _I64, _I64, _D, _D, _I64, ctypes.c_int32]
    lib.oracle_ce_cells.restype = ctypes.c_int
    lib.oracle_band_normalize.argtypes = [_D, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64,
                                          ctypes.c_int32, _D]
    lib.oracle_band_normalize.restype = ctypes.c_int
    return lib


def load(mutant: int = 0):
    """The compiled oracle as a ctypes library (built on first use)."""
    with _lock:
        if mutant not in _libs:
            _libs[mutant] = _bind(ctypes.CDLL(build(mutant)))
        return _libs[mutant]


def _p(a, typ):
    return a.ctypes.data_as(typ)


class Oracle:
    """numpy front end of one compiled oracle build (mutant 0 = the real one)."""

    def __init__(self, mutant: int = 0):
        self.lib = load(mutant)
        self.mutant = mutant

    # --- single steps -------------------------------------------------------
    def mag_bins(self, mags, n_mag):
        m = np.ascontiguousarray(mags, dtype=np.float64)
        out = np.empty(m.shape[0], dtype=np.int32)
        self.lib.oracle_mag_bins(_p(m, _D), m.shape[0], int(n_mag), _p(out, _I32))
        return out

    def trial_constants(self, period, pdot):
        f = ctypes.c_double()
        a = ctypes.c_double()
        self.lib.oracle_trial_constants(float(period), float(pdot), ctypes.byref(f), ctypes.byref(a))
        return f.value, a.value

    def phase_bin(self, tau, f, a, n_phase):
        y = ctypes.c_double()
        j = self.lib.oracle_phase_bin(float(tau), float(f), float(a), int(n_phase), ctypes.byref(y))
        return j, y.value

    def entropy(self, counts):
        c = np.ascontiguousarray(counts, dtype=np.int64)
        n_mag, n_phase = c.shape
        return self.lib.oracle_entropy(_p(c, _I64), n_mag, n_phase)

    def cell(self, t, m, t0, period, pdot, n_phase, n_mag, overlap=False):
        """(H, counts[n_mag, n_phase], dmin) of one curve at one trial."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        counts = np.zeros((n_mag, n_phase), dtype=np.int64)
        dmin = ctypes.c_double()
        h = self.lib.oracle_cell(_p(t, _D), _p(m, _D), t.shape[0], float(t0), float(period),
                                 float(pdot), int(n_phase), int(n_mag), int(bool(overlap)),
                                 _p(counts, _I64), ctypes.byref(dmin))
        return h, counts, dmin.value

    def band_normalize(self, mags, bands, offsets, n_bands):
        """Multi-filter input (Sec. 2.3): every (curve, filter) median/std normalised
        (oracle_band_normalize, curve by curve).  Raises on a band index >= n_bands."""
        mags = np.ascontiguousarray(mags, dtype=np.float64)
        bands = np.ascontiguousarray(bands, dtype=np.uint8)
        offsets = np.asarray(offsets, dtype=np.int64)
        out = np.empty_like(mags)
        for c in range(offsets.shape[0] - 1):
            lo, hi = int(offsets[c]), int(offsets[c + 1])
            m, b, o = mags[lo:hi], bands[lo:hi], out[lo:hi]
            r = self.lib.oracle_band_normalize(_p(m, _D), b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                               hi - lo, int(n_bands), _p(o, _D))
            if r != 0:
                raise ValueError("band index >= n_bands")
        return out

    # --- batches ------------------------------------------------------------
    def ce_grid(self, times, mags, offsets, periods, pdots, n_phase, n_mag, t0=0.0,
                n_threads=0, with_dmin=False, overlap=False):
        """H[n_curves, n_pdots, n_periods] (float64); with_dmin adds the edge distance."""
        times = np.ascontiguousarray(times, dtype=np.float64)
        mags = np.ascontiguousarray(mags, dtype=np.float64)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        periods = np.ascontiguousarray(periods, dtype=np.float64)
        pdots = np.ascontiguousarray(pdots, dtype=np.float64)
        nc = offsets.shape[0] - 1
        out = np.empty((nc, pdots.shape[0], periods.shape[0]), dtype=np.float64)
        dmin = np.empty_like(out) if with_dmin else None
        used = self.lib.oracle_ce_grid(
            _p(times, _D), _p(mags, _D), _p(offsets, _I64), nc, _p(periods, _D),
            periods.shape[0], _p(pdots, _D), pdots.shape[0], int(n_phase), int(n_mag),
            float(t0), int(bool(overlap)), _p(out, _D), _p(dmin, _D) if with_dmin else None,
            int(n_threads))
        self.threads_used = used
        return (out, dmin) if with_dmin else out

    def ce_cells(self, times, mags, offsets, periods, pdots, n_phase, n_mag, cell_curve,
                 cell_trial, t0=0.0, with_counts=False, n_threads=0, overlap=False):
        """(H[n_cells], dmin[n_cells], counts[n_cells, n_mag, n_phase] or None)."""
        times = np.ascontiguousarray(times, dtype=np.float64)
        mags = np.ascontiguousarray(mags, dtype=np.float64)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        periods = np.ascontiguousarray(periods, dtype=np.float64)
        pdots = np.ascontiguousarray(pdots, dtype=np.float64)
        cc = np.ascontiguousarray(cell_curve, dtype=np.int64)
        ct = np.ascontiguousarray(cell_trial, dtype=np.int64)
        n = cc.shape[0]
        h = np.empty(n, dtype=np.float64)
        dmin = np.empty(n, dtype=np.float64)
        counts = np.zeros((n, n_mag, n_phase), dtype=np.int64) if with_counts else None
        used = self.lib.oracle_ce_cells(
            _p(times, _D), _p(mags, _D), _p(offsets, _I64), _p(periods, _D), periods.shape[0],
            _p(pdots, _D), int(n_phase), int(n_mag), float(t0), int(bool(overlap)), n,
            _p(cc, _I64), _p(ct, _I64),
            _p(h, _D), _p(dmin, _D), _p(counts, _I64) if with_counts else None, int(n_threads))
        self.threads_used = used
        return h, dmin, counts


def oracle_significance(grid):
    """Eq. 5 per curve from an oracle grid H[c, q, p]: rho = (mu - H_min) / sigma with
    mu and sigma the mean and population standard deviation (ddof 0; the paper
    does not say which) of all of the curve's CE values.  Returns (mu, sigma,
    rho); rho is 0 where sigma is 0.  The moments are taken of H - H_min (the
    standard deviation does not depend on the shift, and mu - H_min is the mean of
    the shifted values), so a flat grid has sigma = 0 exactly."""
    flat = grid.reshape(grid.shape[0], -1)
    h_min = flat.min(axis=1)
    d = flat - h_min[:, None]
    gap = d.mean(axis=1)
    sd = d.std(axis=1)
    rho = np.where(sd > 0, gap / np.where(sd > 0, sd, 1.0), 0.0)
    return h_min + gap, sd, rho


def oracle_topk(grid, k):
    """Per-curve k smallest cells of an oracle grid H[c, q, p]: the first k of the
    stable sort by (H, flat index q * n_periods + p) -- ties go to the smaller
    flat index (Sec. 2.3 takes the grid minimum; ties are not discussed there)."""
    flat = grid.reshape(grid.shape[0], -1)
    idx = np.argsort(flat, axis=1, kind="stable")[:, :k]
    return np.take_along_axis(flat, idx, axis=1), idx.astype(np.int64)
