"""Short curves share a trial tile: curves of at most 256 points are scheduled
tile-major, so one CTA takes a tile's trial constants once and runs them over
consecutive short curves, each with its own staged points, segment starts,
counters and top-k.  Every cell of such batches is checked against the oracle."""
import numpy as np
import pytest

import synth
from gpu_util import TOL_H, compare_grid, dev_args, gpu_grid

import paper_2006_06866_gb300 as g

pytestmark = pytest.mark.gpu
MODES = ["fp64", "split32", "fixed32"]


def batch_of(lengths, seed, n_periods=1300, pdots=(0.0,), t0=0.0):
    rng = np.random.default_rng(seed)
    ts, ms = [], []
    for n in lengths:
        t = np.sort(rng.uniform(0, 3 * 365 * 86400.0, size=n))
        p0 = np.exp(rng.uniform(np.log(300), np.log(4000)))
        cyc = synth.lightcurves.chirp_cycles(t, p0, -1e-11)
        m = 15 + synth.lightcurves.eclipse_signal(cyc, 0.6, 0.05, 0.3) + rng.normal(0, 0.02, n)
        ts.append(t)
        ms.append(m)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    k = len(lengths)
    return synth.LightCurveBatch("short", np.concatenate(ts), np.concatenate(ms), offs,
                                 synth.log_periods(300.0, 4000.0, n_periods), np.asarray(pdots),
                                 15, 10, np.zeros(k), np.zeros(k), np.zeros(k), t0=t0)


@pytest.fixture(scope="module")
def h():
    hh = g.Handle(0)
    yield hh
    hh.close()


@pytest.mark.parametrize("mode", MODES)
def test_short_curves_share_tiles_every_cell(h, orc, mode):
    """Lengths 1, 2, 7, 33, 50, 63, 64, 65 in one launch: every curve is short, so
    every tile is taken tile-major across all eight curves; 1300 periods give
    several tiles and a ragged last one."""
    b = batch_of([1, 2, 7, 33, 50, 63, 64, 65], seed=31)
    got = gpu_grid(h, dev_args(b), mode)
    ref, dmin = orc.ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, 15, 10,
                            with_dmin=True)
    compare_grid(mode, got, ref, dmin)


@pytest.mark.parametrize("mode", MODES)
def test_long_and_short_curves_in_one_launch(h, orc, mode):
    """Long curves (curve-major) and short ones (tile-major) in one launch, with
    a Pdot axis, t0 inside the baseline and 50 %-overlapping bins: every cell, and
    the top-k, against the oracle."""
    lengths = [700, 3, 257, 256, 1, 90, 1200, 65, 64, 400, 2]
    b = batch_of(lengths, seed=32, n_periods=700, pdots=(0.0, -2e-11, 1e-11), t0=3.0e7)
    args = dev_args(b)
    for ovl in (False, True):
        cfg = g.Config(15, 10, mode, t0=b.t0, overlap=ovl)
        got = g.gce_ce_grid(h, cfg=cfg, **args)
        assert g.gce_stream_status(h) == g.GCE_OK
        got = got.cpu().numpy().astype(np.float64)
        ref, dmin = orc.ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, 15, 10, t0=b.t0,
                                with_dmin=True, overlap=ovl)
        compare_grid(mode, got, ref, dmin)
        tH, tI = g.gce_ce_topk(h, cfg=cfg, k=4, **args)
        tH, tI = tH.cpu().numpy(), tI.cpu().numpy()
        flat = got.reshape(b.n_curves, -1)
        for c in range(b.n_curves):
            order = np.lexsort((np.arange(flat.shape[1]), flat[c]))[:4]
            assert np.array_equal(tI[c], order), (ovl, c)
