"""GPU parity of the rows beyond the core search: 50 %-overlapping phase bins
(Sec. 2.3) and the significance rho of the minimum (Eq. 5) with moments merged
across trial tiles (Sec. 4).

Tolerances for the moments: the device's H values are float32 and each tile's
moments are summed in FP32 around a shift before a FP64 merge, so against
statistics of the same float32 grid taken in float64: |d mean| <= 1e-6,
|d std| <= 1e-4 std, |d rho| <= 1e-3 max(1, rho).  Against the oracle (FP64
fold, |dH| <= 1e-6 per cell) the same bounds plus 1e-6 / std on rho."""
import numpy as np
import pytest
import torch

import oracle
import paper_2006_06866_gb300 as g
import synth
from gpu_util import EPS_PHASE, TOL_H, compare_grid, dev_args, sample_cells

pytestmark = pytest.mark.gpu
MODES = ["fp64", "split32", "fixed32"]


@pytest.fixture(scope="module")
def h():
    hh = g.Handle(0)
    yield hh
    hh.close()


def batch(seed=21, n_curves=6, pdots=(0.0, -4e-11, 1e-11), n_periods=900):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(30, 1500, size=n_curves)
    ts, ms = [], []
    for n in lengths:
        t = np.sort(rng.uniform(0, 9.46e7, int(n)))
        p0 = float(np.exp(rng.uniform(np.log(250), np.log(4000))))
        cyc = synth.lightcurves.chirp_cycles(t, p0, -3e-11)
        ms.append(15 + synth.lightcurves.eclipse_signal(cyc, 0.5, 0.04, 0.1)
                  + rng.normal(0, 0.03, int(n)))
        ts.append(t)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    return synth.LightCurveBatch("rows", np.concatenate(ts), np.concatenate(ms), offs,
                                 synth.log_periods(250, 4000, n_periods), np.asarray(pdots), 15,
                                 10, np.zeros(n_curves), np.zeros(n_curves), np.zeros(n_curves))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n_phase", [2, 15, 50])
def test_overlapping_bins_grid(h, mode, n_phase):
    b = batch()
    args = dev_args(b)
    cfg = g.Config(n_phase, 10, mode, overlap=True)
    got = g.gce_ce_grid(h, cfg=cfg, **args)
    assert g.gce_stream_status(h) == g.GCE_OK
    got = got.cpu().numpy().astype(np.float64)
    ref, dmin = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, n_phase,
                                        10, with_dmin=True, overlap=True)
    compare_grid(mode, got, ref, dmin)
    if mode == "fp64":
        rng = np.random.default_rng(3)
        cc, ct = sample_cells(rng, b.n_curves, b.periods.size * b.pdots.size, 200)
        cnt = g.gce_ce_counts(h, cfg=cfg, cell_curve=torch.tensor(cc, device="cuda"),
                              cell_trial=torch.tensor(ct, device="cuda"), **args)
        _, _, rc = oracle.Oracle().ce_cells(b.times, b.mags, b.offsets, b.periods, b.pdots,
                                            n_phase, 10, cc, ct, with_counts=True, overlap=True)
        assert np.array_equal(cnt.cpu().numpy().astype(np.int64), rc)
        single = g.gce_ce_grid_single(h, cfg=cfg, **args).cpu().numpy()
        assert np.array_equal(single, got.astype(np.float32))


@pytest.mark.parametrize("mode", MODES)
def test_overlap_packed_counter_limits(h, mode):
    """Overlapping bins on curves of 1023 points (the largest with two segments and the
    cumulative count packed in one counter word) and 1024 (the snapshot format): at the
    trial period P0 every point folds into one fine bin, half of them in the first
    magnitude segment and half in the last, so both segment fields, the cumulative field
    and the sums of two fine words reach their largest values (and H = ln 2 there).  Every cell against the
    oracle, with trials on both sides of P0."""
    p0, n_phase = 1.7, 50
    ts, ms, lengths = [], [], (1023, 1024)
    for n in lengths:
        k = np.arange(n, dtype=np.float64)
        ts.append(p0 * (k + 0.3 / n_phase))  # phase 0.006 at P0: inside fine bin 0
        ms.append(np.where(k < n // 2, 15.0, 16.0))
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    periods = p0 * (1.0 + 2e-5 * np.linspace(-1.0, 1.0, 33))
    assert periods[16] == p0
    b = synth.LightCurveBatch("limits", np.concatenate(ts), np.concatenate(ms), offs, periods,
                              np.zeros(1), n_phase, 10, np.zeros(2), np.zeros(2), np.zeros(2))
    cfg = g.Config(n_phase, 10, mode, overlap=True)
    got = g.gce_ce_grid(h, cfg=cfg, **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK
    got = got.cpu().numpy().astype(np.float64)
    ref, dmin = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, n_phase,
                                        10, with_dmin=True, overlap=True)
    # at P0 each overlapping bin holds the two segments half and half: H = ln 2
    assert abs(ref[1, 0, 16] - np.log(2.0)) < 1e-12
    compare_grid(mode, got, ref, dmin)


def test_overlap_needs_two_bins(h):
    b = batch()
    with pytest.raises(g.GceError):
        g.gce_ce_grid(h, cfg=g.Config(1, 10, "fp64", overlap=True), **dev_args(b))


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("mode", MODES)
def test_significance(h, mode, overlap):
    b = batch(seed=22, n_curves=5, n_periods=3001)  # several tiles with a ragged tail
    args = dev_args(b)
    cfg = g.Config(15, 10, mode, overlap=overlap)
    k = 4
    tH, tI, mu, sd, rho = g.gce_ce_detect(h, cfg=cfg, k=k, **args)
    assert g.gce_stream_status(h) == g.GCE_OK
    rH, rI = g.gce_ce_topk(h, cfg=cfg, k=k, **args)
    assert torch.equal(tH, rH) and torch.equal(tI, rI)
    mu, sd, rho = mu.cpu().numpy(), sd.cpu().numpy(), rho.cpu().numpy().astype(np.float64)
    # against the statistics of the device's own float32 grid
    grid = g.gce_ce_grid(h, cfg=cfg, **args).cpu().numpy().astype(np.float64)
    gm, gs, gr = oracle.oracle_significance(grid)
    assert np.all(np.abs(mu - gm) <= 1e-6)
    assert np.all(np.abs(sd - gs) <= 1e-4 * gs)
    assert np.all(np.abs(rho - gr) <= 1e-3 * np.maximum(1.0, gr))
    # against the oracle
    ref = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, 15, 10,
                                  overlap=overlap)
    om, osd, orho = oracle.oracle_significance(ref)
    if mode == "fp64":
        assert np.all(np.abs(mu - om) <= 2e-6)
        assert np.all(np.abs(sd - osd) <= 1e-4 * osd + 1e-6)
        assert np.all(np.abs(rho - orho) <= 1e-3 * np.maximum(1.0, orho) + 2e-6 / osd)
    else:
        # a few near-edge cells may differ by one point's bin: compare loosely
        assert np.all(np.abs(mu - om) <= 1e-3)
        assert np.all(np.abs(rho - orho) <= 5e-2 * np.maximum(1.0, orho))


def test_significance_separates_signal_from_noise(h):
    """Eq. 5 on the device: injected on-grid eclipses clear the rho = 10 threshold of
    Sec. 3.2, pure noise does not."""
    periods = synth.log_periods(300.0, 600.0, 2000)
    b, pi, qi = synth.make_onegrid_injection(91, 6, 600, periods, [0.0], noise=0.02)
    rng = np.random.default_rng(92)
    noise_m = 15 + rng.normal(0, 0.02, b.times.size)
    _, _, _, _, rho_s = g.gce_ce_detect(h, cfg=g.Config(15, 10, "split32"), k=1, **dev_args(b))
    nb = synth.LightCurveBatch("noise", b.times, noise_m, b.offsets, b.periods, b.pdots, 15, 10,
                               b.truth_p0, b.truth_pdot, b.truth_class)
    _, _, _, _, rho_n = g.gce_ce_detect(h, cfg=g.Config(15, 10, "split32"), k=1, **dev_args(nb))
    assert float(rho_s.min()) > 10.0 and float(rho_n.max()) < 10.0


@pytest.mark.parametrize("mode", MODES)
def test_significance_flat_grid(h, mode):
    """A curve whose grid is flat (constant magnitudes, or a single point: H = 0 in
    every cell) has sigma = 0 and rho = 0 exactly on the device, as in the oracle;
    the other curves of the batch are unaffected."""
    b = batch(seed=23, n_curves=3, n_periods=1500)
    n0 = int(b.offsets[1])
    mags = b.mags.copy()
    mags[:n0] = 15.25
    times = np.r_[b.times, 1234.5]
    mags = np.r_[mags, 16.0]
    offs = np.r_[b.offsets, b.offsets[-1] + 1].astype(np.int64)
    fb = synth.LightCurveBatch("flat", times, mags, offs, b.periods, b.pdots, 15, 10,
                               np.zeros(4), np.zeros(4), np.zeros(4))
    tH, _, mu, sd, rho = g.gce_ce_detect(h, cfg=g.Config(15, 10, mode), k=3, **dev_args(fb))
    assert g.gce_stream_status(h) == g.GCE_OK
    mu, sd, rho = mu.cpu().numpy(), sd.cpu().numpy(), rho.cpu().numpy()
    for c in (0, 3):
        assert tH[c].abs().max().item() == 0.0
        assert mu[c] == 0.0 and sd[c] == 0.0 and rho[c] == 0.0
    ref = oracle.Oracle().ce_grid(fb.times, fb.mags, fb.offsets, fb.periods, fb.pdots, 15, 10)
    om, osd, orho = oracle.oracle_significance(ref)
    assert osd[0] == 0.0 and orho[0] == 0.0 and osd[3] == 0.0 and orho[3] == 0.0
    assert np.all(np.abs(rho[1:3] - orho[1:3]) <= 5e-2 * np.maximum(1.0, orho[1:3]))
