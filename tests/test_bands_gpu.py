"""GPU parity of multi-filter input (Sec. 2.3: each filter of a curve median/std
normalised on its own, then combined): the device grid and top-k / significance
against the oracle fed the oracle's own normalised magnitudes, a calibrated copy
of a filter leaving the grid unchanged on the device, and the input checks.

Tolerances are those of the single-filter path (tests/gpu_util.py): the device
normalisation follows the same operation order as the oracle (exact median,
sequential binary64 moments), so FP64 mode is held to |dH| <= 1e-6 everywhere."""
import numpy as np
import pytest
import torch

import oracle
import paper_2006_06866_gb300 as g
import synth
from gpu_util import EPS_PHASE, TOL_H, compare_grid, dev_args

pytestmark = pytest.mark.gpu
MODES = ["fp64", "split32", "fixed32"]


@pytest.fixture(scope="module")
def h():
    hh = g.Handle(0)
    yield hh
    hh.close()


@pytest.fixture(scope="module")
def mb():
    b, bands = synth.make_multiband(61, n_curves=12, n_obs=500, n_bands=3, n_periods=700,
                                    pdots=(0.0, -2e-11))
    z = oracle.Oracle().band_normalize(b.mags, bands, b.offsets, 3)
    ref, dmin = oracle.Oracle().ce_grid(b.times, z, b.offsets, b.periods, b.pdots, 15, 10,
                                        with_dmin=True)
    return b, bands, ref, dmin


@pytest.mark.parametrize("mode", MODES)
def test_multiband_grid(h, mb, mode):
    b, bands, ref, dmin = mb
    got = g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=3,
                              cfg=g.Config(15, 10, mode), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK
    compare_grid(mode, got.cpu().numpy().astype(np.float64), ref, dmin)


@pytest.mark.parametrize("mode", MODES)
def test_multiband_overlapping_bins(h, mb, mode):
    """Multi-filter input with the paper's 50 half-overlapping phase bins."""
    b, bands, _, _ = mb
    z = oracle.Oracle().band_normalize(b.mags, bands, b.offsets, 3)
    ref, dmin = oracle.Oracle().ce_grid(b.times, z, b.offsets, b.periods, b.pdots, 50, 10,
                                        with_dmin=True, overlap=True)
    got = g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=3,
                              cfg=g.Config(50, 10, mode, overlap=True), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK
    compare_grid(mode, got.cpu().numpy().astype(np.float64), ref, dmin)


@pytest.mark.parametrize("mode", MODES)
def test_multiband_detect(h, mb, mode):
    b, bands, ref, dmin = mb
    k = 4
    tH, tI, mu, sd, rho = g.gce_ce_detect_bands(h, bands=torch.tensor(bands, device="cuda"),
                                                n_bands=3, cfg=g.Config(15, 10, mode), k=k,
                                                **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK
    tH, tI = tH.cpu().numpy().astype(np.float64), tI.cpu().numpy()
    flat, dm = ref.reshape(ref.shape[0], -1), dmin.reshape(ref.shape[0], -1)
    for c in range(ref.shape[0]):
        assert np.all(np.diff(tH[c]) >= 0)
        near = dm[c, tI[c]] <= 4 * EPS_PHASE[mode]
        assert np.all(np.abs(flat[c, tI[c]] - tH[c])[~near] <= TOL_H[mode])
    om, osd, orho = oracle.oracle_significance(ref)
    rho = rho.cpu().numpy().astype(np.float64)
    # the device top-k is exactly the k smallest of the device grid (ties by index)
    grid = g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=3,
                               cfg=g.Config(15, 10, mode), **dev_args(b))
    grid = grid.cpu().numpy().reshape(ref.shape[0], -1)
    for c in range(ref.shape[0]):
        order = np.lexsort((np.arange(grid.shape[1]), grid[c]))[:k]
        assert np.array_equal(tI[c], order), c
    if mode == "fp64":
        oH, _ = oracle.oracle_topk(ref, k)
        assert np.abs(tH - oH).max() <= TOL_H["fp64"]
        assert np.all(np.abs(mu.cpu().numpy() - om) <= 2e-6)
        assert np.all(np.abs(rho - orho) <= 1e-3 * np.maximum(1.0, orho) + 2e-6 / osd)
    else:
        assert np.all(np.abs(rho - orho) <= 5e-2 * np.maximum(1.0, orho))
    # top-k alone (no moments) gives the same cells
    tH2, tI2, m2, s2, r2 = g.gce_ce_detect_bands(h, bands=torch.tensor(bands, device="cuda"),
                                                 n_bands=3, cfg=g.Config(15, 10, mode), k=k,
                                                 significance=False, **dev_args(b))
    assert m2 is None and np.array_equal(tI2.cpu().numpy(), tI)


@pytest.mark.parametrize("mode", MODES)
def test_calibrated_copy_leaves_grid_unchanged(h, mode):
    """Every observation repeated in a second filter through 2 m + 3 (dyadic data, 64
    points, so the normalisation is exact): the device grid equals the one-filter
    grid.  Doubling every count leaves Eq. 4 unchanged; the device's fixed-point
    table rounds c ln c and 2c ln 2c independently, so H may move by one float32
    ulp, while a single point in another bin would move it by more than 1e-3."""
    rng = np.random.default_rng(62)
    n = 64
    t = np.sort(rng.uniform(0.0, 9e7, n))
    m0 = np.round((15.0 + 0.4 * np.sin(2 * np.pi * t / 1234.5) + rng.normal(0, 0.05, n))
                  * 1024.0) / 1024.0
    per = synth.log_periods(300.0, 3000.0, 900)
    pd = np.array([0.0, -1e-11])
    one = synth.LightCurveBatch("one", t, m0, np.array([0, n]), per, pd, 15, 10,
                                np.zeros(1), np.zeros(1), np.zeros(1))
    two = synth.LightCurveBatch("two", np.r_[t, t], np.r_[m0, 2.0 * m0 + 3.0],
                                np.array([0, 2 * n]), per, pd, 15, 10, np.zeros(1), np.zeros(1),
                                np.zeros(1))
    cfg = g.Config(15, 10, mode)
    g1 = g.gce_ce_grid_bands(h, bands=torch.zeros(n, dtype=torch.uint8, device="cuda"),
                             n_bands=1, cfg=cfg, **dev_args(one))
    b2 = torch.tensor(np.r_[np.zeros(n), np.ones(n)].astype(np.uint8), device="cuda")
    g2 = g.gce_ce_grid_bands(h, bands=b2, n_bands=2, cfg=cfg, **dev_args(two))
    assert g.gce_stream_status(h) == g.GCE_OK
    assert (g1.double() - g2.double()).abs().max().item() <= 1e-6


def test_band_index_checked_on_device(h, mb):
    b, bands, _, _ = mb
    bad = bands.copy()
    bad[5] = 3
    g.gce_ce_grid_bands(h, bands=torch.tensor(bad, device="cuda"), n_bands=3,
                        cfg=g.Config(15, 10, "split32"), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_ERR_INVALID
    g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=3,
                        cfg=g.Config(15, 10, "split32"), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK


@pytest.mark.parametrize("n_bands", [0, 9])
def test_band_count_range(h, mb, n_bands):
    b, bands, _, _ = mb
    with pytest.raises(g.GceError):
        g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=n_bands,
                            cfg=g.Config(15, 10, "fp64"), **dev_args(b))


def test_multiband_signed_magnitudes(h):
    """Values of both signs (the median's radix selection orders binary64 keys through
    their sign bit): FP64 grid against the oracle."""
    b, bands = synth.make_multiband(63, n_curves=6, n_obs=301, n_bands=2, n_periods=400)
    b.mags = b.mags - 15.3  # straddles zero in every filter
    z = oracle.Oracle().band_normalize(b.mags, bands, b.offsets, 2)
    ref = oracle.Oracle().ce_grid(b.times, z, b.offsets, b.periods, b.pdots, 15, 10)
    got = g.gce_ce_grid_bands(h, bands=torch.tensor(bands, device="cuda"), n_bands=2,
                              cfg=g.Config(15, 10, "fp64"), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK
    assert np.abs(got.cpu().numpy().astype(np.float64) - ref).max() <= TOL_H["fp64"]
