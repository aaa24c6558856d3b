"""GPU edge cases, device-side input checks, determinism, graph replay and the
host-buffer entry point."""
import math

import numpy as np
import pytest
import torch
from scipy.stats import entropy as shannon

import oracle
import paper_2006_06866_gb300 as g
import synth
from gpu_util import compare_grid, dev_args, gpu_grid

pytestmark = pytest.mark.gpu
MODES = ["fp64", "split32", "fixed32"]


@pytest.fixture(scope="module")
def h():
    hh = g.Handle(0)
    yield hh
    hh.close()


def small_batch(seed=0, n_curves=3, n_obs=200, n_periods=300, pdots=(0.0,)):
    rng = np.random.default_rng(seed)
    ts = [np.sort(rng.uniform(0, 9e7, n_obs)) for _ in range(n_curves)]
    ms = [15 + 0.3 * np.sin(2 * np.pi * t / 1234.5) + rng.normal(0, 0.05, n_obs) for t in ts]
    offs = np.arange(n_curves + 1, dtype=np.int64) * n_obs
    return synth.LightCurveBatch("small", np.concatenate(ts), np.concatenate(ms), offs,
                                 synth.log_periods(300, 3000, n_periods), np.asarray(pdots), 15, 10,
                                 np.zeros(n_curves), np.zeros(n_curves), np.zeros(n_curves))


def test_empty_batch_is_noop(h):
    b = small_batch()
    args = dev_args(b)
    args["offsets"] = np.zeros(1, dtype=np.int64)
    out = torch.full((0, 1, b.periods.size), 7.0, device="cuda")
    g.gce_ce_grid(h, cfg=g.Config(), out=out, **args)
    assert g.gce_stream_status(h) == g.GCE_OK


@pytest.mark.parametrize("mode", MODES)
def test_degenerate_cases(h, mode):
    """N = 1 and constant magnitudes give H = 0; one magnitude bin gives 0; one
    phase bin gives the magnitude histogram's Shannon entropy at every trial."""
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 9e7, 300))
    m = 15 + rng.normal(0, 0.1, 300)
    parts = [(t[:1], m[:1]), (t[:50], np.full(50, 15.5)), (t, m)]
    offs = np.concatenate([[0], np.cumsum([len(x) for x, _ in parts])]).astype(np.int64)
    b = synth.LightCurveBatch("deg", np.concatenate([x for x, _ in parts]),
                              np.concatenate([y for _, y in parts]), offs,
                              synth.log_periods(300, 3000, 257), np.array([0.0, -1e-11]), 15, 10,
                              np.zeros(3), np.zeros(3), np.zeros(3))
    args = dev_args(b)
    H = gpu_grid(h, args, mode)
    assert np.all(H[0] == 0.0) and np.all(H[1] == 0.0)
    assert np.all(gpu_grid(h, args, mode, n_mag=1) == 0.0)
    H1 = gpu_grid(h, args, mode, n_phase=1)
    bins = oracle.Oracle().mag_bins(m, 10)
    expect = shannon(np.bincount(bins, minlength=10).astype(float))
    assert np.abs(H1[2] - expect).max() <= 1e-6


@pytest.mark.parametrize("bins", [(1, 1), (2, 3), (50, 10), (256, 255), (7, 200)])
def test_bin_counts_range(h, bins):
    n_phase, n_mag = bins
    b = small_batch(seed=4, n_curves=2, n_obs=300, n_periods=130, pdots=(0.0, -2e-11))
    args = dev_args(b)
    got = gpu_grid(h, args, "fp64", n_phase=n_phase, n_mag=n_mag)
    ref = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, n_phase, n_mag)
    assert np.abs(got - ref).max() <= 1e-6


@pytest.mark.parametrize("mode", MODES)
def test_bad_inputs_flagged_on_device(h, mode):
    b = small_batch(seed=5)
    for field, idx, val in [("times", 17, np.nan), ("mags", 3, np.inf), ("periods", 5, 0.0),
                            ("periods", 9, -3.0), ("pdots", 0, np.nan)]:
        args = dev_args(b)
        args[field][idx] = val
        g.gce_ce_grid(h, cfg=g.Config(15, 10, mode), **args)
        assert g.gce_stream_status(h) == g.GCE_ERR_INVALID, (field, val)
    # a clean call afterwards is fine again
    g.gce_ce_grid(h, cfg=g.Config(15, 10, mode), **dev_args(b))
    assert g.gce_stream_status(h) == g.GCE_OK


def test_out_of_range_fold_is_unsupported(h):
    """SPLIT32 needs |tau|/P < 2^21 cycles: 1e9 s at a 100 s period is refused."""
    b = small_batch(seed=6, n_periods=64)
    args = dev_args(b)
    args["times"] = args["times"] * 12.0
    args["periods"] = torch.full_like(args["periods"], 100.0)
    g.gce_ce_grid(h, cfg=g.Config(15, 10, "split32"), **args)
    assert g.gce_stream_status(h) == g.GCE_ERR_UNSUPPORTED
    g.gce_ce_grid(h, cfg=g.Config(15, 10, "fixed32"), **args)
    assert g.gce_stream_status(h) == g.GCE_OK


@pytest.mark.parametrize("overlap", [False, True])
def test_split_fold_near_cycle_limit(h, overlap):
    """The SPLIT32 fold at the edge of its range (up to 0.99 2^21 cycles, where its
    residual strays farthest from [-1/2, 1/2]), with and without the Pdot term and
    with phase-bin counts from 2 to 256: every count still reaches the entropy
    (the epilogue reads only the slots the fold's bound allows), so the grid
    matches the oracle's."""
    rng = np.random.default_rng(41)
    n_obs, n_curves = 300, 3
    ts = [np.sort(rng.uniform(0.0, 2.0e8, n_obs)) for _ in range(n_curves)]
    ts[0][-1] = 2.0e8
    ms = [15 + 0.3 * np.sin(2 * np.pi * t / 97.1) + rng.normal(0, 0.05, n_obs) for t in ts]
    offs = np.arange(n_curves + 1, dtype=np.int64) * n_obs
    periods = np.linspace(96.0, 500.0, 257)  # 2e8 s / 96 s = 0.993 2^21 cycles
    b = synth.LightCurveBatch("edge", np.concatenate(ts), np.concatenate(ms), offs, periods,
                              np.array([0.0, -1e-13]), 15, 10, np.zeros(n_curves),
                              np.zeros(n_curves), np.zeros(n_curves))
    args = dev_args(b)
    for n_phase in (2, 3, 15, 16, 64, 256):
        cfg = g.Config(n_phase, 10, "split32", overlap=overlap)
        got = g.gce_ce_grid(h, cfg=cfg, **args)
        assert g.gce_stream_status(h) == g.GCE_OK
        ref, dmin = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots,
                                            n_phase, 10, with_dmin=True, overlap=overlap)
        compare_grid("split32", got.cpu().numpy().astype(np.float64), ref, dmin)


@pytest.mark.parametrize("pdots", [(0.0,), (0.0, -1e-11, -2e-11)])
def test_autotune_on_the_job(h, pdots):
    """Tuning on a slice of the job itself caches a valid shape under the job's key
    and leaves the results unchanged."""
    b = small_batch(seed=10, n_curves=3, n_obs=400, n_periods=3000, pdots=pdots)
    args = dev_args(b)
    cfg = g.Config(15, 10, "split32")
    before = g.gce_ce_grid(h, cfg=cfg, **args).cpu().numpy()
    g.gce_autotune_job(h, cfg=cfg, **args)
    t = g.gce_get_tuning(h, cfg, 400, n_pdots=len(pdots))
    assert t["block"] in (128, 256, 512) and t["tpt"] in (1, 2, 4)
    assert t["slot_range"] in (0, 1)  # the tuner may keep the mid SPLIT32 slot range
    after = g.gce_ce_grid(h, cfg=cfg, **args).cpu().numpy()
    assert np.array_equal(before, after)


def test_four_trials_per_thread_not_built_for_fp64(h):
    with pytest.raises(g.GceError):
        g.gce_set_tuning(h, g.Config(15, 10, "fp64"), 500, block=128, tpt=4)
    with pytest.raises(g.GceError):  # slot ranges: 0 (wide) and 1 (mid) only
        g.gce_set_tuning(h, g.Config(15, 10, "split32"), 500, block=128, tpt=2, slot_range=2)
    g.gce_set_tuning(h, g.Config(15, 10, "split32"), 500, block=128, tpt=4)


@pytest.mark.parametrize("n_phase", [2, 15, 50])
def test_split_narrow_slots_without_pdot(h, n_phase):
    """A job with a Pdot axis keeps SPLIT32's narrow slot range, so its tiles whose Pdot
    values are all 0 re-reduce the residual too: near the fold's cycle limit the grid
    equals the one-Pdot grid (wide slot range) bit for bit and the oracle's."""
    rng = np.random.default_rng(43)
    n_obs, n_curves = 300, 3
    ts = [np.sort(rng.uniform(0.0, 2.0e8, n_obs)) for _ in range(n_curves)]
    ms = [15 + 0.3 * np.sin(2 * np.pi * t / 97.1) + rng.normal(0, 0.05, n_obs) for t in ts]
    offs = np.arange(n_curves + 1, dtype=np.int64) * n_obs
    periods = np.linspace(96.0, 500.0, 257)
    mk = lambda pd: synth.LightCurveBatch("narrow", np.concatenate(ts), np.concatenate(ms), offs,
                                          periods, np.asarray(pd), 15, 10, np.zeros(n_curves),
                                          np.zeros(n_curves), np.zeros(n_curves))
    cfg = g.Config(n_phase, 10, "split32")
    for tpt in (1, 2, 4):  # flat tiles and period-major tiles
        g.gce_set_tuning(h, cfg, n_obs, block=128, tpt=tpt, chunk=512)
        two = g.gce_ce_grid(h, cfg=cfg, **dev_args(mk([0.0, 0.0]))).cpu().numpy()
        one = g.gce_ce_grid(h, cfg=cfg, **dev_args(mk([0.0]))).cpu().numpy()
        assert g.gce_stream_status(h) == g.GCE_OK
        assert np.array_equal(two[:, 0], one[:, 0]) and np.array_equal(two[:, 1], one[:, 0])
    ref, dmin = oracle.Oracle().ce_grid(np.concatenate(ts), np.concatenate(ms), offs, periods,
                                        np.array([0.0]), n_phase, 10, with_dmin=True)
    compare_grid("split32", one.astype(np.float64), ref, dmin)


@pytest.mark.parametrize("n_phase,overlap", [(2, False), (15, False), (50, False), (15, True),
                                             (50, True)])
def test_split_mid_slot_range(h, n_phase, overlap):
    """SPLIT32's mid slot range (slot_range = 1) keeps fewer counter slots; the warps
    whose trials could fold outside it (here the periods below about 400, a third of
    the grid, at 2e8 time units) re-reduce their residuals, the others do not.  Either
    way the counts are those of the wide range: the grids agree bit for bit at every
    trials-per-thread, and with the oracle."""
    rng = np.random.default_rng(47)
    n_obs, n_curves = 300, 3
    ts = [np.sort(rng.uniform(0.0, 2.0e8, n_obs)) for _ in range(n_curves)]
    ms = [15 + 0.3 * np.sin(2 * np.pi * t / 731.3) + rng.normal(0, 0.05, n_obs) for t in ts]
    offs = np.arange(n_curves + 1, dtype=np.int64) * n_obs
    periods = np.geomspace(96.0, 5000.0, 257)
    b = synth.LightCurveBatch("mid", np.concatenate(ts), np.concatenate(ms), offs, periods,
                              np.zeros(1), n_phase, 10, np.zeros(n_curves), np.zeros(n_curves),
                              np.zeros(n_curves))
    cfg = g.Config(n_phase, 10, "split32", overlap=overlap)
    grids = {}
    for tpt in (1, 2, 4):
        for sr in (0, 1):
            g.gce_set_tuning(h, cfg, n_obs, block=128, tpt=tpt, chunk=512, slot_range=sr)
            assert g.gce_get_tuning(h, cfg, n_obs)["slot_range"] == sr
            grids[tpt, sr] = g.gce_ce_grid(h, cfg=cfg, **dev_args(b)).cpu().numpy()
            assert g.gce_stream_status(h) == g.GCE_OK
        assert np.array_equal(grids[tpt, 0], grids[tpt, 1])
    g.gce_set_tuning(h, cfg, n_obs, block=256, tpt=2, chunk=2048)
    ref, dmin = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, n_phase,
                                        10, with_dmin=True, overlap=overlap)
    compare_grid("split32", grids[2, 1].astype(np.float64), ref, dmin)


@pytest.mark.parametrize("mode", MODES)
def test_longest_curve(h, mode):
    """A curve of the maximum length (65,535 points: counts above the 2048 c ln c entries
    kept in shared memory read the table from global memory, and the points are staged
    in many chunks) beside a 3-point curve, with and without a Pdot axis."""
    rng = np.random.default_rng(44)
    n_long = 65535
    t_long = np.sort(rng.uniform(0.0, 9e7, n_long))
    m_long = 15 + 0.3 * np.sin(2 * np.pi * t_long / 1234.5) + rng.normal(0, 0.05, n_long)
    t_short, m_short = np.array([1e6, 2e6, 3.5e6]), np.array([15.0, 15.4, 15.1])
    offs = np.array([0, n_long, n_long + 3], dtype=np.int64)
    for pdots in ((0.0,), (0.0, -2e-11)):
        b = synth.LightCurveBatch("long", np.r_[t_long, t_short], np.r_[m_long, m_short], offs,
                                  synth.log_periods(600.0, 3000.0, 64), np.asarray(pdots), 15, 10,
                                  np.zeros(2), np.zeros(2), np.zeros(2))
        got = gpu_grid(h, dev_args(b), mode)
        ref, dmin = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, 15,
                                            10, with_dmin=True)
        compare_grid(mode, got, ref, dmin)


def test_host_checks_raise(h):
    b = small_batch()
    args = dev_args(b)
    args["offsets"] = np.array([0, 200, 100, 600], dtype=np.int64)
    with pytest.raises(g.GceError):
        g.gce_ce_grid(h, cfg=g.Config(), **args)


@pytest.mark.parametrize("mode", MODES)
def test_deterministic_and_batch_invariant(h, mode):
    b = small_batch(seed=7, n_curves=5, pdots=(0.0, -5e-11))
    args = dev_args(b)
    a1 = gpu_grid(h, args, mode)
    a2 = gpu_grid(h, args, mode)
    assert np.array_equal(a1, a2)
    for c in (0, 3):
        one = b.subset([c])
        alone = gpu_grid(h, dev_args(one), mode)
        assert np.array_equal(alone[0], a1[c])


@pytest.mark.parametrize("use_graph", [True, False])
def test_graph_replay_with_new_inputs(h, use_graph):
    """Same shapes, different data and buffers: the captured graph is updated, not
    reused stale."""
    orc = oracle.Oracle()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for seed in (11, 12, 13):
            b = small_batch(seed=seed, pdots=(0.0, -1e-11))
            got = gpu_grid(h, dev_args(b), "fp64", use_graph=use_graph)
            ref = orc.ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, 15, 10)
            assert np.abs(got - ref).max() <= 1e-6


def test_graph_replay_sees_new_contents_in_place(h):
    """Same shape and the same device arrays, new contents written in place
    (including a new t0 and new curve lengths at the same total): the cached graph
    is replayed without a new capture and computes on the new contents."""
    orc = oracle.Oracle()
    s = torch.cuda.Stream()
    b0 = small_batch(seed=21, pdots=(0.0, -1e-11))
    args = dev_args(b0)
    out = torch.empty((b0.n_curves, b0.pdots.size, b0.periods.size), dtype=torch.float32,
                      device="cuda")
    with torch.cuda.stream(s):
        for seed, t0 in ((21, 0.0), (22, 0.0), (23, 0.0), (24, 0.0), (25, 3.0e7)):
            b = small_batch(seed=seed, pdots=(0.0, -1e-11))
            offs = b.offsets.copy()
            if seed == 24:  # other lengths, same total number of points
                offs[1:-1] += np.array([50, -30])
            args["times"].copy_(torch.tensor(b.times))
            args["mags"].copy_(torch.tensor(b.mags))
            args["offsets"] = offs
            cfg = g.Config(15, 10, "fp64", t0=t0)
            g.gce_ce_grid(h, cfg=cfg, out=out, stream=s, **args)
            assert g.gce_stream_status(h, s) == g.GCE_OK
            ref = orc.ce_grid(b.times, b.mags, offs, b.periods, b.pdots, 15, 10, t0=t0)
            assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6, seed


@pytest.mark.parametrize("mode", ["fp64", "fixed32"])
def test_host_entry_point_matches_device(h, mode):
    b = small_batch(seed=8, n_curves=4, pdots=(0.0, -2e-11))
    cfg = g.Config(15, 10, mode)
    dH, dI = g.gce_ce_topk(h, cfg=cfg, k=4, **dev_args(b))
    pin = lambda a: torch.tensor(a).pin_memory()
    hH, hI = g.gce_ce_topk_host(h, pin(b.times), pin(b.mags), b.offsets, pin(b.periods),
                                pin(b.pdots), cfg, 4)
    assert torch.equal(dH.cpu(), hH) and torch.equal(dI.cpu(), hI)
    # numpy (pageable) inputs work as well
    nH, nI = g.gce_ce_topk_host(h, b.times, b.mags, b.offsets, b.periods, b.pdots, cfg, 4)
    assert torch.equal(nH, hH) and torch.equal(nI, hI)


def test_autotune_keeps_results(h):
    b = small_batch(seed=9, n_curves=2, n_obs=500, n_periods=2000)
    cfg = g.Config(15, 10, "fixed32")
    before = gpu_grid(h, dev_args(b), "fixed32")
    g.gce_autotune(h, cfg, 500, 20000)
    t = g.gce_get_tuning(h, cfg, 500)
    assert t["block"] in (128, 256, 512) and t["tpt"] in (1, 2, 4)
    tp = g.gce_get_tuning(h, cfg, 500, n_pdots=8)  # tuned separately for a Pdot axis
    assert tp["block"] in (128, 256, 512) and tp["tpt"] in (1, 2, 4)
    after = gpu_grid(h, dev_args(b), "fixed32")
    assert np.array_equal(before, after)
    g.gce_set_tuning(h, cfg, 500, block=128, tpt=2, chunk=512)  # forces both entries
    assert g.gce_get_tuning(h, cfg, 500) == g.gce_get_tuning(h, cfg, 500, n_pdots=8)
    with pytest.raises(g.GceError):
        g.gce_get_tuning(h, cfg, 500, n_pdots=0)


@pytest.mark.parametrize("mode", MODES)
def test_topk_limits(h, mode):
    """k at its maximum (GCE_MAX_TOPK over several trial tiles) and k = every trial of
    a small grid: the device top-k is exactly the k smallest cells of the device grid,
    ties to the smaller flat index; larger k is refused before any launch."""
    for n_periods, pdots, k in ((700, (0.0, -1e-11), g.GCE_MAX_TOPK), (20, (0.0,), 20)):
        b = small_batch(seed=9, n_periods=n_periods, pdots=pdots)
        args = dev_args(b)
        cfg = g.Config(15, 10, mode)
        grid = gpu_grid(h, args, mode).reshape(b.n_curves, -1)
        for detect in (False, True):
            if detect:
                tH, tI, _, _, _ = g.gce_ce_detect(h, cfg=cfg, k=k, **args)
            else:
                tH, tI = g.gce_ce_topk(h, cfg=cfg, k=k, **args)
            assert g.gce_stream_status(h) == g.GCE_OK
            tH, tI = tH.cpu().numpy().astype(np.float64), tI.cpu().numpy()
            for c in range(b.n_curves):
                order = np.lexsort((np.arange(grid.shape[1]), grid[c]))[:k]
                assert np.array_equal(tI[c], order), (c, detect)
                assert np.array_equal(tH[c], grid[c, order])
        for bad in (min(k + 1, grid.shape[1] + 1), g.GCE_MAX_TOPK + 1):
            with pytest.raises(g.GceError):
                g.gce_ce_topk(h, cfg=cfg, k=bad, **args)


@pytest.mark.parametrize("mode", ["split32", "fixed32"])
def test_topk_two_level_merge(h, mode):
    """Grids with thousands of trial tiles per curve are merged in two levels (groups
    of tiles first, then the groups): the top-k is still exactly the k smallest cells
    of the device grid, and the merged moments match the grid's own statistics."""
    for n_periods, pdots, k in ((1_000_000, (0.0, -1e-11), 5), (200_000, (0.0, 2e-12), 64)):
        b = small_batch(seed=11, n_curves=3, n_obs=90, n_periods=n_periods, pdots=pdots)
        args = dev_args(b)
        cfg = g.Config(15, 10, mode)
        grid = gpu_grid(h, args, mode).reshape(b.n_curves, -1)
        tH, tI, mu, sd, rho = g.gce_ce_detect(h, cfg=cfg, k=k, **args)
        assert g.gce_stream_status(h) == g.GCE_OK
        rH, rI = g.gce_ce_topk(h, cfg=cfg, k=k, **args)
        assert torch.equal(tH, rH) and torch.equal(tI, rI)
        tH, tI = tH.cpu().numpy().astype(np.float64), tI.cpu().numpy()
        for c in range(b.n_curves):
            order = np.lexsort((np.arange(grid.shape[1]), grid[c]))[:k]
            assert np.array_equal(tI[c], order), c
            assert np.array_equal(tH[c], grid[c, order])
        gm, gs, gr = oracle.oracle_significance(grid.reshape(b.n_curves, 1, -1))
        mu, sd, rho = mu.cpu().numpy(), sd.cpu().numpy(), rho.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(mu - gm) <= 1e-6)
        assert np.all(np.abs(sd - gs) <= 1e-4 * gs)
        assert np.all(np.abs(rho - gr) <= 1e-3 * np.maximum(1.0, gr))


def test_launch_count():
    """gce_last_launches counts the kernels of the last call: checks, scan, trial
    constants, preparation, the CE kernel, then the top-k merge (two levels on
    grids with many tiles per curve); the c ln c table once per handle; one launch
    per curve for the single-launch baseline; nothing for an empty batch."""
    hh = g.Handle(0)
    try:
        b = small_batch(seed=12, n_curves=3, n_obs=120, n_periods=300)
        args = dev_args(b)
        cfg = g.Config(15, 10, "split32")
        g.gce_ce_topk(hh, cfg=cfg, k=5, **args)
        assert g.gce_last_launches(hh) == 7  # + the c ln c table, built by the first call
        g.gce_ce_topk(hh, cfg=cfg, k=5, **args)
        assert g.gce_last_launches(hh) == 6
        g.gce_ce_grid(hh, cfg=cfg, **args)
        assert g.gce_last_launches(hh) == 5
        g.gce_ce_grid_single(hh, cfg=g.Config(15, 10, "fp64"), **args)
        assert g.gce_last_launches(hh) == 4 + b.n_curves
        big = dev_args(small_batch(seed=12, n_curves=3, n_obs=120, n_periods=2_000_000))
        g.gce_ce_detect(hh, cfg=cfg, k=5, **big)
        assert g.gce_last_launches(hh) == 7  # the merge's first level over groups of tiles
        bands = torch.zeros(b.times.size, dtype=torch.uint8, device="cuda")
        g.gce_ce_grid_bands(hh, bands=bands, n_bands=1, cfg=cfg, **args)
        assert g.gce_last_launches(hh) == 6  # + the per-filter statistics
        empty = dict(args, offsets=np.zeros(1, dtype=np.int64))
        g.gce_ce_topk(hh, cfg=cfg, k=1, **empty)
        assert g.gce_last_launches(hh) == 0
        assert g.gce_stream_status(hh) == g.GCE_OK
    finally:
        hh.close()
