"""Multi-rank partition of the search on CPU: a world-size-2 gloo run where each
rank searches its shard with the oracle; the gathered shards equal the full
search.  No collective touches the data path except this test's check."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2006_06866_gb300.sharding import shard_arrays, shard_curves


def test_shards_cover_once_and_balance():
    rng = np.random.default_rng(0)
    n_obs = rng.integers(50, 2000, size=1001)
    for world in (1, 2, 3, 8):
        shards = shard_curves(n_obs, world)
        allc = np.sort(np.concatenate(shards))
        assert np.array_equal(allc, np.arange(n_obs.size))
        loads = [int(n_obs[s].sum()) for s in shards]
        assert max(loads) - min(loads) <= n_obs.max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = synth.make_config(3, n_curves=9, n_periods=40)
    shards = shard_curves(b.n_obs, world)
    t, m, offs = shard_arrays(b.times, b.mags, b.offsets, shards[rank])
    grid = oracle.Oracle().ce_grid(t, m, offs, b.periods, b.pdots, b.n_phase, b.n_mag,
                                   n_threads=1)
    out = [None] * world
    dist.all_gather_object(out, (shards[rank].tolist(), grid))
    if rank == 0:
        full = oracle.Oracle().ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots,
                                       b.n_phase, b.n_mag, n_threads=1)
        merged = np.empty_like(full)
        for curves, g in out:
            merged[curves] = g
        q.put(bool(np.array_equal(merged, full)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_search_equals_full():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=10) is True
