#!/usr/bin/env python
"""Benchmark of the CE (P, Pdot) search on GB300: folded point-trials per second.

Workload (default): 1000 light curves x 1000 observations (nightly cadence,
3-year baseline, detached eclipsing binaries), 1e5 log-spaced trial periods,
Pdot = 0, 15 phase x 10 magnitude bins, per-curve top-5.  One step is one full
search of that batch through the C ABI (input checks, trial constants,
per-curve preparation, the persistent CE kernel, the top-k merge), with inputs
resident on the device; `e2e` repeats it through gce_ce_topk_host with host
buffers, copies included.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gce|reference]
Under torchrun each rank searches its own copy of the batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "folded point-trials/s (N_obs×N_P×N_Ṗ) on 1 GB300; FP64 vs split-FP32 phase"
UNIT = "point-trials/s"
# Roofline of k_main.  The FP32 folds are bound by instruction issue (ncu: issue
# slots ~82 % busy, no pipe above ~60 %): the peak is 4 schedulers x 32 lanes =
# 128 thread-instructions per clock per SM, and the algorithmic work is the
# instructions a thread-per-trial fold cannot avoid per point-trial -- the
# fold's arithmetic, one slot address and one shared-memory increment:
#   split32: 6 FP32 operations (rounding FMA, subtract, residual FMA, two cross
#            FMAs, bin FMA); with Pdot 15 (the Pdot product reduced the same
#            way, two more cross FMAs, the sum reduced once more);
#   fixed32: multiply-add, multiply-high, cross FMA, add, bin multiply-high;
#            with Pdot 8 (two more integer products, one more cross FMA).
# The FP64 fold is bound by the FP64 pipe (2 lanes/clk/SM): 5 FP64 operations
# (mul, floor, sub, mul, convert), 7 with Pdot (mul, FMA).
FOLD_OPS = {"split32": (6, 15), "fixed32": (5, 8), "fp64": (5, 7)}
ISSUE_LANES = 128
FP32_LANES = 128
FP64_LANES = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gce", choices=["gce", "reference"])
    ap.add_argument("--mode", default="split32", choices=["split32", "fixed32", "fp64"])
    ap.add_argument("--workload", type=int, default=1, help="synthetic workload index (0..5)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 / SPLIT32 / one-launch-per-curve comparison legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU seconds of the oracle baseline sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="total oracle seconds of the reference arm (spread over its steps)")
    ap.add_argument("--curves", type=int, default=0,
                    help="use only the first N curves of the workload (profiling runs)")
    ap.add_argument("--phase-bins", type=int, default=0,
                    help="override the workload's phase-bin count (0 = the workload's)")
    ap.add_argument("--overlap", action="store_true",
                    help="50%%-overlapping phase bins (the paper's 50-bin production setting)")
    ap.add_argument("--bands", type=int, default=0,
                    help="multi-filter input: give every point one of N filters (seeded) and "
                         "search through gce_ce_detect_bands (0 = single filter)")
    ap.add_argument("--pdots", type=int, default=0,
                    help="override the Pdot-axis length of workloads 2, 4 and 5 (Sec. 3 runs "
                         "32, 128 and 512; 0 = the workload's)")
    ap.add_argument("--shape", default="",
                    help="block,tpt,chunk[,slot_range]: fixed launch shape instead of autotuning "
                         "(profiling runs)")
    return ap.parse_args()


def profiled_traffic(mode, workload, n_curves):
    """DRAM bytes per full launch of k_main recorded under profiles/ for the batch
    workload, or None when the kernel sources changed since that capture (their
    hash no longer matches) or the run is not that workload."""
    prof = os.path.join(ROOT, "profiles", f"k_main_{mode}_batch_100curves.md")
    if workload != 1 or n_curves != 1000 or not os.path.exists(prof):
        return None
    rec = {}
    for line in open(prof):
        if ":" in line and line.split(":")[0] in ("traffic_bytes_full_launch",
                                                  "kernel_sources_sha256_16"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel_sources_sha256_16") != kernel_code_hash():
        return None
    return int(rec["traffic_bytes_full_launch"]) if "traffic_bytes_full_launch" in rec else None


def kernel_code_hash():
    """SHA-256 (first 16 hex digits) of the CE kernel's sources with comments and
    blank lines removed, so that a comment-only edit keeps a capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("gce_kernel.cuh", "gce_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2006_06866_gb300", "csrc", f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = line.split("//", 1)[0].rstrip()
            if line.strip():
                h.update((line + "\n").encode())
    return h.hexdigest()[:16]


def workload_overrides(args):
    """Keyword overrides of synth.make_config from the command line."""
    if not args.pdots:
        return {}
    if args.workload not in (2, 4, 5):
        raise SystemExit("--pdots applies to workloads 2, 4 and 5 (the ones with a Pdot axis)")
    return {"n_pdots": int(args.pdots)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ---------------------------------------------------------------- oracle leg

def _oracle_sample(batch, pt_want, min_curves):
    """The first curves of the workload x a strided subset of its periods x all
    its Pdot values, holding about pt_want point-trials."""
    n_obs = float(np.mean(batch.n_obs))
    per_curve = n_obs * batch.periods.size * batch.pdots.size
    n_curves = int(min(batch.n_curves, max(min_curves, int(np.ceil(pt_want / per_curve)))))
    n_periods = int(min(batch.periods.size,
                        max(64, pt_want / (n_curves * n_obs * batch.pdots.size))))
    stride = max(1, batch.periods.size // n_periods)
    return batch.subset(list(range(n_curves)), periods=batch.periods[::stride]), stride


def _describe(sample, batch, stride, dt, threads):
    which = "all" if stride == 1 else f"a stride-{stride} subset"
    return (f"first {sample.n_curves} curves x {sample.periods.size} periods ({which} of "
            f"{batch.periods.size}) x {sample.pdots.size} Pdot = {sample.point_trials:.3g} "
            f"point-trials in {dt:.2f} s on {threads} thread{'s' if threads > 1 else ''}")


def oracle_rate(batch, seconds, n_threads=0, overlap=False, keep=False, single=True):
    """The CPU oracle on bounded samples of the workload: one thread for about a
    fifth of `seconds` (at most 4 s), then all `n_threads` threads for about
    `seconds`.  The oracle splits its grid into (curve, Pdot, run of 64
    periods) rows, so a sample of a few curves still keeps every thread busy.
    Returns a dict (point-trials/s on all threads and on one, the threads used,
    the samples) and, with keep, the all-thread sample with its oracle grid and
    edge distances (the parity block reuses them)."""
    import oracle
    orc = oracle.Oracle()
    threads = n_threads or os.cpu_count() or 1

    def run(sample, nt):
        t0 = time.perf_counter()
        out = orc.ce_grid(sample.times, sample.mags, sample.offsets, sample.periods, sample.pdots,
                          batch.n_phase, batch.n_mag, t0=batch.t0, n_threads=nt, with_dmin=True,
                          overlap=overlap)
        return out, time.perf_counter() - t0

    # calibration: one curve x about 200 periods on one thread
    cal = batch.subset([0], periods=batch.periods[:: max(1, batch.periods.size // 200)],
                       pdots=batch.pdots[:1])
    _, dt = run(cal, 1)
    rate1 = cal.point_trials / max(dt, 1e-4)
    res = {}
    if single:
        one, s1 = _oracle_sample(batch, rate1 * min(4.0, max(0.5, seconds / 5)), 1)
        _, dt1 = run(one, 1)
        rate1 = one.point_trials / dt1
        res = {"single_thread_value": rate1,
               "single_thread_sample": _describe(one, batch, s1, dt1, 1)}
    sample, stride = _oracle_sample(batch, rate1 * threads * seconds, 1)
    (ref, dmin), dt = run(sample, threads)
    used = orc.threads_used
    res = {"value": sample.point_trials / dt, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": _describe(sample, batch, stride, dt, used), **res}
    return (res, (sample, ref, dmin)) if keep else (res, None)


def oracle_c1_full(n_threads):
    """The small single-curve configuration (workload 0: one 100-point curve x
    1000 periods, 15 x 10 bins) in full on the oracle: median of five runs."""
    import oracle
    import synth
    orc = oracle.Oracle()
    b = synth.make_config(0)
    out = {}
    for nt, key in ((1, "single_thread_s"), (n_threads, "all_threads_s")):
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            orc.ce_grid(b.times, b.mags, b.offsets, b.periods, b.pdots, b.n_phase, b.n_mag,
                        n_threads=nt)
            ts.append(time.perf_counter() - t0)
        out[key] = float(np.median(ts))
    out["point_trials"] = int(b.point_trials)
    out["threads"] = int(n_threads)
    return out


# Parity contract of the GPU folds against the oracle: |dH| bound per fold, and
# the fold's phase-error bound eps in cycles (cells whose points all lie farther
# than 4 eps from a phase-bin edge are held to the |dH| bound; 0 = every cell).
PARITY_TOL = {"fp64": 1e-6, "split32": 1e-4, "fixed32": 1e-4}
PARITY_EPS = {"fp64": 0.0, "split32": 2.5e-7, "fixed32": 4e-9}


def parity_block(g, h, dev, stream, sample, ref, dmin, overlap, n_count_cells=2000):
    """Per fold: CE error and argmin agreement of the device grid against the
    oracle grid of the CPU-baseline sample, and exact-count agreement on seeded
    sampled cells (gce_ce_counts against the oracle's counts)."""
    import torch
    nc = sample.n_curves
    flat, dm = ref.reshape(nc, -1), dmin.reshape(nc, -1)
    args = dict(times=torch.tensor(sample.times, device=dev),
                mags=torch.tensor(sample.mags, device=dev),
                offsets=np.asarray(sample.offsets, dtype=np.int64),
                periods=torch.tensor(sample.periods, device=dev),
                pdots=torch.tensor(sample.pdots, device=dev))
    rng = np.random.default_rng(20200611)
    n_trials = flat.shape[1]
    cc = rng.integers(0, nc, size=n_count_cells).astype(np.int64)
    ct = rng.integers(0, n_trials, size=n_count_cells).astype(np.int64)
    import oracle
    _, cdmin, rcounts = oracle.Oracle().ce_cells(
        sample.times, sample.mags, sample.offsets, sample.periods, sample.pdots, sample.n_phase,
        sample.n_mag, cc, ct, t0=sample.t0, with_counts=True, overlap=overlap)
    # the oracle's best and runner-up cell per curve (ties: the smaller flat index)
    best = flat.argmin(axis=1)
    masked = flat.copy()
    masked[np.arange(nc), best] = np.inf
    second = masked.argmin(axis=1) if flat.shape[1] > 1 else best
    del masked
    out = {"cells": int(flat.size), "curves": nc, "count_cells": n_count_cells}
    with torch.cuda.stream(stream):
        for mode in ("fp64", "split32", "fixed32"):
            cfg = g.Config(sample.n_phase, sample.n_mag, mode, t0=sample.t0, overlap=overlap)
            got = g.gce_ce_grid(h, cfg=cfg, stream=stream, **args)
            cnt = g.gce_ce_counts(h, cfg=cfg, cell_curve=torch.tensor(cc, device=dev),
                                  cell_trial=torch.tensor(ct, device=dev), stream=stream, **args)
            if g.gce_stream_status(h, stream) != g.GCE_OK:
                out[mode] = {"error": "device input check failed"}
                continue
            got = got.cpu().numpy().astype(np.float64).reshape(nc, -1)
            cnt = cnt.cpu().numpy().astype(np.int64)
            err = np.abs(got - flat)
            near = dm <= 4 * PARITY_EPS[mode]
            agree = ambiguous = 0
            dev_best = got.argmin(axis=1)  # first occurrence: ties to the smaller index
            for c in range(nc):
                b, s2 = best[c], second[c]
                if (s2 != b and flat[c, s2] - flat[c, b] <= 1e-4) or near[c, b]:
                    ambiguous += 1
                    continue
                agree += int(dev_best[c] == b)
            cfar = cdmin > 4 * PARITY_EPS[mode]
            same = np.all(cnt == rcounts, axis=(1, 2))
            out[mode] = {
                "tol": PARITY_TOL[mode], "eps_cycles": PARITY_EPS[mode],
                "max_abs_dH": float(err.max()),
                "max_abs_dH_off_edge": float(err[~near].max()) if (~near).any() else 0.0,
                "near_edge_frac": float(near.mean()),
                "argmin_agree": agree, "argmin_decided": nc - ambiguous,
                "argmin_tie_ambiguous": ambiguous,
                "counts_exact": int(same.sum()), "counts_exact_off_edge": int(same[cfar].sum()),
                "count_cells_off_edge": int(cfar.sum()),
                "pass": bool(err[~near].max() <= PARITY_TOL[mode] if (~near).any() else True)
                and agree == nc - ambiguous
                and (mode != "fp64" or bool(same.all())),
            }
    return out


def run_reference(args, rank, world):
    """The oracle as the reference arm: timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    import synth
    batch = synth.make_config(args.workload, **workload_overrides(args))
    if args.phase_bins:
        batch.n_phase = int(args.phase_bins)
    per_step = max(0.5, args.ref_seconds / max(1, args.steps + args.warmup))
    threads = os.cpu_count() or 1
    rates = []
    info = single = None
    for s in range(args.warmup + args.steps):
        info, _ = oracle_rate(batch, per_step, n_threads=threads, overlap=bool(args.overlap),
                              single=single is None)
        if single is None:  # the one-thread rate, measured once
            single = {k: v for k, v in info.items() if k.startswith("single_thread")}
        if s >= args.warmup:
            rates.append(info["value"])
    value = float(np.median(rates))
    cpu = dict(info, value=value, **single)
    cpu["sample"] = f"median over {len(rates)} steps, each {info['sample']}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{synth.CONFIG_NAMES[args.workload]}: {batch.n_curves} curves, "
                               f"{batch.periods.size} periods x {batch.pdots.size} Pdot, "
                               f"{batch.n_phase}x{batch.n_mag} bins"
                               + (", 50 % overlapping" if args.overlap else ""),
                   "cpu": cpu_model()},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = subprocess.Popen(
            ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
             "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.tmp,
            stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.tmp.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def query_max_sm_mhz(device_index):
    """The device's maximum SM clock from nvidia-smi (MHz), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(device_index),
                              "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=30).stdout
        return float(out.strip().splitlines()[0])
    except Exception:
        return None


# ---------------------------------------------------------------- GPU leg

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    import paper_2006_06866_gb300 as g
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    batch = synth.make_config(args.workload, **workload_overrides(args))
    if args.curves:
        batch = batch.subset(list(range(min(args.curves, batch.n_curves))))
    if world > 1:
        # weak scaling: the global batch is the workload once per rank; each rank
        # searches its own shard of it (balanced by points), no data-path collective
        from paper_2006_06866_gb300.sharding import shard_arrays, shard_curves
        n = batch.n_curves
        glob = batch.subset(list(range(n)) * world)
        mine = shard_curves(glob.n_obs, world)[rank]
        t_s, m_s, o_s = shard_arrays(glob.times, glob.mags, glob.offsets, mine)
        batch = synth.LightCurveBatch(batch.name, t_s, m_s, o_s, batch.periods, batch.pdots,
                                      batch.n_phase, batch.n_mag, glob.truth_p0[mine],
                                      glob.truth_pdot[mine], glob.truth_class[mine], batch.t0,
                                      batch.topk)
    if args.phase_bins:
        batch.n_phase = int(args.phase_bins)
    ovl = bool(args.overlap)
    k = batch.topk or 5
    pt_step = batch.point_trials
    t_d = torch.tensor(batch.times, device=dev)
    m_d = torch.tensor(batch.mags, device=dev)
    p_d = torch.tensor(batch.periods, device=dev)
    q_d = torch.tensor(batch.pdots, device=dev)
    offs = np.asarray(batch.offsets, dtype=np.int64)
    h = g.Handle(local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    out_H = torch.empty((batch.n_curves, k), dtype=torch.float32, device=dev)
    out_I = torch.empty((batch.n_curves, k), dtype=torch.int64, device=dev)

    nb = int(args.bands)
    bands_h = (np.random.default_rng(20200611 + 100 * args.workload + nb)
               .integers(0, nb, size=batch.times.size).astype(np.uint8) if nb else None)
    b_d = torch.tensor(bands_h, device=dev) if nb else None

    def step(mode, time_kernel=False):
        cfg = g.Config(batch.n_phase, batch.n_mag, mode, t0=batch.t0, time_kernel=time_kernel,
                       overlap=ovl)
        if nb:
            g.gce_ce_detect_bands(h, t_d, m_d, b_d, nb, offs, p_d, q_d, cfg, k,
                                  significance=False, stream=stream)
        else:
            g.gce_ce_topk(h, t_d, m_d, offs, p_d, q_d, cfg, k, out_H, out_I, stream=stream)

    tuned = {}
    launches = {}
    host_ms = {}  # mean host time of one step's call (argument checks, planning, enqueue)

    def timed_steps(mode, warmup, steps, with_kernel=False):
        if mode not in tuned:  # launch-shape autotuning is part of the untimed warm-up
            cfg = g.Config(batch.n_phase, batch.n_mag, mode, t0=batch.t0, overlap=ovl)
            if args.shape:
                sh = [int(x) for x in args.shape.split(",")]
                g.gce_set_tuning(h, cfg, int(batch.n_obs.max()), block=sh[0], tpt=sh[1], chunk=sh[2],
                                 slot_range=sh[3] if len(sh) > 3 else 0)
            else:  # tuned on a bounded slice of this very job
                g.gce_autotune_job(h, t_d, m_d, offs, p_d, q_d, cfg)
            tuned[mode] = g.gce_get_tuning(h, cfg, int(batch.n_obs.max()), int(batch.pdots.size))
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step(mode)
            stream.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
            kern = []
            host = []
            barrier()
            torch.cuda.synchronize()
            wall0 = time.perf_counter()
            for i in range(steps):
                flush.zero_()
                evs[i][0].record(stream)
                h0 = time.perf_counter()
                step(mode, time_kernel=with_kernel)
                host.append(time.perf_counter() - h0)
                evs[i][1].record(stream)
                if with_kernel:
                    kern.append(g.gce_kernel_time(h))
            stream.synchronize()
            barrier()
            torch.cuda.synchronize()
            wall = time.perf_counter() - wall0
        launches[mode] = g.gce_last_launches(h) * steps  # every timed step runs the same graph
        st = g.gce_stream_status(h, stream)
        if st != g.GCE_OK:
            raise RuntimeError(f"device input check failed: status {st}")
        ms = sum(a.elapsed_time(b) for a, b in evs)
        host_ms[mode] = 1e3 * float(np.mean(host))
        return ms, wall, kern

    # ---- headline: the batched persistent kernel in the headline fold mode
    sampler = ClockSampler(local)
    sampler.start()
    ms, wall, kern = timed_steps(args.mode, args.warmup, args.steps, with_kernel=True)
    clocks = sampler.stop()
    t_rank = ms / 1e3
    if pg is not None:
        tt = torch.tensor([t_rank], device=dev, dtype=torch.float64)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_rank = float(tt.item())
    value = pt_step * args.steps * world / t_rank
    ms_per_step = t_rank * 1e3 / args.steps
    kern_ms = float(np.mean(kern)) if kern else None

    # ---- end to end through the host-buffer entry point (pinned host memory)
    pin = lambda a: torch.tensor(a).pin_memory()
    ht, hm, hp, hq = pin(batch.times), pin(batch.mags), pin(batch.periods), pin(batch.pdots)
    hH = torch.empty((batch.n_curves, k), dtype=torch.float32).pin_memory()
    hI = torch.empty((batch.n_curves, k), dtype=torch.int64).pin_memory()
    cfg = g.Config(batch.n_phase, batch.n_mag, args.mode, t0=batch.t0, overlap=ovl)
    hb = pin(bands_h) if nb else None

    def e2e_step():
        if not nb:
            g.gce_ce_topk_host(h, ht, hm, offs, hp, hq, cfg, k, hH, hI, stream=stream)
            return
        # multi-filter input has no host-buffer entry point: the same copies, by hand
        dt, dm, db, dp, dq = (x.to(dev, non_blocking=True) for x in (ht, hm, hb, hp, hq))
        tH_, tI_, _, _, _ = g.gce_ce_detect_bands(h, dt, dm, db, nb, offs, dp, dq, cfg, k,
                                                  significance=False, stream=stream)
        hH.copy_(tH_, non_blocking=True)
        hI.copy_(tI_, non_blocking=True)
        stream.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        e2e_t = 0.0
        for _ in range(args.steps):
            flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            e2e_t += time.perf_counter() - t0
    if pg is not None:
        tt = torch.tensor([e2e_t], device=dev, dtype=torch.float64)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        e2e_t = float(tt.item())
    h2d = 8 * (batch.times.size + batch.mags.size + batch.periods.size + batch.pdots.size) + (
        batch.times.size if nb else 0)
    d2h = (4 + 8) * batch.n_curves * k

    extras = {}
    # rough rates (point-trials/s) used only to skip comparison legs longer than a minute
    est_rate = {"split32": 1e12, "fixed32": 8e11, "fp64": 1e11}
    if rank == 0 and world == 1 and not args.no_extras:
        for mode, n in (("split32", 2), ("fixed32", 2), ("fp64", 1)):
            if mode == args.mode:
                continue
            if pt_step * n / est_rate[mode] > 60.0:
                extras[mode] = {"skipped": "one step would take more than a minute"}
                continue
            ms_m, _, kern_m = timed_steps(mode, 1, n, with_kernel=True)
            extras[mode] = {"value": pt_step * n / (ms_m / 1e3), "ms_per_step": ms_m / n,
                            "kernel_ms": float(np.mean(kern_m))}
        # the plain FP64 one-launch-per-curve kernel (speedup denominator)
        grid_bytes = 4 * batch.n_curves * batch.pdots.size * batch.periods.size
        if pt_step / 6e10 > 60.0 or grid_bytes > 8e9:
            extras["fp64_single_launch"] = {"skipped": "one step would take more than a minute"}
        else:
            cfg64 = g.Config(batch.n_phase, batch.n_mag, "fp64", t0=batch.t0, time_kernel=True,
                             overlap=ovl)
            with torch.cuda.stream(stream):
                out = torch.empty((batch.n_curves, batch.pdots.size, batch.periods.size),
                                  dtype=torch.float32, device=dev)
                g.gce_ce_grid_single(h, t_d, m_d, offs, p_d, q_d, cfg64, out=out, stream=stream)
                stream.synchronize()
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.gce_ce_grid_single(h, t_d, m_d, offs, p_d, q_d, cfg64, out=out, stream=stream)
                e1.record(stream)
                stream.synchronize()
                del out
            ms_single = e0.elapsed_time(e1)
            extras["fp64_single_launch"] = {"value": pt_step / (ms_single / 1e3),
                                            "ms_per_step": ms_single}
            extras["speedup_vs_fp64_single_launch"] = (
                value / world / extras["fp64_single_launch"]["value"])

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            threads = os.cpu_count() or 1
            cpu, kept = oracle_rate(batch, args.cpu_seconds, n_threads=threads, overlap=ovl,
                                    keep=not nb)
            cpu["cpu"] = cpu_model()
            cpu["plain_single_curve_full"] = oracle_c1_full(threads)
        except Exception as e:  # the baseline is context; never fail the bench on it
            cpu = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                   "sample": f"unavailable: {e}"}
            kept = None
        if kept is not None:
            # per-fold CE error and argmin agreement against the oracle, on the
            # grid the oracle has just computed for the baseline
            parity = parity_block(g, h, dev, stream, *kept, overlap=ovl)
            parity["sample"] = cpu["sample"]

    roof = None
    if kern_ms:
        has_pdot = bool(np.any(batch.pdots != 0.0))
        fold = FOLD_OPS[args.mode][1 if has_pdot else 0]
        rate = pt_step / (kern_ms / 1e3)
        # the peak's SM count and maximum SM clock are the device's own: the SM
        # count from the device properties, the clock from the sampler (the
        # maximum nvidia-smi reports while the timed steps ran)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_max = clocks.get("sm_max_mhz") or query_max_sm_mhz(local)
        clk = n_sm * sm_max * 1e6
        if args.mode == "fp64":
            ops, lanes, pipe = fold, FP64_LANES, "FP64 pipe"
        else:
            ops, lanes = fold + 2, ISSUE_LANES
            pipe = "issue slots (fold arithmetic + slot address + shared increment)"
        achieved = ops * rate / 1e9
        peak = lanes * clk / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(args.mode, args.workload, batch.n_curves),
                "kernel": "k_main", "kernel_ms": kern_ms, "kernel_point_trials_per_s": rate,
                "pipe": pipe,
                "peak_basis": f"{n_sm} SMs x {lanes} lanes/clk x {sm_max:.0f} MHz",
                "sm_count": n_sm, "sm_max_mhz": sm_max,
                "sm_count_from": "torch.cuda.get_device_properties().multi_processor_count",
                "sm_max_mhz_from": "nvidia-smi clocks.max.sm, sampled during the timed steps"
                if clocks.get("sm_max_mhz") else "nvidia-smi clocks.max.sm, queried once",
                "ops_per_point_trial": ops}
        if args.mode == "split32":
            roof["fp32_pipe_frac"] = fold * rate / (FP32_LANES * clk)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fixed32": "u32", "split32": "f32", "fp64": "f64"}[args.mode],
            "data": "synthetic",
            "config": {"workload": f"{synth.CONFIG_NAMES[args.workload]}: {batch.n_curves} curves "
                                   f"x {int(batch.n_obs.mean())} obs, {batch.periods.size} periods "
                                   f"x {batch.pdots.size} Pdot, {batch.n_phase}x{batch.n_mag} "
                                   f"bins, top-{k}",
                       "phase_mode": args.mode, "point_trials_per_step": pt_step,
                       "launch_shape": tuned.get(args.mode),
                       "l2": "256 MB buffer written between timed steps",
                       "parallelism": f"replica per GPU x{world}",
                       **({"filters": f"{nb} (seeded filter index per point; per-filter "
                                      "median/std normalisation)"} if nb else {}),
                       **({"phase_bins": "50 % overlapping"} if ovl else {})},
            "e2e": {"value": pt_step * args.steps * world / e2e_t, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches[args.mode],
            "host_call_ms": host_ms.get(args.mode),
            "clocks": clocks,
            "roofline": roof,
            "cpu_baseline": cpu,
            "parity": parity,
            "modes": extras,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
