"""Throughput of the two-grid MLQMC level evaluation on one GB300 (or N, one process per GPU).

A step is one pass of the whole hot path over one batch of synthetic input: every level of the
workload, every shift, every lattice point -- lattice points, centroid coefficients, coarse
eigensolves, fine shifted solves, Rayleigh quotients, level differences and per-shift sums.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision fp64|mixed]
    python bench.py --impl reference ...     # the FP64 CPU oracle on a bounded sample

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic_inputs import WORKLOADS, shared_shifts, shifts, shifts_for_rank  # noqa: E402

METRIC = "two-grid eigen-samples/s at rel. err<=1e-10 vs FP64 oracle; mixed vs plain GPU"
# the largest workload that fits one GPU: six levels, meshes 1/32 .. 1/1024, 516,096 samples
DEFAULT_WORKLOAD = "mlqmc6_h32_1024"
# One step evaluates the fraction 1/F of every level's lattice points (all shifts): step i takes the
# window i mod F of each level, so F consecutive steps cover the whole workload once.  The six-level
# workload takes tens of seconds per full pass; 1/32 of it keeps a bench run within minutes while
# every level still streams at full occupancy (its finest level: 16 points x 16 shifts of 1,046,529
# unknowns per step).
STEP_FRACTION = {"mlqmc6_h32_1024": 32}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-baseline", action="store_true", help="skip the timed CPU oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-graph", action="store_true", help="skip the graph-schedule run")
    ap.add_argument("--baseline-seconds", type=float, default=20.0)
    ap.add_argument("--fraction", type=int, default=0,
                    help="evaluate 1/F of every level's points per step (0: the workload's default)")
    ap.add_argument("--schedule", default="graph", choices=["graph", "concurrent", "sequential"],
                    help="graph: every step one replay of one CUDA graph holding all levels' windows (the "
                         "headline; one process); sequential: levels one after another through the host "
                         "API; concurrent: all levels at once on their own streams (mq_eval_levels_device). "
                         "The sequential run always times the per-kernel rooflines")
    return ap.parse_args()


def max_over_ranks(ms, world, device="cuda"):
    """The slowest rank's time: the whole job ends when its last rank does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(samples_per_rank, world, steps, ms):
    """Samples per second of all ranks together (weak scaling: every rank evaluates its own
    shifts of the full workload)."""
    return samples_per_rank * world * steps / (ms / 1e3)


def fine_dof_solves(wl):
    """Fine unknowns solved per step: every sample of level l solves on mesh h_l and, for l > 0, on
    h_{l-1} (direct levels count their eigensolve's unknowns once)."""
    tot = 0
    for l, lv in enumerate(wl.levels):
        per = (lv.n_fine - 1) ** 2
        if l > 0:
            per += (wl.levels[l - 1].n_fine - 1) ** 2
        tot += lv.N * lv.R * per
    return tot


def gather_rank_sums(level_sums, world):
    """All ranks' per-level shift sums, shifts of rank 0 first: [level][R * world] (one exchange of
    (L+1) x R doubles per rank at the end; nothing on the data path)."""
    if world <= 1:
        return [np.asarray(x, dtype=np.float64) for x in level_sums]
    import torch
    import torch.distributed as dist

    flat = torch.tensor(np.concatenate(level_sums), dtype=torch.float64)
    if dist.get_backend() == "nccl":
        flat = flat.cuda()
    parts = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(parts, flat)
    parts = [p.cpu().numpy() for p in parts]
    out, off = [], 0
    for x in level_sums:
        out.append(np.concatenate([p[off:off + len(x)] for p in parts]))
        off += len(x)
    return out


def merged_estimate(binding, level_sums, npoints, world, shared=False):
    """The workload's estimate from every rank's shifts (mq_estimate_sums over R * world shifts)."""
    allsums = gather_rank_sums(level_sums, world)
    m, se, lm, lv = binding.mq_estimate_sums(allsums, npoints, shared)
    return {"mean": m, "std_err": se, "level_mean": list(lm), "level_var": list(lv),
            "shifts_per_level": [len(x) for x in allsums], "points_per_shift": list(npoints),
            "ranks": world}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.reasons = set()
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        q = ("index,clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                f = [x.strip() for x in out.stdout.strip().split(",")]
                if len(f) >= 8:
                    self.samples.append((float(f[1]), float(f[2])))
                    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                    for nm, v in zip(names, f[4:8]):
                        if v.lower().startswith("active"):
                            self.reasons.add(nm)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": sorted(self.reasons), "samples": 0}
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples), "reasons": sorted(self.reasons),
                "samples": len(self.samples)}


# ------------------------------------------------------------------------------------------
def setup_context(binding, wl, stream_ptr, prec, rank=0, world=1):
    """A context on the workload; with several ranks, this rank's share of the workload's shifts.
    The reuse workload (shared shifts) uses one embedded lattice and the library's reuse scheme."""
    ctx = binding.Context(0, stream_ptr)
    if wl.family == 2:
        ctx.mq_set_islands(max(lv.s for lv in wl.levels), *wl.decays)
    else:
        ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(wl.levels)
    shared = wl.extra.get("shared", False)
    if shared:
        z = binding.mq_cbc_embedded_lattice(wl.extra["m_min"], wl.extra["m_max"], max(lv.s for lv in wl.levels),
                                            wl.decay)
        zs = [z[: lv.s] for lv in wl.levels]
        ds = shared_shifts(wl.seed, wl.levels, rank, world)
    else:
        zs = [binding.mq_cbc_lattice(lv.N, lv.s, wl.decay) for lv in wl.levels]
        ds = shifts_for_rank(wl.seed, wl.levels, rank, world)
    for l in range(len(wl.levels)):
        if shared:
            ctx.mq_set_lattice_embedded(l, zs[l], wl.extra["m_max"])
        else:
            ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(binding.MQ_PREC_MIXED if prec == "mixed" else binding.MQ_PREC_FP64)
    if shared:
        ctx.mq_set_reuse(1)
    return ctx, zs, ds


def step_fraction(wl, args):
    return args.fraction if args.fraction > 0 else STEP_FRACTION.get(wl.name, 1)


def windows(wl, F, step):
    """Point range [k0, k1) of every level in step `step`: window step mod F of 1/F of the points."""
    out = []
    for lv in wl.levels:
        n = max(1, lv.N // F)
        w = step % max(1, lv.N // n)
        out.append((w * n, w * n + n))
    return out


def step_samples(wl, F):
    return sum(lv.R * (k1 - k0) for lv, (k0, k1) in zip(wl.levels, windows(wl, F, 0)))


def run_device_step(ctx, wl, outs, sums, F, step, sequential=True):
    if sequential:
        for l, (k0, k1) in enumerate(windows(wl, F, step)):
            ctx.mq_eval_level_device(l, k0, k1, outs[l], sums[l])
    else:  # all levels at once, each on its own stream (the library's concurrent schedule)
        ctx.mq_eval_levels_device(list(range(len(wl.levels))), outs, sums)


def time_device(binding, torch, wl, prec, steps, warmup, stream, F, rank=0, world=1, sequential=True):
    if not sequential and F != 1:
        raise SystemExit("the concurrent schedule evaluates whole levels: use --fraction 1")
    ctx, zs, ds = setup_context(binding, wl, stream.cuda_stream, prec, rank, world)
    win = windows(wl, F, 0)
    outs = [torch.empty((lv.R, k1 - k0, 4), dtype=torch.float64, device="cuda") for lv, (k0, k1) in zip(wl.levels, win)]
    sums = [torch.empty(lv.R, dtype=torch.float64, device="cuda") for lv in wl.levels]
    for i in range(warmup):
        run_device_step(ctx, wl, outs, sums, F, i, sequential)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ctx.mq_reset_sums()  # also clears the per-level device timers
    ctx.mq_set_kernel_probe(1)  # live timing of the streaming operator sweep over the timed steps
    ev0.record(stream)
    for i in range(steps):
        run_device_step(ctx, wl, outs, sums, F, warmup + i, sequential)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    probe = ctx.mq_get_kernel_probe()
    ctx.mq_set_kernel_probe(0)
    # per-level device time of the timed region (CUDA events on the launching stream)
    timing = [ctx.mq_get_level_timing(l) + ctx.mq_get_kernel_timing(l) for l in range(len(wl.levels))]
    launches = ctx.mq_get_launch_count()
    level_sums = [ctx.mq_get_sums(l) for l in range(len(wl.levels))]  # estimator state of the timed steps
    last = [o.cpu().numpy() for o in outs]  # per-sample results of the last timed step
    # iteration counts from one more (untimed) pass over the last step's windows
    kstats = {}
    for l, (k0, k1) in enumerate(windows(wl, F, warmup + steps - 1)):
        ctx.mq_eval_level_device(l, k0, k1, outs[l], sums[l])
        kstats[l] = [ctx.mq_get_stats()]
    return ctx, ms, timing, kstats, last, launches, level_sums, probe


def time_graph(binding, torch, wl, prec, steps, warmup, stream, F, ref_outs):
    """The graph schedule: the windows of every level captured once as one CUDA graph
    (mq_graph_capture), replayed once per step on that step's windows (mq_graph_launch with the new
    start points): one graph launch per step, no host reads inside it."""
    ctx, zs, ds = setup_context(binding, wl, stream.cuda_stream, prec)
    win = windows(wl, F, 0)
    outs = [torch.empty((lv.R, k1 - k0, 4), dtype=torch.float64, device="cuda") for lv, (k0, k1) in zip(wl.levels, win)]
    ranges = [(l, k0, k1) for l, (k0, k1) in enumerate(win)]
    t0 = time.perf_counter()
    ctx.mq_graph_capture(ranges, outs, None)
    capture_s = time.perf_counter() - t0
    _, nodes = ctx.mq_get_graph_info()
    for i in range(warmup):
        ctx.mq_graph_launch([k0 for k0, _ in windows(wl, F, i)])
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(steps):
        ctx.mq_graph_launch([k0 for k0, _ in windows(wl, F, warmup + i)])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    same = all(torch.equal(torch.from_numpy(r).to(o.device), o) for r, o in zip(ref_outs, outs))
    ctx.close()
    samples = step_samples(wl, F)
    return {"value": samples * steps / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms / steps,
            "graph_launches_per_step": 1, "kernel_nodes": nodes, "capture_s": capture_s,
            "equal_to_sequential_bit_for_bit": bool(same),
            "note": "one CUDA graph per step (all levels' windows; streaming loops as conditional WHILE nodes)"}


def max_rel_diff(a_levels, b_levels):
    """Largest relative difference of lambda_H, lambda^l, lambda^{l-1} (each relative to itself)
    and of the level difference (relative to lambda^l) between two runs' per-sample results."""
    worst = 0.0
    for a, b in zip(a_levels, b_levels):
        den = np.abs(b[..., :3]) + (b[..., :3] == 0)
        worst = max(worst, float((np.abs(a[..., :3] - b[..., :3]) / den).max()),
                    float((np.abs(a[..., 3] - b[..., 3]) / np.abs(b[..., 1])).max()))
    return worst


def time_e2e(binding, wl, prec, steps, warmup, stream_ptr, F):
    """End to end through the public host API: every step uploads the lattices and shifts from
    host memory, evaluates the step's windows and reads every per-sample result back."""
    import torch

    ctx, zs, ds = setup_context(binding, wl, stream_ptr, prec)
    h2d = sum(z.nbytes + d.nbytes for z, d in zip(zs, ds))
    d2h = sum(lv.R * (k1 - k0) * 4 * 8 + lv.R * 8 for lv, (k0, k1) in zip(wl.levels, windows(wl, F, 0)))
    for l, (k0, k1) in enumerate(windows(wl, F, 0)):  # one untimed pass
        ctx.mq_eval_level(l, k0, k1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        ctx.mq_reset_sums()
        shared = wl.extra.get("shared", False)
        for l in range(len(wl.levels)):
            if shared:
                ctx.mq_set_lattice_embedded(l, zs[l], wl.extra["m_max"])
            else:
                ctx.mq_set_lattice(l, zs[l])
            ctx.mq_set_shifts(l, ds[l])
        if shared:
            ctx.mq_set_reuse(1)
        for l, (k0, k1) in enumerate(windows(wl, F, warmup + i)):
            ctx.mq_eval_level(l, k0, k1)
        ctx.mq_estimate()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    return dt, h2d, d2h


# ------------------------------------------------------------------------------------------
def _oracle_worker(args):
    """Evaluates oracle samples of one level one after another until `budget` seconds have passed
    (at least one sample); returns (samples, seconds)."""
    import os as _os

    _os.environ.setdefault("OMP_NUM_THREADS", "1")
    _os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import mlqmc

    lv, pv, z, delta, ks, coef, budget = args
    t0 = time.perf_counter()
    n = 0
    for i, k in enumerate(ks):
        mlqmc.level_samples(lv, pv, z, delta[i % delta.shape[0]][None, :], [k], *coef)
        n += 1
        if time.perf_counter() - t0 >= budget:
            break
    return n, time.perf_counter() - t0


def _pool_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"


def oracle_level_rates(wl, zs, ds, levels, budget, pool, cores):
    """Per-sample oracle time of each listed level: the host cores are shared out among the levels
    (the finest levels, whose single samples take longest, get one process each), every process
    runs samples of its level until the budget is spent, all levels at once."""
    procs = {l: 1 for l in levels}
    spare = max(0, cores - len(levels))
    cheap = [l for l in levels if wl.levels[l].n_fine <= 256] or list(levels)
    for i in range(spare):
        procs[cheap[i % len(cheap)]] += 1
    jobs, owner = [], []
    for l in levels:
        lv = wl.levels[l]
        pv = wl.levels[l - 1] if l > 0 else None
        for p in range(procs[l]):
            ks = [(p * 7919 + i * 104729) % lv.N for i in range(100000)]
            jobs.append((lv, pv, zs[l], ds[l], ks, (wl.a0, wl.coef_decay, wl.family), budget))
            owner.append(l)
    res = pool.map(_oracle_worker, jobs, chunksize=1)
    per = {}
    for l, (n, dt) in zip(owner, res):
        c, t = per.get(l, (0, 0.0))
        per[l] = (c + n, t + dt)
    return {l: (n, dt) for l, (n, dt) in per.items()}


def oracle_rate(wl, per_level, cores):
    """Samples/s of the whole workload on `cores` processes from per-level (samples, seconds)."""
    cpu_s = sum(lv.N * lv.R * per_level[l][1] / per_level[l][0] for l, lv in enumerate(wl.levels))
    return wl.samples * cores / cpu_s


def cpu_baseline(wl, seconds_budget, zs, ds):
    """Times the oracle as it stands on a bounded sample of every level (all levels at once, one
    sample per process at a time on every host core) and scales to samples/s of the workload."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores, initializer=_pool_init) as pool:
        per = oracle_level_rates(wl, zs, ds, list(range(len(wl.levels))), seconds_budget, pool, cores)
    value = oracle_rate(wl, per, cores)
    sample = "; ".join(f"level {l}: {n} samples in {dt:.1f} process-s" for l, (n, dt) in sorted(per.items()))
    return {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": sample + f" (all levels at once on {cores} processes, first samples with cold per-process "
                               f"caches; extrapolated to the {wl.samples} samples of the workload by the "
                               f"per-level rates, {cores} samples at a time)"}


# ------------------------------------------------------------------------------------------
# Roofline models.
#
# Per-sample kernel (one CTA per sample, workspace on chip): bounded by the FP64 units, whose
# peak is 152 SMs x 2 FP64 FMA lanes per cycle x 2 flops x the SM clock.  FP64 operations
# counted from the kernel source (a fused multiply-add counts two):
#   coarse LOBPCG: 73 per coarse unknown and iteration (residual 6, A w and M w 19, Gram matrix
#   24, update of x, Ax, Mx, p, Ap, Mp 24) + 46 per unknown and eigensolve (two operator
#   applications with normalisation);
#   fine solve with FP32 inner iterations: 23 per fine unknown (interpolation and right-hand side
#   19, FP64 edge weights of the preconditioner 4) + 40 per unknown and refinement step (solution
#   update 2, FP64 residual with the Rayleigh-quotient partials 38);
#   fine solve with FP64 inner iterations (FP64 path, same-mesh solves): + 135 per unknown and
#   inner iteration (operator 24, MINRES updates 12, V-cycle 99).
FP64_EIG_IT, FP64_EIG_CALL, FP64_FINE_SETUP, FP64_FINE_OUTER, FP64_INNER = 73, 46, 23, 40, 135


def stream_min_default(prec):
    return 32 if prec == "mixed" else 256


def percta_fp64_flops(wl, level, st, prec, samples):
    """FP64 operations of one launch of the per-sample kernel on `level` over `samples` samples."""
    lv = wl.levels[level]
    nc = lv.n_coarse
    per = (nc - 1) ** 2 * (FP64_EIG_IT * st["coarse_iters_mean"] + FP64_EIG_CALL)
    solves = []
    if not (lv.n_fine == nc and lv.s == lv.S):
        solves.append(lv.n_fine)
    if level > 0:
        pv = wl.levels[level - 1]
        if not (pv.n_fine == nc and pv.s == lv.S):
            solves.append(pv.n_fine)
    I, O = st["fine_iters_mean"], st["outer_iters_mean"]
    streamed = lv.n_fine >= stream_min_default(prec) and not (lv.n_fine == nc and lv.s == lv.S)
    for n in solves:
        if streamed and n != nc:
            continue  # batched streaming tier
        inner64 = prec == "fp64" or n == nc
        per += (n - 1) ** 2 * (FP64_FINE_SETUP + FP64_FINE_OUTER * O + (FP64_INNER * I if inner64 else 0))
    return per * samples


# Streaming tier (fine meshes >= 1/32 mixed): bounded by HBM.  Bytes per fine unknown with every
# kernel reading and writing each of its arrays once (e = 4 bytes, FP32 inner vectors; the
# default V(1,1) smoothing of this tier):
#   per inner MINRES iteration: MINRES sweeps 14 e (operator + pending update 10 e, Lanczos
#   vector 4 e) + V-cycle 11.5 e on the fine level (restriction of the first sweep's residual
#   4.25 e, prolongation + sweep + dot 7.25 e) + 10.5 e / 4 and / 16 on the coarser streamed
#   levels (the on-chip sub-cycle below 1/32 is not counted);
#   per refinement step: 12 e + 48 bytes (inner start 6 e, final update 5 e, FP64 solution update
#   e + 16, FP64 residual with FP64 weights e + 32) + one V-cycle;
#   per solve: 20 e + 72 bytes (clearing 8 e + 16, FP32 and FP64 weights 3 e + 32, interpolation
#   and right-hand side e + 24, operators of the coarser levels ~8 e).
def stream_bytes(wl, level, st, prec, samples):
    e = 4 if prec == "mixed" else 8
    lv = wl.levels[level]
    vcyc = 11.5 * e + 10.5 * e * (1 / 4 + 1 / 16)
    I, O = st["fine_iters_mean"], st["outer_iters_mean"]
    solves = []
    if lv.n_fine >= stream_min_default(prec) and not (lv.n_fine == lv.n_coarse and lv.s == lv.S):
        solves.append(lv.n_fine)
    if level > 0:
        pv = wl.levels[level - 1]
        if lv.n_fine >= stream_min_default(prec) and pv.n_fine != lv.n_coarse:
            solves.append(pv.n_fine)
    per = 0.0
    for n in solves:
        per += (n - 1) ** 2 * ((14 * e + vcyc) * I + (12 * e + 48 + vcyc) * O + 20 * e + 72)
    return per * samples


# ncu DRAM traffic of the per-sample kernel's launch on a level (one launch of the benchmark's size:
# level 1 of the six-level workload, 4,096 samples; summarised under profiles/), valid only for the
# kernel source it was measured on
SAMPLE_KERNEL_TRAFFIC = {"source_sha256": "7861a6430fbac9e0c146a8aa2dfbd3247634376d533e93997ab395a81abc1a8e",
                         "level": 1, "precision": "mixed", "bytes_per_launch": 140.174592e6 + 41.903360e6}


# ncu DRAM traffic of the operator sweep k_minres_q per algorithmic byte: one launch with the pending
# MINRES update (10 arrays per node) on mesh 1/1024, 16 samples of the six-level workload's finest
# level (summarised under profiles/), scaled to a launch by its algorithmic bytes; valid only for
# the kernel source it was measured on
KMINRES_TRAFFIC = {"source_sha256": "22f59b77c3bc4dc0a0e79efd7d578bdcdaa1e7ff1ab891b96076f838197586da",
                   "dram_per_algorithmic": (471.794432e6 + 170.729984e6) / (16 * 1023 * 1023 * 40)}


def _stream_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("mq_stream.cu", "mq_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2103_03407_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kminres_roofline(probe, steps):
    """Roofline of the largest kernel of the step: the streaming operator sweep, timed live with
    CUDA events around its launches over the timed region; algorithmic bytes counted on the device
    (per active sample and node: 4 arrays, 10 with the pending MINRES update)."""
    ms, launches, nbytes = probe
    if launches == 0 or ms <= 0:
        return None
    per_launch_ms = ms / launches
    bytes_per_launch = nbytes / launches
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    peak, kind = hbm_peak()
    t = KMINRES_TRAFFIC
    traffic = None
    if t["dram_per_algorithmic"] and t["source_sha256"] == _stream_source_hash():
        traffic = t["dram_per_algorithmic"] * bytes_per_launch
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": f"k_minres_q (streaming operator sweep: {launches // max(1, steps)} launches "
                                          f"per step, {per_launch_ms:.3f} ms per launch)",
            "algorithmic_bytes_per_launch": bytes_per_launch, "peak_kind": kind,
            "traffic_note": "ncu DRAM bytes per algorithmic byte of one captured launch x this launch average"}


def _percta_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("mq_sample.cu", "mq_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2103_03407_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"


def fp64_peak_tflops(sm_max_mhz=None):
    """FP64 FMA throughput from the unit counts: 152 SMs x 2 lanes x 2 flops per cycle."""
    mhz = sm_max_mhz or 2070.0
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


def percta_roofline(wl, level, st, prec, ms_per_launch, sm_max_mhz, samples, measured_peak=None):
    flops = percta_fp64_flops(wl, level, st, prec, samples)
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    peak = measured_peak or fp64_peak_tflops(sm_max_mhz)
    lv = wl.levels[level]
    t = SAMPLE_KERNEL_TRAFFIC
    traffic = None
    if t["source_sha256"] == _percta_source_hash() and t["level"] == level and t["precision"] == prec:
        traffic = t["bytes_per_launch"]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "kernel": f"sample_kernel (level {level}: {samples} samples per launch, "
                      f"{ms_per_launch:.2f} ms per launch)",
            "algorithmic_flops": flops,
            "peak_kind": ("measured: FP64 FMA chains kernel (mq_measure_fp64_peak)" if measured_peak else
                          f"derived: FP64 units, 152 SMs x 4 flop/cycle x {sm_max_mhz or 2070:.0f} MHz")}


def stream_roofline(wl, level, st, prec, ms_per_launch, samples):
    nbytes = stream_bytes(wl, level, st, prec, samples)
    achieved = nbytes / (ms_per_launch * 1e-3) / 1e9
    peak, kind = hbm_peak()
    lv = wl.levels[level]
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": f"streaming fine solves (level {level}: {samples} samples per pass, "
                                       f"{ms_per_launch:.2f} ms per pass, all kernels of the stage)",
            "algorithmic_bytes": nbytes, "peak_kind": kind}


def main():
    args = parse()
    rank, world, local = dist_env()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return main_reference(args, wl, rank, world)
    import torch

    from paper_2103_03407_gb300 import binding, build

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(local)
    build.build()
    binding.load()
    stream = torch.cuda.Stream()
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    F = step_fraction(wl, args)
    samples = step_samples(wl, F)  # samples per step (every level's window, every shift)
    use_graph = args.schedule == "graph" and world == 1
    with torch.cuda.stream(stream):
        with sampler:
            ctx, ms, timing, kstats, outs, launches, lsums, probe = time_device(
                binding, torch, wl, args.precision, args.steps, args.warmup, stream, F, rank=rank, world=world,
                sequential=args.schedule != "concurrent")
    # one exchange of the per-level shift sums: the estimate over every rank's shifts
    estimate = merged_estimate(binding, [x[0] for x in lsums], [x[1] for x in lsums], world,
                               shared=wl.extra.get("shared", False))
    if world > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(ms, world, "cuda")
    seq_value = whole_job_rate(samples, world, args.steps, ms)
    graph = None
    if use_graph or (not args.no_graph and world == 1 and args.schedule == "sequential"):
        # the graph schedule on the same windows, with its own clock record (the headline when chosen)
        gsampler = ClockSampler(local)
        with torch.cuda.stream(stream):
            with gsampler:
                graph = time_graph(binding, torch, wl, args.precision, args.steps, args.warmup, stream, F, outs)
        graph["clocks"] = gsampler.summary()
    if use_graph:
        value, ms_step, head_clocks = graph["value"], graph["ms_per_step"], graph["clocks"]
    else:
        value, ms_step, head_clocks = seq_value, ms / args.steps, None
    dof_rate = fine_dof_solves(wl) / F * world / (ms_step / 1e3)
    plain = None
    if not args.no_plain and args.precision == "mixed" and rank == 0:
        # the plain FP64 GPU path on the same steps (same windows) and warm-up
        with torch.cuda.stream(stream):
            ctxp, msp, _, _, outs_p, _, _, _ = time_device(binding, torch, wl, "fp64", args.steps, args.warmup,
                                                           stream, F, sequential=args.schedule != "concurrent")
        ctxp.close()
        plain = {"value": samples * args.steps / (msp / 1e3), "unit": "samples/s", "ms_per_step": msp / args.steps,
                 "steps": args.steps, "warmup": args.warmup,
                 "max_rel_diff_mixed_vs_fp64": max_rel_diff(outs, outs_p),
                 "note": "per-sample results of the last timed step of both paths compared"}
    e2e = None
    if not args.no_e2e:
        steps_e2e = max(1, args.steps)
        dt, h2d, d2h = time_e2e(binding, wl, args.precision, steps_e2e, args.warmup, stream.cuda_stream, F)
        e2e = {"value": samples * steps_e2e / dt, "unit": "samples/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    # dominant kernel: the per-sample kernel launch with the largest device time; the streaming
    # stage of the level where it takes longest is reported beside it
    nl = len(wl.levels)
    lst = [kstats[l][-1] for l in range(nl)]
    per = lambda l, i: timing[l][i] / max(1, timing[l][2])  # per launch
    coef_ms = [per(l, 0) for l in range(nl)]
    sample_ms = [per(l, 1) for l in range(nl)]
    percta_ms = [per(l, 3) for l in range(nl)]
    stream_ms = [per(l, 4) for l in range(nl)]
    win = windows(wl, F, 0)
    # samples per launch: all samples a level evaluated in the timed region over its launches
    per_launch = [wl.levels[l].R * (win[l][1] - win[l][0]) * args.steps / max(1, timing[l][2]) for l in range(nl)]
    clocks = head_clocks or sampler.summary()
    top = int(np.argmax(percta_ms))
    fp64_peak = None
    try:
        fp64_peak = binding.mq_measure_fp64_peak(0)[0]
    except Exception:
        pass
    roofline_sample = percta_roofline(wl, top, lst[top], args.precision, percta_ms[top], clocks.get("sm_max_mhz"),
                                      per_launch[top], fp64_peak)
    # the dominant kernel of the step (largest share of the launch list): the streaming operator
    # sweep where the workload streams; the per-sample kernel otherwise
    roofline = kminres_roofline(probe, args.steps) or roofline_sample
    stop = int(np.argmax(stream_ms))
    roofline_stream = (stream_roofline(wl, stop, lst[stop], args.precision, stream_ms[stop], per_launch[stop])
                       if stream_ms[stop] > 0 else None)
    result = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": dict(workload_config(wl, args.precision, world, F),
                       schedule="graph" if use_graph else ("concurrent" if args.schedule == "concurrent" else
                                                           "sequential")),
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "roofline_stream": roofline_stream,
        "roofline_sample_kernel": roofline_sample, "fp64_peak_measured_tflops": fp64_peak,
        "graph_schedule": graph,
        "sequential_schedule": {"value": seq_value, "unit": "samples/s", "ms_per_step": ms / args.steps,
                                "clocks": sampler.summary(),
                                "note": "the same steps level by level through the host API; the per-kernel "
                                        "rooflines, per-level timings and gpu_launches come from this run"},
        "clocks": clocks,
        "per_level": [{"level": l, "kernel_ms": coef_ms[l] + sample_ms[l], "coef_ms": coef_ms[l],
                       "sample_ms": sample_ms[l], "percta_ms": percta_ms[l], "stream_ms": stream_ms[l],
                       "coarse_iters_mean": lst[l]["coarse_iters_mean"],
                       "fine_iters_mean": lst[l]["fine_iters_mean"], "outer_iters_mean": lst[l]["outer_iters_mean"],
                       "blocks": lst[l]["blocks"], "threads": lst[l]["threads"], "smem": lst[l]["smem_bytes"],
                       "workspace": lst[l]["workspace_bytes"]} for l in range(len(wl.levels))],
        "plain_fp64": plain,
        "estimate": estimate,
        "fine_dof_solves_per_s": dof_rate,
        "gpu_launches_note": "kernels launched in the timed region, counted by the library",
    }
    if rank == 0 and not args.no_baseline:
        result["cpu_baseline"] = cpu_baseline(wl, args.baseline_seconds, ctx_lattices(wl, binding),
                                              shifts(wl.seed, wl.levels))
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        torch.distributed.destroy_process_group()


def workload_config(wl, precision, world, F=1):
    win = windows(wl, F, 0)
    return {"workload": wl.name, "levels": [lv.__dict__ for lv in wl.levels], "samples_per_step": step_samples(wl, F),
            "workload_samples": wl.samples,
            "step": (f"1/{F} of every level's lattice points, all shifts: step i evaluates window i mod {F} "
                     f"({', '.join(str(k1 - k0) for k0, k1 in win)} points per shift on levels 0..{len(win) - 1}); "
                     f"{F} steps cover the workload once") if F > 1 else "every point of every level",
            "precision": precision, "l2": "inputs larger than L2 (coefficient fields of the finest level exceed "
            "129 MB)", "parallelism": f"dp{world} (the workload's shifts partitioned across ranks; per-level shift "
            f"sums merged once at the end)"}


def ctx_lattices(wl, binding):
    return [binding.mq_cbc_lattice(lv.N, lv.s, wl.decay) for lv in wl.levels]


def main_reference(args, wl, rank, world):
    """The oracle as it stands on the host cores.  Levels whose single oracle sample takes more than
    a few seconds (meshes finer than 1/256) are timed once, in the first warm-up step; every other
    step times a bounded sample of the remaining levels and the value combines the latest per-level
    rates (extrapolated to the whole workload, as stated in the line)."""
    if rank != 0:
        return
    import multiprocessing as mp

    from oracle import lattice

    zs = [lattice.cbc(lv.N, lv.s, wl.decay) for lv in wl.levels]
    ds = shifts(wl.seed, wl.levels)
    cores = os.cpu_count() or 1
    slow = [l for l, lv in enumerate(wl.levels) if lv.n_fine > 256]
    fast = [l for l in range(len(wl.levels)) if l not in slow]
    per = {}
    vals = []
    t_steps = []
    with mp.get_context("spawn").Pool(cores, initializer=_pool_init) as pool:
        if slow:
            per.update(oracle_level_rates(wl, zs, ds, slow, 1.0, pool, cores))
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            if fast:
                per.update(oracle_level_rates(wl, zs, ds, fast, 4.0, pool, cores))
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                vals.append(oracle_rate(wl, per, cores))
                t_steps.append(dt)
    value = float(np.mean(vals))
    F = step_fraction(wl, args)
    samples = step_samples(wl, F)
    ms = samples / value * 1e3
    sample = "; ".join(f"level {l}: {n} samples in {dt:.1f} process-s" for l, (n, dt) in sorted(per.items()))
    note = (f"levels {slow} timed once before the steps (one sample per process); " if slow else "") + \
        f"each step times levels {fast} for ~4 s on {cores} processes; ms_per_step is extrapolated from the " \
        f"per-level rates to the bench step of {samples} samples"
    out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_kind": "extrapolated", "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(wl, "fp64 (CPU oracle)", world, F),
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample + "; " + note, "value": value,
                            "unit": "samples/s"},
           "wall_s_per_timed_step": float(np.mean(t_steps)) if t_steps else None,
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
