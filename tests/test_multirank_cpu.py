"""The multi-rank (one process per GPU) logic of the benchmark, run as two gloo ranks on CPU:
every rank evaluates its share of one workload's shifts, the timed region ends with the slowest
rank, the reported rate counts the samples of all ranks, and the per-level shift sums of all ranks
are merged into one estimate.  No GPU: the per-sample values come from the oracle, the merge and
the estimate from the library's host code.  (Unmeasured on hardware: the GPU runs of this build
have one GPU.)"""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# two small levels: a direct level on mesh 1/8 and a two-grid level on 1/16 from it
def _levels():
    from synthetic_inputs import Level

    return [Level(8, 8, 4, 4, 8, 4), Level(16, 8, 8, 4, 4, 4)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _level_sums(levels, ds, zs):
    """Per-level shift sums of the level differences (oracle values) and points per shift."""
    from oracle import mlqmc

    out = []
    for l, lv in enumerate(levels):
        ps = mlqmc.level_samples(lv, levels[l - 1] if l else None, zs[l], ds[l], list(range(lv.N)))
        out.append(ps[..., 3].sum(axis=1))
    return out, [lv.N for lv in levels]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from oracle import lattice
    from paper_2103_03407_gb300 import binding
    from synthetic_inputs import WORKLOADS, shifts_for_rank

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = WORKLOADS["qmc_h16_s16"]
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")  # rank 1 is the slower one
        rate = bench.whole_job_rate(wl.samples, world, 3, ms)
        levels = _levels()
        zs = [lattice.cbc(lv.N, lv.s) for lv in levels]
        ds = shifts_for_rank(7, levels, rank, world)
        sums, npts = _level_sums(levels, ds, zs)
        est = bench.merged_estimate(binding, sums, npts, world)
        results[rank] = (ms, rate, ds[0].copy(), est)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_count_all_samples_and_merge_the_estimate():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), results), nprocs=world, join=True)
        res = dict(results)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        ms, rate, _, _ = res[rank]
        assert ms == 150.0  # the max over ranks, seen by every rank
        assert rate == 2048 * world * 3 / 0.150
    # the ranks hold disjoint shares of one draw of R * world shifts
    from oracle import lattice, mlqmc
    from paper_2103_03407_gb300 import binding
    from synthetic_inputs import shifts_for_rank

    levels = _levels()
    full = shifts_for_rank(7, [type(lv)(lv.n_fine, lv.n_coarse, lv.s, lv.S, lv.N, lv.R * world) for lv in levels], 0, 1)
    assert np.array_equal(res[0][2], full[0][: levels[0].R]) and np.array_equal(res[1][2], full[0][levels[0].R:])
    # the merged estimate equals, bit for bit, one process evaluating all R * world shifts, and the
    # oracle's estimate of the same samples
    zs = [lattice.cbc(lv.N, lv.s) for lv in levels]
    sums, npts = _level_sums(levels, full, zs)
    one = binding.mq_estimate_sums(sums, npts)
    for rank in range(world):
        est = res[rank][3]
        assert est["mean"] == one[0] and est["std_err"] == one[1]
        assert est["shifts_per_level"] == [lv.R * world for lv in levels]
    om, ose, _, _ = mlqmc.estimate([s / n for s, n in zip(sums, npts)])
    assert abs(one[0] - om) <= 1e-14 * abs(om) and abs(one[1] - ose) <= 1e-13 * ose


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1000, 1, 2, 500.0) == 4000.0
