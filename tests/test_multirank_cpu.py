"""The multi-rank (one process per GPU) logic of the benchmark, run as two gloo ranks on CPU:
every rank evaluates its own shard of shifts, the timed region ends with the slowest rank, and the
reported rate counts the samples of all ranks.  No GPU."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from synthetic_inputs import WORKLOADS, shifts

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = WORKLOADS["qmc_h16_s16"]
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")  # rank 1 is the slower one
        rate = bench.whole_job_rate(wl.samples, world, 3, ms)
        ds = shifts(bench.shard_seed(wl.seed, rank), wl.levels)
        results[rank] = (ms, rate, ds[0].copy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_count_all_samples():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), results), nprocs=world, join=True)
        res = dict(results)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        ms, rate, _ = res[rank]
        assert ms == 150.0  # the max over ranks, seen by every rank
        assert rate == 2048 * world * 3 / 0.150
    # the shards draw different shifts; rank 0 keeps the workload's own
    assert not np.array_equal(res[0][2], res[1][2])
    from synthetic_inputs import WORKLOADS, shifts

    wl = WORKLOADS["qmc_h16_s16"]
    assert np.array_equal(res[0][2], shifts(wl.seed, wl.levels)[0])


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1000, 1, 2, 500.0) == 4000.0
