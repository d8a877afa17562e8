"""CPU checks of the synthetic workload table and of the benchmark's reference arm (the oracle
timed on the host cores).  No GPU."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from synthetic_inputs import WORKLOADS, shared_shifts, shifts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pow2(n):
    return n >= 1 and (n & (n - 1)) == 0


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_workload_levels_follow_the_readings(name):
    wl = WORKLOADS[name]
    shared = wl.extra.get("shared", False)
    for l, lv in enumerate(wl.levels):
        # nested uniform meshes: powers of two, the coarse mesh divides the fine one
        assert _pow2(lv.n_fine) and _pow2(lv.n_coarse) and lv.n_coarse <= lv.n_fine
        direct = lv.n_fine == lv.n_coarse and lv.s == lv.S
        if shared:
            # reuse scheme: level 0 direct, every other level on level 0's coarse problem
            # (H_l = h_0, S_l = s_0 >= ceil(sqrt(s_l))), point counts powers of two
            lv0 = wl.levels[0]
            assert (l == 0 and direct) or (lv.n_coarse == lv0.n_fine and lv.S == lv0.s)
            assert lv.S >= math.isqrt(lv.s - 1) + 1 and _pow2(lv.N) and lv.N <= 1 << wl.extra["m_max"]
            assert lv.N >= 1 << wl.extra["m_min"] and lv.R == lv0.R
            continue
        # coarse truncation S = ceil(sqrt(s)) on two-grid levels (a direct level uses S = s)
        assert direct or lv.S == math.isqrt(lv.s - 1) + 1
        assert 1 <= lv.S <= lv.s and lv.N >= 1 and lv.R >= 2
        if l > 0:  # finer meshes and longer truncations level by level
            pv = wl.levels[l - 1]
            assert lv.n_fine > pv.n_fine and lv.s >= pv.s
    assert wl.samples == sum(lv.N * lv.R for lv in wl.levels)
    if wl.family == 2:
        # the second test problem: four decays, every mesh resolves the islands (width 1/8)
        assert len(wl.decays) == 4 and wl.coef_decay == wl.decays
        assert all(lv.n_coarse >= 8 for lv in wl.levels)
    else:
        assert wl.coef_decay == wl.decay


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_shifts_are_seeded_uniform_draws(name):
    wl = WORKLOADS[name]
    ds = shifts(wl.seed, wl.levels)
    again = shifts(wl.seed, wl.levels)
    assert len(ds) == len(wl.levels)
    for lv, d, e in zip(wl.levels, ds, again):
        assert d.shape == (lv.R, lv.s) and np.array_equal(d, e)
        assert np.all((d >= 0.0) & (d < 1.0))


def test_shared_shifts_are_prefixes_of_one_draw():
    wl = WORKLOADS["shared_mlqmc4_h16_128"]
    ds = shared_shifts(wl.seed, wl.levels)
    for lv, d in zip(wl.levels, ds):
        assert d.shape == (lv.R, lv.s) and np.array_equal(d, ds[-1][:, : lv.s])
    assert np.array_equal(ds[-1], shared_shifts(wl.seed, wl.levels)[-1])


def test_bench_reference_arm_prints_the_contract_line():
    # the reference arm times the oracle on a bounded sample of every level (no GPU needed)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "qmc_h16_s16"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "samples/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "qmc_h16_s16"


def test_fine_dof_solves_counts_both_meshes_of_a_level():
    sys.path.insert(0, ROOT)
    import bench

    wl = WORKLOADS["mlqmc4_h16_128"]
    # 4096*16*15^2 + 2048*16*(31^2+15^2) + 1024*16*(63^2+31^2) + 512*16*(127^2+63^2)
    assert bench.fine_dof_solves(wl) == 65536 * 225 + 32768 * 1186 + 16384 * 4930 + 8192 * 20098


def test_bench_traffic_pins_match_the_kernel_sources():
    # bench.py reports ncu DRAM figures beside two rooflines only while the kernel sources are the
    # ones the figures were measured on (sha256 of the files); a kernel change without a new
    # capture would silently turn them into null
    import bench

    assert bench.KMINRES_TRAFFIC["source_sha256"] == bench._stream_source_hash()
    assert bench.SAMPLE_KERNEL_TRAFFIC["source_sha256"] == bench._percta_source_hash()
    assert 0.9 < bench.KMINRES_TRAFFIC["dram_per_algorithmic"] <= 1.05
