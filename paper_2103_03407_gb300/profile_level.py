"""Runs one level of a workload on a subset of its lattice points (for profilers and timing).

    python -m paper_2103_03407_gb300.profile_level --workload mlqmc4_h16_128 --level 1 --points 64 \
        --precision mixed [--repeat 2]
    python -m paper_2103_03407_gb300.profile_level --workload mlqmc6_h32_1024 --level 0 ... --level 5 --fraction 32

Prints the device time and iteration statistics of each evaluation as JSON lines.

    python -m paper_2103_03407_gb300.profile_level --gemm 256 1024 256 [--repeat 2]

runs only the coefficient evaluation a = a0 + Y Psi (mixed precision: the tensor-core GEMM) on
mesh 1/n with s terms for B random parameter vectors.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mlqmc4_h16_128")
    ap.add_argument("--level", type=int, action="append")
    ap.add_argument("--points", type=int, default=64)
    ap.add_argument("--fraction", type=int, default=0,
                    help="evaluate N_l / F points of every level instead of --points (F = 32: one benchmark step)")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--stream-min", type=int, default=0, help="fine meshes from 1/n on run in the streaming tier")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA of the per-sample kernel (0: default)")
    ap.add_argument("--nu", type=int, default=0, help="Jacobi steps per side of the V-cycle (0: default)")
    ap.add_argument("--tol-inner", type=float, default=0.0,
                    help="relative reduction of each inner solve (0: the library's default)")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("N", "S", "B"),
                    help="time the coefficient evaluation alone on mesh 1/N with S terms for B samples")
    a = ap.parse_args()
    if a.gemm:
        return gemm(a)
    from paper_2103_03407_gb300 import binding, build
    from synthetic_inputs import WORKLOADS, shifts

    build.build()
    wl = WORKLOADS[a.workload]
    ctx = binding.Context(0)
    if wl.family == 2:
        ctx.mq_set_islands(max(lv.s for lv in wl.levels), *wl.decays)
    else:
        ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(wl.levels)
    ds = shifts(wl.seed, wl.levels)
    for l, lv in enumerate(wl.levels):
        ctx.mq_set_lattice(l, binding.mq_cbc_lattice(lv.N, lv.s, wl.decay))
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(binding.MQ_PREC_MIXED if a.precision == "mixed" else binding.MQ_PREC_FP64)
    if a.stream_min:
        ctx.mq_set_tier(a.stream_min)
    if a.nu:
        ctx.mq_set_smoothing(a.nu)
    if a.tol_inner:
        ctx.mq_set_solver_options(a.tol_inner, 0, 0)
    if a.threads:
        for l in range(len(wl.levels)):
            ctx.mq_set_cta_threads(l, a.threads)
    for l in a.level or [len(wl.levels) - 1]:
        n = max(1, wl.levels[l].N // a.fraction) if a.fraction else min(a.points, wl.levels[l].N)
        for _ in range(a.repeat):
            ctx.mq_eval_level(l, 0, n, per_sample=False)
            st = ctx.mq_get_stats()
            print(json.dumps({"level": l, "points": n, "samples": n * wl.levels[l].R, "stream_min": a.stream_min,
                              "threads_req": a.threads, "nu": a.nu, "tol_inner": a.tol_inner, **st}))
    ctx.close()


def gemm(a):
    import time

    import torch

    from paper_2103_03407_gb300 import binding, build
    from synthetic_inputs import Level, random_points

    build.build()
    n, s, B = a.gemm
    ctx = binding.Context(0)
    ctx.mq_set_coefficient(1.0, s, 0, 2.0)
    ctx.mq_set_levels([Level(n, n, s, s, 1, 2)])
    ctx.mq_set_precision(binding.MQ_PREC_MIXED if a.precision == "mixed" else binding.MQ_PREC_FP64)
    Y = torch.from_numpy(random_points(1, B, s)).cuda()
    out = torch.empty((B, 2 * n * n), dtype=torch.float64, device="cuda")
    ctx.mq_coefficients_device(n, s, Y, B, s, out)  # builds the tables
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.mq_coefficients_device(n, s, Y, B, s, out)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        flops = 2.0 * B * s * 2 * n * n
        print(json.dumps({"gemm": [n, s, B], "ms": dt * 1e3, "algorithmic_tflops": flops / dt / 1e12}))
    ctx.close()


if __name__ == "__main__":
    main()
