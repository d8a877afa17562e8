"""The large workloads at full size, in the launch configuration of the benchmark, with sampled
outputs checked against the FP64 oracle one by one, at the metric's 1e-10 relative tolerance.

The oracle solves a 1,046,529-unknown system per sample on the finest meshes, so only a few
samples per level are drawn: the first point of the first shift, the last point of the last
shift and two random (shift, point) pairs.  The oracle samples run in a pool of processes
(started with ``spawn``, one sample per process) while the GPU evaluates the levels.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import lattice, mlqmc
from synthetic_inputs import WORKLOADS, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


@pytest.fixture(scope="module")
def pool():
    # one BLAS thread per process: the pool is sized to the host cores
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    p = mp.get_context("spawn").Pool(max(2, min(16, os.cpu_count() or 2)))
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    yield p
    p.terminate()
    p.join()


def setup(B, wl, levels=None):
    levels = levels or wl.levels
    ctx = B.Context(0)
    ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(levels)
    zs = [lattice.cbc(lv.N, lv.s, wl.decay) for lv in levels]
    ds = shifts(wl.seed, wl.levels)[: len(levels)]
    for l in range(len(levels)):
        ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(B.MQ_PREC_MIXED if wl.precision == "mixed" else B.MQ_PREC_FP64)
    return ctx, zs, ds


def picks_for(lv, rng):
    """The edge samples (first point of the first shift, last point of the last shift) and two
    random ones."""
    out = [(0, 0), (lv.R - 1, lv.N - 1)]
    while len(out) < 4:
        p = (int(rng.integers(lv.R)), int(rng.integers(lv.N)))
        if p not in out:
            out.append(p)
    return out


def submit(pool, wl, l, zs, ds, picks):
    lv = wl.levels[l]
    pv = wl.levels[l - 1] if l > 0 else None
    return [pool.apply_async(mlqmc.level_samples, (lv, pv, zs[l], ds[l][r : r + 1], [k], wl.a0, wl.decay, wl.family))
            for r, k in picks]


def rel_errors(wl, l, got, ref):
    """Relative errors of (lambda_H, lambda^l, lambda^{l-1}) and of the difference (relative to
    lambda^l, the size of the values it is formed from)."""
    e = [abs(got[0] - ref[0]) / abs(ref[0]), abs(got[1] - ref[1]) / abs(ref[1]),
         abs(got[2] - ref[2]) / abs(ref[2]) if l > 0 else abs(got[2]),
         abs(got[3] - ref[3]) / abs(ref[1])]
    return e


def check_level(wl, l, ps, picks, futures, report):
    worst = np.zeros(4)
    for (r, k), f in zip(picks, futures):
        ref = f.get()[0, 0]
        worst = np.maximum(worst, rel_errors(wl, l, ps[r, k], ref))
    report.append((wl.name, l, worst))
    print(f"{wl.name} level {l}: max rel err lambda_H {worst[0]:.2e}, lambda^l {worst[1]:.2e}, "
          f"lambda^(l-1) {worst[2]:.2e}, diff {worst[3]:.2e}")
    return worst


def assert_report(report, tol):
    bad = [(name, l, w) for name, l, w in report if not (w[0] <= 1e-12 and w[1] <= tol and w[2] <= tol
                                                         and w[3] <= 2 * tol)]
    assert not bad, "beyond tolerance: " + "; ".join(
        f"{n} level {l}: {w[0]:.2e} {w[1]:.2e} {w[2]:.2e} {w[3]:.2e}" for n, l, w in bad)


@pytest.mark.parametrize("name", ["single_h512_s256", "stress_h1024_s1024"])
def test_large_single_level_workload(B, pool, name):
    wl = WORKLOADS[name]
    assert wl.tol == 1e-10
    lv = wl.levels[0]
    ctx, zs, ds = setup(B, wl)
    picks = picks_for(lv, np.random.default_rng(4))
    fut = submit(pool, wl, 0, zs, ds, picks)
    ps, sums = ctx.mq_eval_level(0, 0, lv.N)
    assert np.all(np.isfinite(ps))
    assert np.allclose(sums, ps[..., 3].sum(axis=1), rtol=1e-12)
    report = []
    check_level(wl, 0, ps, picks, fut, report)
    assert_report(report, wl.tol)
    m, se, _, _ = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0
    ctx.close()


def test_six_level_workload(B, pool):
    wl = WORKLOADS["mlqmc6_h32_1024"]
    assert wl.tol == 1e-10
    ctx, zs, ds = setup(B, wl)
    rng = np.random.default_rng(3)
    picks = [picks_for(lv, rng) for lv in wl.levels]
    # the finest levels' oracle samples take longest: submit them first
    futs = {l: submit(pool, wl, l, zs, ds, picks[l]) for l in reversed(range(len(wl.levels)))}
    report = []
    for l, lv in enumerate(wl.levels):
        ps, sums = ctx.mq_eval_level(l, 0, lv.N)
        assert np.all(np.isfinite(ps))
        assert np.allclose(sums, ps[..., 3].sum(axis=1), rtol=1e-12)
        check_level(wl, l, ps, picks[l], futs[l], report)
    assert_report(report, wl.tol)
    m, se, lm, lvar = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0 and np.all(lvar >= 0)
    ctx.close()


def test_six_level_estimate_on_a_subsample(B, pool):
    # the estimator (eq. tg-mlqmc, eq. sample_var) of the three coarsest levels of the six-level
    # workload on the first four points of every shift, against the oracle's estimate of the same
    # 3 x 64 samples
    wl = WORKLOADS["mlqmc6_h32_1024"]
    levels = wl.levels[:3]
    ctx, zs, ds = setup(B, wl, levels)
    npts = 4
    futs = []
    for l, lv in enumerate(levels):
        pv = levels[l - 1] if l else None
        futs.append(pool.apply_async(mlqmc.level_samples, (lv, pv, zs[l], ds[l], list(range(npts)), wl.a0, wl.decay,
                                                           wl.family)))
    got = [ctx.mq_eval_level(l, 0, npts)[0] for l in range(len(levels))]
    m, se, lm, lvar = ctx.mq_estimate()
    refs = [f.get() for f in futs]
    om, ose, olm, olv = mlqmc.estimate([mlqmc.shift_means(r[..., 3], npts) for r in refs])
    print(f"subsample estimate: mean {m!r} vs {om!r}, se {se!r} vs {ose!r}")
    assert m == pytest.approx(om, rel=1e-10)
    for l in range(len(levels)):
        assert lm[l] == pytest.approx(olm[l], rel=1e-10, abs=1e-10 * abs(refs[l][..., 1]).max())
    # SE = sqrt(sum_l Vhat_l) is 1-Lipschitz in the scaled deviations (Qhat_l - Q^(r)_l) /
    # sqrt(R (R - 1)); a per-sample error of at most e moves every shift mean by at most e, every
    # deviation by at most 2 e, and so SE by at most 2 e sqrt((L + 1) / (R - 1))
    e = max(np.abs(g[..., 3] - r[..., 3]).max() for g, r in zip(got, refs))
    bound = 2.0 * e * np.sqrt(len(levels) / (levels[0].R - 1)) + 1e-14 * ose
    print(f"subsample SE: |diff| {abs(se - ose):.2e}, bound {bound:.2e} (relative {abs(se - ose) / ose:.2e})")
    assert abs(se - ose) <= bound
    ctx.close()
