"""The large workloads at full size, in the launch configuration of the benchmark, with sampled
outputs checked against the FP64 oracle one by one (the oracle solves a 1,046,529-unknown system
per sample on the finest meshes, so only a few samples are drawn)."""
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


def setup(B, wl):
    ctx = B.Context(0)
    ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(wl.levels)
    zs = [lattice.cbc(lv.N, lv.s, wl.decay) for lv in wl.levels]
    ds = shifts(wl.seed, wl.levels)
    for l in range(len(wl.levels)):
        ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(B.MQ_PREC_MIXED if wl.precision == "mixed" else B.MQ_PREC_FP64)
    return ctx, zs, ds


def check_samples(wl, l, ps, zs, ds, picks):
    lv = wl.levels[l]
    pv = wl.levels[l - 1] if l > 0 else None
    for r, k in picks:
        ref = mlqmc.level_samples(lv, pv, zs[l], ds[l][r : r + 1], [k], wl.a0, wl.decay, wl.family)[0, 0]
        got = ps[r, k]
        assert got[0] == pytest.approx(ref[0], rel=1e-12), (l, r, k)
        assert got[1] == pytest.approx(ref[1], rel=wl.tol), (l, r, k)
        if pv is not None:
            assert got[2] == pytest.approx(ref[2], rel=wl.tol), (l, r, k)
        assert abs(got[3] - ref[3]) <= 2 * wl.tol * abs(ref[1]), (l, r, k)


@pytest.mark.parametrize("name", ["single_h512_s256", "stress_h1024_s1024"])
def test_large_single_level_workload(B, name):
    wl = WORKLOADS[name]
    lv = wl.levels[0]
    ctx, zs, ds = setup(B, wl)
    ps, sums = ctx.mq_eval_level(0, 0, lv.N)
    assert np.all(np.isfinite(ps))
    assert np.allclose(sums, ps[..., 3].sum(axis=1), rtol=1e-12)
    check_samples(wl, 0, ps, zs, ds, [(0, 0), (lv.R - 1, lv.N - 1)])
    m, se, _, _ = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0
    ctx.close()


def test_six_level_workload(B):
    wl = WORKLOADS["mlqmc6_h32_1024"]
    ctx, zs, ds = setup(B, wl)
    rng = np.random.default_rng(3)
    for l, lv in enumerate(wl.levels):
        ps, sums = ctx.mq_eval_level(l, 0, lv.N)
        assert np.all(np.isfinite(ps))
        picks = [(int(rng.integers(lv.R)), int(rng.integers(lv.N)))]
        if l <= 2:
            picks.append((int(rng.integers(lv.R)), int(rng.integers(lv.N))))
        check_samples(wl, l, ps, zs, ds, picks)
    m, se, lm, lvar = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0 and np.all(lvar >= 0)
    ctx.close()
