"""Embedded lattice rules and the reuse scheme across levels on the GPU, against the oracle.

Sec. 2.5 (embedded rules, radical-inverse order) and Sec. 4.3, the paragraphs after Algorithm 2:
with shared shifts and nested points, every level l >= 1 takes its coarse pair from level 0 and
lambda^{l-1} from level l-1 instead of solving for them.  Tolerances as in test_gpu_parity.py:
lattice points bit-exact, coarse eigenvalues 1e-12 relative, two-grid values 1e-10 relative;
values taken from the store (lambda^{l-1}) equal the level below's bit for bit.
"""
import numpy as np
import pytest

from oracle import lattice, mlqmc
from synthetic_inputs import WORKLOADS, Level, shared_shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


# level 0 direct on 1/16 (s_0 = 16), levels 1-3 on 1/32 .. 1/128 from level 0's coarse problem;
# N halves level by level; an embedded rule of 2^5 points
LEVELS = [Level(16, 16, 16, 16, 16, 3), Level(32, 16, 32, 16, 8, 3), Level(64, 16, 64, 16, 4, 3),
          Level(128, 16, 128, 16, 2, 3)]
MBITS = 5


def make_reuse_ctx(B, levels=LEVELS, mbits=MBITS, prec=1, seed=21, reuse=True):
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, max(lv.s for lv in levels), 0, 2.0)
    ctx.mq_set_levels(levels)
    z = lattice.embedded_cbc(1, mbits, max(lv.s for lv in levels))
    ds = shared_shifts(seed, levels)
    for l, lv in enumerate(levels):
        ctx.mq_set_lattice_embedded(l, z[: lv.s], mbits)
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    if reuse:
        ctx.mq_set_reuse(1)
    return ctx, z, ds


def test_embedded_lattice_points_bit_exact(B):
    ctx, z, ds = make_reuse_ctx(B, reuse=False)
    l, lv = 2, LEVELS[2]
    d = torch.empty((lv.R, 3, lv.s), dtype=torch.float64, device="cuda")
    ctx.mq_lattice_points_device(l, 1, 4, d)
    got = d.cpu().numpy()
    for r in range(lv.R):
        assert np.array_equal(got[r], lattice.embedded_points(z[: lv.s], MBITS, ds[l][r], np.arange(1, 4)))
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_reuse_scheme_matches_oracle(B, prec):
    ctx, z, ds = make_reuse_ctx(B, prec=prec)
    got = []
    for l, lv in enumerate(LEVELS):
        ps, _ = ctx.mq_eval_level(l, 0, lv.N)
        got.append(ps)
    full = ds[-1]
    for r in range(LEVELS[0].R):
        ref = mlqmc.shared_samples(LEVELS, z, MBITS, full[r], list(range(LEVELS[0].N)))
        for l, lv in enumerate(LEVELS):
            g, o = got[l][r], ref[l, : lv.N]
            assert np.all(np.abs(g[:, 0] - o[:, 0]) <= 1e-12 * np.abs(o[:, 0])), (l, r)
            assert np.all(np.abs(g[:, 1] - o[:, 1]) <= 1e-10 * np.abs(o[:, 1])), (l, r)
            if l > 0:
                # lambda^{l-1} is the stored value of level l-1 itself, and the coarse eigenvalue
                # the stored level-0 one
                assert np.array_equal(g[:, 2], got[l - 1][r][: lv.N, 1])
                assert np.array_equal(g[:, 0], got[0][r][: lv.N, 0])
                assert np.array_equal(g[:, 3], g[:, 1] - g[:, 2])
    # the estimate with shared shifts: the standard error of the per-shift totals
    m, se, lm, lv_ = ctx.mq_estimate()
    qs = [mlqmc.shift_means(got[l][..., 3], lv.N) for l, lv in enumerate(LEVELS)]
    om, ose, olm, olv = mlqmc.estimate_shared(qs)
    assert m == pytest.approx(om, rel=1e-13) and se == pytest.approx(ose, rel=1e-10)
    assert np.allclose(lm, olm, rtol=1e-13) and np.allclose(lv_, olv, rtol=1e-10)
    ctx.close()


def test_reuse_equals_recomputing_every_level(B):
    # the same levels without the store (each level solves its own coarse problem, which is level
    # 0's, and its own previous-level problem): equal to the solver tolerances
    ctx_r, _, _ = make_reuse_ctx(B)
    ctx_n, _, _ = make_reuse_ctx(B, reuse=False)
    for l, lv in enumerate(LEVELS):
        a, _ = ctx_r.mq_eval_level(l, 0, lv.N)
        b, _ = ctx_n.mq_eval_level(l, 0, lv.N)
        assert np.all(np.abs(a[..., 0] - b[..., 0]) <= 1e-12 * np.abs(b[..., 0]))
        assert np.all(np.abs(a[..., 1:3] - b[..., 1:3]) <= 1e-10 * np.abs(b[..., 1:3]) + 1e-300)
    ctx_r.close()
    ctx_n.close()


def test_reuse_needs_the_lower_levels_first_and_valid_setup(B):
    ctx, z, ds = make_reuse_ctx(B)
    with pytest.raises(B.MQError) as e:  # level 1 before level 0
        ctx.mq_eval_level(1, 0, 2)
    assert e.value.status == B.MQ_ESTATE
    ctx.mq_eval_level(0, 0, 4)
    ctx.mq_eval_level(1, 0, 4)
    with pytest.raises(B.MQError) as e:  # points 4, 5 of level 0 not evaluated yet
        ctx.mq_eval_level(1, 2, 6)
    assert e.value.status == B.MQ_ESTATE
    ctx.mq_eval_level(0, 4, 16)  # doubling the points of level 0 (the next prefix of the rule)
    ctx.mq_eval_level(1, 4, 8)
    ctx.mq_eval_level(2, 0, 4)
    with pytest.raises(B.MQError) as e:  # concurrent levels cannot depend on one another
        ctx.mq_eval_levels_device([0, 1], None, None)
    assert e.value.status == B.MQ_ESTATE
    # shifts that are not prefixes of one draw are rejected; a new setter switches reuse off
    ctx.mq_set_shifts(1, np.full((3, 32), 0.25))
    with pytest.raises(B.MQError) as e:
        ctx.mq_set_reuse(1)
    assert e.value.status == B.MQ_EINVAL
    ctx.close()
    # a plain-order lattice, or a level not on level 0's coarse problem, is rejected
    ctx, z, ds = make_reuse_ctx(B, reuse=False)
    ctx.mq_set_lattice(1, z[:32] % 8 | 1)
    with pytest.raises(B.MQError):
        ctx.mq_set_reuse(1)
    ctx.close()
    bad = [LEVELS[0], Level(32, 8, 32, 16, 8, 3)]
    ctx, _, _ = make_reuse_ctx(B, levels=bad, reuse=False)
    with pytest.raises(B.MQError):
        ctx.mq_set_reuse(1)
    ctx.close()


def test_shared_workload_sampled(B):
    # the reuse workload at full size (levels 0-3: 4096 .. 512 points x 16 shifts) in the
    # benchmark's launch configuration, edge and random samples against the oracle
    wl = WORKLOADS["shared_mlqmc4_h16_128"]
    m_min, m_max = wl.extra["m_min"], wl.extra["m_max"]
    ctx = B.Context(0)
    ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(wl.levels)
    z = lattice.embedded_cbc(m_min, m_max, max(lv.s for lv in wl.levels), wl.decay)
    ds = shared_shifts(wl.seed, wl.levels)
    for l, lv in enumerate(wl.levels):
        ctx.mq_set_lattice_embedded(l, z[: lv.s], m_max)
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(B.MQ_PREC_MIXED)
    ctx.mq_set_reuse(1)
    got = [ctx.mq_eval_level(l, 0, lv.N)[0] for l, lv in enumerate(wl.levels)]
    rng = np.random.default_rng(6)
    R = wl.levels[0].R
    picks = [(0, 0), (R - 1, wl.levels[-1].N - 1)] + [(int(rng.integers(R)), int(rng.integers(wl.levels[-1].N)))
                                                      for _ in range(2)]
    for r, k in picks:
        ref = mlqmc.shared_samples(wl.levels, z, m_max, ds[-1][r], [k])
        for l in range(len(wl.levels)):
            g, o = got[l][r, k], ref[l, 0]
            assert abs(g[0] - o[0]) <= 1e-12 * abs(o[0]), (l, r, k)
            assert abs(g[1] - o[1]) <= 1e-10 * abs(o[1]), (l, r, k)
            assert abs(g[3] - o[3]) <= 2e-10 * abs(o[1]), (l, r, k)
    m, se, _, _ = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0
    ctx.close()
