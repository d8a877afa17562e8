"""The second test problem of Sec. 5 (four islands, reaction term b u) and the eigenfunction
functional G(u) on the GPU, through the C ABI, against the FP64 oracle.

Tolerances: coefficients a and b to FP64 rounding of their terms (as for the other families);
the reaction stencil to FP64 rounding; per-sample eigenvalues to 1e-12 (coarse) and 1e-10 (two-grid)
relative, as for the other families.  The functional G(w) of the two-grid solution w is a
normalised linear functional of w, so it moves to first order with the part of the solve error
orthogonal to the eigenvector (the part along it only rescales w): at the solver's default residual
targets (1e-5 relative with FP32 inner solves) that part is ~1e-5 times |lambda_1 - lambda_H| / gap,
and the values agree to ~1e-8; with the residual target at 1e-10 the tests ask for 1e-10.
"""
import numpy as np
import pytest

from oracle import fem, lattice, mlqmc
from synthetic_inputs import WORKLOADS, Level, random_points, random_vectors, shared_shifts, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DECAYS = (4.0 / 3.0, 2.0, 4.0 / 3.0, 2.0)  # p_a, p_a', p_b, p_b' (the left case of the paper's figure)


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


def make_ctx(B, levels, prec=1, decays=DECAYS, seed=31, qoi=0, tol_linear=0.0, family=2):
    ctx = B.Context(0)
    s_max = max(lv.s for lv in levels)
    if family == 2:
        ctx.mq_set_islands(s_max, *decays)
    else:
        ctx.mq_set_coefficient(1.0, s_max, family, 2.0)
    ctx.mq_set_levels(levels)
    zs = [lattice.cbc(lv.N, lv.s, 4.0 / 3.0) for lv in levels]
    ds = shifts(seed, levels)
    for l in range(len(levels)):
        ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec, tol_linear)
    ctx.mq_set_qoi(qoi)
    return ctx, zs, ds


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,s,nb", [(8, 16, 5), (16, 37, 130), (64, 64, 9)])
def test_island_coefficients_match_oracle(B, prec, n, s, nb):
    ctx, _, _ = make_ctx(B, [Level(n, n, s, s, 8, 2)], prec=prec)
    Y = random_points(n + s + nb, nb, s)
    dY = torch.from_numpy(Y).cuda()
    da = torch.empty((nb, 2 * n * n), dtype=torch.float64, device="cuda")
    db = torch.empty_like(da)
    ctx.mq_coefficients_device(n, s, dY, nb, s, da)
    ctx.mq_reaction_coefficients_device(n, s, dY, nb, s, db)
    ga, gb = da.cpu().numpy(), db.cpu().numpy()
    for b in range(nb):
        ra, rb = fem.problem2_coefficients(n, Y[b], DECAYS)
        # to a few roundings of the largest value (the two sides add the terms in different orders)
        eps = np.finfo(np.float64).eps
        assert np.abs(ga[b] - ra).max() <= 16 * eps * np.abs(ra).max()
        assert np.abs(gb[b] - rb).max() <= 16 * eps * np.abs(rb).max()
    # the reaction coefficient is undefined for the other families
    ctx0, _, _ = make_ctx(B, [Level(n, n, s, s, 8, 2)], prec=prec, family=0)
    with pytest.raises(B.MQError) as e:
        ctx0.mq_reaction_coefficients_device(n, s, dY, nb, s, db)
    assert e.value.status == B.MQ_ESTATE
    ctx.close()
    ctx0.close()


@pytest.mark.parametrize("n", [2, 4, 8, 32])
def test_reaction_stencil_matches_assembled_matrix(B, n):
    ctx, _, _ = make_ctx(B, [Level(8, 8, 1, 1, 8, 2)])
    nb = 3
    rng = np.random.default_rng(n)
    bt = 0.1 + 2.0 * rng.random((nb, 2 * n * n))
    x = random_vectors(n + 7, nb, (n - 1) ** 2)
    db, dx = torch.from_numpy(bt).cuda(), torch.from_numpy(x).cuda()
    dy = torch.empty_like(dx)
    for which in (3, 4):
        ctx.mq_apply_operator_device(n, nb, db, which, 0.0, dx, dy)
        got = dy.cpu().numpy()
        for b in range(nb):
            _, _, Bm = fem.assemble(n, np.ones(2 * n * n), b_t=bt[b])
            ref = Bm @ x[b]
            assert np.abs(got[b] - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max()) * 8
    ctx.close()


# level 0 direct on 1/8 (s = 16); levels 1, 2 two-grid from (1/8, S = 4) on 1/16 and 1/32; the
# previous-level solve of level 1 runs on the coarse mesh itself (FP64 inner solve)
LEVELS = [Level(8, 8, 16, 16, 6, 2), Level(16, 8, 16, 4, 5, 2), Level(32, 8, 16, 4, 3, 2)]


def _oracle(levels, zs, ds, decay, family, qoi, l):
    lv, pv = levels[l], (levels[l - 1] if l else None)
    return mlqmc.level_samples(lv, pv, zs[l], ds[l], list(range(lv.N)), 1.0, decay, family, qoi=qoi)


@pytest.mark.parametrize("prec", [0, 1])
def test_problem2_eigenvalue_samples_match_oracle(B, prec):
    ctx, zs, ds = make_ctx(B, LEVELS, prec=prec)
    for l, lv in enumerate(LEVELS):
        ps, _ = ctx.mq_eval_level(l, 0, lv.N)
        ref = _oracle(LEVELS, zs, ds, DECAYS, 2, "eigenvalue", l)
        e0 = np.max(np.abs(ps[..., 0] - ref[..., 0]) / np.abs(ref[..., 0]))
        e1 = np.max(np.abs(ps[..., 1] - ref[..., 1]) / np.abs(ref[..., 1]))
        e2 = np.max(np.abs(ps[..., 2] - ref[..., 2]) / np.maximum(np.abs(ref[..., 2]), 1e-300)) if l else 0.0
        print(f"problem 2 prec {prec} level {l}: lambda_H {e0:.2e} lambda^l {e1:.2e} lambda^(l-1) {e2:.2e}")
        assert e0 <= 1e-12 and e1 <= 1e-10 and e2 <= 1e-10
        assert np.all(np.abs(ps[..., 3] - ref[..., 3]) <= 2e-10 * np.abs(ref[..., 1]))
    st = ctx.mq_get_stats()
    print(f"iterations: coarse {st['coarse_iters_mean']:.1f}, inner {st['fine_iters_mean']:.1f}, "
          f"outer {st['outer_iters_mean']:.1f}")
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tol,bound", [(0.0, 1e-7), (1e-10, 1e-10)])
def test_problem2_functional_samples_match_oracle(B, prec, tol, bound):
    ctx, zs, ds = make_ctx(B, LEVELS, prec=prec, qoi=B.MQ_QOI_FUNCTIONAL, tol_linear=tol)
    worst = 0.0
    for l, lv in enumerate(LEVELS):
        ps, _ = ctx.mq_eval_level(l, 0, lv.N)
        ref = _oracle(LEVELS, zs, ds, DECAYS, 2, "functional", l)
        assert np.all(np.abs(ps[..., 0] - ref[..., 0]) <= 1e-12 * np.abs(ref[..., 0]))  # lambda_H
        e = np.abs(ps[..., 1:3] - ref[..., 1:3]) / np.abs(ref[..., 1:2])
        worst = max(worst, e.max())
        assert np.array_equal(ps[..., 3], ps[..., 1] - ps[..., 2])
    print(f"problem 2 functional, prec {prec}, residual target {tol or 'default'}: max rel err {worst:.2e}")
    assert worst <= bound
    m, se, _, _ = ctx.mq_estimate()
    assert np.isfinite(m) and se > 0 and 0.1 < m < 1.0
    ctx.close()


@pytest.mark.parametrize("tier", [0, 1])
def test_functional_on_both_tiers(B, tier):
    # family 0 (no reaction) with the fine solves of mesh 1/64 in the per-sample kernel (tier 0) or
    # the streaming tier (tier 1); FP32 inner solves, residual target 1e-10
    levels = [Level(16, 8, 16, 4, 4, 2), Level(64, 16, 32, 6, 3, 2)]
    ctx, zs, ds = make_ctx(B, levels, prec=1, family=0, qoi=B.MQ_QOI_FUNCTIONAL, tol_linear=1e-10)
    ctx.mq_set_level_config(1, tier, 0, 0)
    for l, lv in enumerate(levels):
        ps, _ = ctx.mq_eval_level(l, 0, lv.N)
        ref = _oracle(levels, zs, ds, 2.0, 0, "functional", l)
        e = np.abs(ps[..., 1:3] - ref[..., 1:3]) / np.abs(ref[..., 1:2])
        print(f"family 0 functional, tier {tier}, level {l}: max rel err {e.max():.2e}")
        assert e.max() <= 1e-10
    ctx.close()


@pytest.mark.parametrize("qoi", [0, 1])
def test_problem2_streaming_tier_matches_oracle_and_per_sample_tier(B, qoi):
    # the reaction term in the streaming tier (mixed precision, V(1,1) with the lumped reaction in the
    # multigrid): fine meshes 1/64 (streamed levels, several multigrid levels and the sub-cycle) and
    # 1/32 (the whole V-cycle in the sub-cycle), against the oracle and against the per-sample tier
    levels = [Level(8, 8, 16, 16, 4, 2), Level(32, 8, 16, 4, 3, 2), Level(64, 8, 16, 4, 3, 2)]
    ctx_s, zs, ds = make_ctx(B, levels, prec=1, qoi=qoi, tol_linear=1e-10)
    ctx_p, _, _ = make_ctx(B, levels, prec=1, qoi=qoi, tol_linear=1e-10)
    for l in (1, 2):
        ctx_s.mq_set_level_config(l, 1, 0, 0)
        ctx_p.mq_set_level_config(l, 0, 0, 0)
    name = "eigenvalue" if qoi == 0 else "functional"
    for l, lv in enumerate(levels):
        a, _ = ctx_s.mq_eval_level(l, 0, lv.N)
        b, _ = ctx_p.mq_eval_level(l, 0, lv.N)
        ref = _oracle(levels, zs, ds, DECAYS, 2, name, l)
        e = np.abs(a[..., 1:3] - ref[..., 1:3]) / np.abs(ref[..., 1:2])
        d = np.abs(a[..., 1:3] - b[..., 1:3]) / np.abs(b[..., 1:2])
        print(f"problem 2 streaming tier ({name}), level {l}: vs oracle {e.max():.2e}, vs per-sample tier {d.max():.2e}")
        assert e.max() <= 1e-10 and d.max() <= 1e-10
    ctx_s.close()
    ctx_p.close()


def test_streaming_tier_rejects_the_reaction_term_in_fp64(B):
    ctx, _, _ = make_ctx(B, LEVELS, prec=0)
    ctx.mq_set_level_config(2, 1, 0, 0)
    with pytest.raises(B.MQError) as e:
        ctx.mq_eval_level(2, 0, 1)
    assert e.value.status == B.MQ_EINVAL
    ctx.mq_set_level_config(2, -1, 0, 0)  # by mesh size: the per-sample kernel
    ps, _ = ctx.mq_eval_level(2, 0, 1)
    assert np.all(np.isfinite(ps))
    ctx.close()


def test_functional_with_reuse_across_levels(B):
    # shared shifts and nested points (the reuse scheme) with the functional: the store carries
    # G values, level l >= 1 takes G^{l-1} from level l-1
    levels = [Level(8, 8, 16, 16, 8, 2), Level(16, 8, 16, 16, 4, 2), Level(32, 8, 16, 16, 2, 2)]
    mbits = 3
    ctx = B.Context(0)
    ctx.mq_set_islands(16, *DECAYS)
    ctx.mq_set_levels(levels)
    z = lattice.embedded_cbc(1, mbits, 16, 4.0 / 3.0)
    ds = shared_shifts(41, levels)
    for l in range(len(levels)):
        ctx.mq_set_lattice_embedded(l, z, mbits)
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(B.MQ_PREC_MIXED, 1e-10)
    ctx.mq_set_qoi(B.MQ_QOI_FUNCTIONAL)
    ctx.mq_set_reuse(1)
    got = [ctx.mq_eval_level(l, 0, lv.N)[0] for l, lv in enumerate(levels)]
    for r in range(2):
        ref = mlqmc.shared_samples(levels, z, mbits, ds[-1][r], list(range(levels[0].N)), 1.0, DECAYS, 2,
                                   qoi="functional")
        for l, lv in enumerate(levels):
            g, o = got[l][r], ref[l, : lv.N]
            assert np.all(np.abs(g[:, 1] - o[:, 1]) <= 1e-10 * np.abs(o[:, 1])), (l, r)
            if l:
                assert np.array_equal(g[:, 2], got[l - 1][r][: lv.N, 1])
    # switching the quantity resets the sums and switches the scheme off
    ctx.mq_set_qoi(B.MQ_QOI_EIGENVALUE)
    with pytest.raises(B.MQError):
        ctx.mq_estimate()
    ctx.close()


def test_problem2_workload_sampled(B):
    # the paper-size workload of the second test problem (levels 0-3, 2048 .. 256 points x 8
    # shifts) in the benchmark's launch configuration, edge and random samples against the oracle
    wl = WORKLOADS["paper_p2_h8_64"]
    ctx = B.Context(0)
    ctx.mq_set_islands(max(lv.s for lv in wl.levels), *wl.decays)
    ctx.mq_set_levels(wl.levels)
    zs = [lattice.cbc(lv.N, lv.s, wl.decay) for lv in wl.levels]
    ds = shifts(wl.seed, wl.levels)
    for l in range(len(wl.levels)):
        ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(B.MQ_PREC_MIXED)
    rng = np.random.default_rng(8)
    for l, lv in enumerate(wl.levels):
        ps, _ = ctx.mq_eval_level(l, 0, lv.N)
        assert np.all(np.isfinite(ps))
        picks = [(0, 0), (lv.R - 1, lv.N - 1), (int(rng.integers(lv.R)), int(rng.integers(lv.N)))]
        pv = wl.levels[l - 1] if l else None
        for r, k in picks:
            ref = mlqmc.level_samples(lv, pv, zs[l], ds[l][r : r + 1], [k], wl.a0, wl.coef_decay, wl.family)[0, 0]
            g = ps[r, k]
            assert abs(g[0] - ref[0]) <= 1e-12 * abs(ref[0])
            assert abs(g[1] - ref[1]) <= wl.tol * abs(ref[1]), (l, r, k, g, ref)
            assert abs(g[3] - ref[3]) <= 2 * wl.tol * abs(ref[1])
    m, se, _, _ = ctx.mq_estimate()
    print(f"paper_p2_h8_64: estimate {m:.10f} +- {se:.2e}")
    assert np.isfinite(m) and se > 0
    ctx.close()
