"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: integer and lattice-point work bit-exact; coefficients 1e-14 absolute (a ~ 1);
operator applications 1e-13 relative; coarse eigenvalues 1e-12 relative, coarse eigenvectors ten
times the eigen-residual target; two-grid
eigenvalues and level differences 1e-10 relative (FP64 and mixed paths), the workload target.
"""
import numpy as np
import pytest

from oracle import fem, lattice, mlqmc, twogrid
from synthetic_inputs import WORKLOADS, Level, random_cell_coefficients, random_points, random_vectors, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_LAMBDA = 1e-10
TOL_EIG = 1e-8  # relative eigen-residual target of the coarse eigensolve when mq_eval_point returns u_H


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


def make_ctx(B, levels, seed=0, prec=0, s_max=None):
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, s_max or max(lv.s for lv in levels), 0, 2.0)
    ctx.mq_set_levels(levels)
    zs, ds = [], shifts(seed, levels)
    for l, lv in enumerate(levels):
        z = lattice.cbc(lv.N, lv.s)
        zs.append(z)
        ctx.mq_set_lattice(l, z)
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    return ctx, zs, ds


def test_lattice_points_bit_exact(B):
    lv = Level(16, 8, 16, 4, 256, 3)
    ctx, zs, ds = make_ctx(B, [lv])
    k0, k1 = 5, 101
    d = torch.empty((lv.R, k1 - k0, lv.s), dtype=torch.float64, device="cuda")
    ctx.mq_lattice_points_device(0, k0, k1, d)
    got = d.cpu().numpy()
    for r in range(lv.R):
        ref = lattice.points(zs[0], lv.N, ds[0][r], np.arange(k0, k1))
        assert np.array_equal(got[r], ref)


@pytest.mark.parametrize("n,s", [(2, 1), (8, 16), (16, 37), (32, 64)])
def test_coefficients_match_oracle(B, n, s):
    ctx, _, _ = make_ctx(B, [Level(n, n, s, s, 8, 2)])
    Y = random_points(n + s, 5, s)
    dY = torch.from_numpy(Y).cuda()
    da = torch.empty((5, 2 * n * n), dtype=torch.float64, device="cuda")
    ctx.mq_coefficients_device(n, s, dY, 5, s, da)
    got = da.cpu().numpy()
    for b in range(5):
        assert np.abs(got[b] - fem.coefficient(n, Y[b])).max() < 1e-14


@pytest.mark.parametrize("n,s,nb,offset", [(2, 1, 3, 0), (4, 5, 9, 1), (8, 16, 5, 0), (16, 37, 130, 0),
                                           (32, 128, 200, 0), (16, 300, 7, 1), (64, 300, 130, 0)])
def test_tensor_core_coefficients_match_oracle(B, n, s, nb, offset):
    # mixed precision: exact BF16 slices on tcgen05 tensor cores, FP64-accurate result; ragged
    # sample counts (130, 200: two 128-row tiles), triangle counts below one 64-wide tile (8, 32),
    # K not a multiple of 16 (37), several 128-wide exact accumulation chunks (300), more tiles
    # than SMs (64 x 64 mesh, 130 samples: 256 tiles, so the persistent CTAs take several each),
    # and an output 8 bytes off 16-byte alignment (offset 1)
    ctx, _, _ = make_ctx(B, [Level(n, n, s, s, 8, 2)], prec=1)
    Y = random_points(n + s + nb, nb, s)
    dY = torch.from_numpy(Y).cuda()
    buf = torch.empty(nb * 2 * n * n + offset, dtype=torch.float64, device="cuda")
    da = buf[offset:].view(nb, 2 * n * n)
    ctx.mq_coefficients_device(n, s, dY, nb, s, da)
    got = da.cpu().numpy()
    ref = np.stack([fem.coefficient(n, Y[b]) for b in range(nb)])
    assert np.abs(got - ref).max() < 5e-15


@pytest.mark.parametrize("n,s,nb,decay", [(128, 128, 3, 2.0), (128, 100, 130, 2.0), (256, 1024, 3, 2.0),
                                           (256, 1024, 2, 4.0 / 3.0), (512, 300, 1, 2.0)])
def test_separable_coefficients_match_oracle(B, n, s, nb, decay):
    # mixed precision on meshes 1/128 and finer: the workload family is evaluated separably (the
    # terms grouped by k1: an FP64 first stage and a tensor-core second stage over the k1 values);
    # ragged row counts (130 samples x 128 rows), the decay below 2 takes a smaller slice scale
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, s, 0, decay)
    ctx.mq_set_levels([Level(n, n, s, s, 8, 2)])
    ctx.mq_set_precision(1)
    Y = random_points(n + s + nb, nb, s)
    dY = torch.from_numpy(Y).cuda()
    da = torch.empty((nb, 2 * n * n), dtype=torch.float64, device="cuda")
    ctx.mq_coefficients_device(n, s, dY, nb, s, da)
    got = da.cpu().numpy()
    for b in range(nb):
        ref = fem.coefficient(n, Y[b], 1.0, decay)
        assert np.abs(got[b] - ref).max() < 5e-15, (b, np.abs(got[b] - ref).max())
    # a truncation shorter than the table's (fewer k1 values) reads a prefix of the term lists
    k = s // 3
    ctx.mq_coefficients_device(n, k, dY, nb, s, da)
    got = da.cpu().numpy()
    assert np.abs(got[0] - fem.coefficient(n, Y[0][:k], 1.0, decay)).max() < 5e-15
    ctx.close()


@pytest.mark.parametrize("n", [2, 4, 8, 16, 64])
def test_operator_apply_matches_assembled_matrices(B, n):
    ctx, _, _ = make_ctx(B, [Level(8, 8, 1, 1, 8, 2)])
    nb = 3
    a = random_cell_coefficients(n, nb, n).reshape(nb, -1)
    x = random_vectors(n + 1, nb, (n - 1) ** 2)
    da, dx = torch.from_numpy(a).cuda(), torch.from_numpy(x).cuda()
    dy = torch.empty_like(dx)
    sigma = 19.5
    for which in range(3):
        ctx.mq_apply_operator_device(n, nb, da, which, sigma, dx, dy)
        got = dy.cpu().numpy()
        for b in range(nb):
            A, M = fem.assemble(n, a[b])
            ref = [A @ x[b], M @ x[b], A @ x[b] - sigma * (M @ x[b])][which]
            assert np.abs(got[b] - ref).max() <= 1e-13 * np.abs(ref).max()


POINT_CASES = [
    # (levels, level index): single level, two levels with a previous fine mesh, direct level 0
    ([Level(16, 8, 16, 4, 8, 2)], 0),
    ([Level(16, 8, 16, 4, 8, 2), Level(32, 8, 32, 6, 8, 2)], 1),
    ([Level(32, 16, 8, 4, 8, 2), Level(64, 16, 16, 4, 8, 2)], 1),
    ([Level(8, 8, 4, 4, 8, 2)], 0),
    ([Level(8, 8, 4, 4, 8, 2), Level(32, 8, 16, 4, 8, 2)], 1),
]


@pytest.mark.parametrize("case", range(len(POINT_CASES)))
@pytest.mark.parametrize("prec", [0, 1])
def test_eval_point_matches_oracle(B, case, prec):
    levels, l = POINT_CASES[case]
    ctx, _, _ = make_ctx(B, levels, prec=prec)
    lv = levels[l]
    pv = levels[l - 1] if l > 0 else None
    for y in random_points(100 + case, 3, lv.s):
        lH, lh, lp, u = ctx.mq_eval_point(l, y, want_u=True)
        rH, rh, rp, rd = mlqmc.sample_level(lv, pv, y)
        assert lH == pytest.approx(rH, rel=1e-12)
        assert lh == pytest.approx(rh, rel=TOL_LAMBDA)
        assert lp == pytest.approx(rp, rel=TOL_LAMBDA, abs=0 if pv else 1e-300)
        _, uref = twogrid.coarse_pair(lv.n_coarse, y[: lv.S])
        # the eigenvector is accurate to the eigen-residual target (1e-8 when it is returned) over the
        # relative spectral gap (about 1.5 for these coefficients); the eigenvalue to its square
        assert np.abs(u - uref).max() < 10 * TOL_EIG * np.abs(uref).max()


def _check_level(per_sample, ref):
    # per-sample (lambda_H, lambda^l, lambda^{l-1}, difference)
    assert np.all(np.abs(per_sample[..., 0] - ref[..., 0]) <= 1e-12 * np.abs(ref[..., 0]))
    assert np.all(np.abs(per_sample[..., 1] - ref[..., 1]) <= TOL_LAMBDA * np.abs(ref[..., 1]))
    assert np.all(np.abs(per_sample[..., 2] - ref[..., 2]) <= TOL_LAMBDA * np.abs(ref[..., 2]))
    # the difference is checked relative to the eigenvalues it is formed from
    assert np.all(np.abs(per_sample[..., 3] - ref[..., 3]) <= 2 * TOL_LAMBDA * np.abs(ref[..., 1]))


@pytest.mark.parametrize("prec", [0, 1])
def test_eval_level_single_level_workload(B, prec):
    wl = WORKLOADS["qmc_h16_s16"]
    lv = wl.levels[0]
    ctx, zs, ds = make_ctx(B, wl.levels, seed=wl.seed, prec=prec)
    k0, k1 = 3, 40  # several warm-start chains and a ragged tail
    ps, sums = ctx.mq_eval_level(0, k0, k1)
    ref = mlqmc.level_samples(lv, None, zs[0], ds[0], list(range(k0, k1)))
    _check_level(ps, ref)
    assert np.allclose(sums, ref[..., 3].sum(axis=1), rtol=1e-12, atol=0)
    m, se, lm, lvv = ctx.mq_estimate()
    om, ose, _, _ = mlqmc.estimate([mlqmc.shift_means(ref[..., 3], k1 - k0)])
    assert m == pytest.approx(om, rel=1e-12)
    # SE is 1-Lipschitz in the scaled deviations (Qhat - Q^(r)) / sqrt(R (R - 1)): a per-sample
    # error of at most e moves it by at most 2 e / sqrt(R - 1) (plus its own rounding)
    e = np.abs(ps[..., 3] - ref[..., 3]).max()
    assert abs(se - ose) <= 2.0 * e / np.sqrt(lv.R - 1) + 1e-14 * ose
    assert se == pytest.approx(ose, rel=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_eval_level_multilevel_workload_sampled(B, prec):
    wl = WORKLOADS["mlqmc4_h16_128"]
    ctx, zs, ds = make_ctx(B, wl.levels, seed=wl.seed, prec=prec)
    for l, (k0, k1) in [(1, (0, 3)), (2, (7, 9)), (3, (0, 1))]:
        lv, pv = wl.levels[l], wl.levels[l - 1]
        ps, _ = ctx.mq_eval_level(l, k0, k1)
        ref = mlqmc.level_samples(lv, pv, zs[l], ds[l], list(range(k0, k1)))
        _check_level(ps, ref)


def test_full_size_level_sampled_outputs(B):
    # the finest level of the 4-level workload at its full point count (8,192 samples), in the
    # launch configuration of the benchmark; a few samples checked against the oracle
    wl = WORKLOADS["mlqmc4_h16_128"]
    ctx, zs, ds = make_ctx(B, wl.levels, seed=wl.seed, prec=1)
    l = 3
    lv, pv = wl.levels[l], wl.levels[l - 1]
    ps, sums = ctx.mq_eval_level(l, 0, lv.N)
    rng = np.random.default_rng(0)
    picks = [(int(r), int(k)) for r, k in zip(rng.integers(0, lv.R, 4), rng.integers(0, lv.N, 4))]
    picks.append((lv.R - 1, lv.N - 1))
    for r, k in picks:
        ref = mlqmc.level_samples(lv, pv, zs[l], ds[l][r : r + 1], [k])[0, 0]
        _check_level(ps[r, k][None, None], ref[None, None])
    assert np.allclose(sums, ps[..., 3].sum(axis=1), rtol=1e-12)
    assert np.all(np.isfinite(ps))


def test_warm_start_does_not_change_results(B):
    lv = Level(16, 8, 16, 4, 64, 2)
    ctx, zs, ds = make_ctx(B, [lv])
    ps, _ = ctx.mq_eval_level(0, 0, 20)
    Y = lattice.points(zs[0], lv.N, ds[0][1], np.arange(20))
    for k in (0, 1, 7, 19):
        lH, lh, _ = ctx.mq_eval_point(0, Y[k])  # a single cold-started sample
        # both starts converge to the same eigenpair; lambda^h then differs by the solve
        # tolerance's effect only (first order, ~3e-7 times the relative residual)
        assert ps[1, k, 0] == pytest.approx(lH, rel=1e-12)
        assert ps[1, k, 1] == pytest.approx(lh, rel=1e-11)


def test_device_outputs_equal_host_outputs(B):
    lv = Level(32, 8, 16, 4, 64, 3)
    ctx, _, _ = make_ctx(B, [lv])
    ps, sums = ctx.mq_eval_level(0, 4, 30)
    d_ps = torch.empty((lv.R, 26, 4), dtype=torch.float64, device="cuda")
    d_s = torch.empty(lv.R, dtype=torch.float64, device="cuda")
    ctx.mq_eval_level_device(0, 4, 30, d_ps, d_s)
    assert np.array_equal(d_ps.cpu().numpy(), ps)
    assert np.array_equal(d_s.cpu().numpy(), sums)


def test_degenerate_direct_level(B):
    # H = h and S = s: the level value is the fine eigenvalue itself
    lv = Level(16, 16, 6, 6, 16, 2)
    ctx, _, _ = make_ctx(B, [lv])
    y = random_points(5, 1, 6)[0]
    lH, lh, _ = ctx.mq_eval_point(0, y)
    ref = twogrid.fine_eigenvalue(16, y)
    assert lH == pytest.approx(ref, rel=1e-12) and lh == lH


def test_empty_range_and_errors(B):
    lv = Level(16, 8, 16, 4, 64, 1)
    ctx, _, _ = make_ctx(B, [lv])
    ps, sums = ctx.mq_eval_level(0, 10, 10)
    assert ps.shape == (1, 0, 4) and sums[0] == 0.0
    with pytest.raises(B.MQError) as e:
        ctx.mq_eval_level(0, 0, 65)
    assert e.value.status == B.MQ_EINVAL
    ctx.mq_eval_level(0, 0, 2)
    with pytest.raises(B.MQError) as e:  # one shift: no standard error
        ctx.mq_estimate()
    assert e.value.status == B.MQ_EINVAL
    with pytest.raises(B.MQError) as e:
        ctx.mq_set_shifts(0, np.full((1, 16), 1.0))
    assert e.value.status == B.MQ_EINVAL
    ctx2 = B.Context(0)
    ctx2.mq_set_coefficient(1.0, 16)
    ctx2.mq_set_levels([lv])
    with pytest.raises(B.MQError) as e:
        ctx2.mq_eval_level(0, 0, 1)
    assert e.value.status == B.MQ_ESTATE


def test_nonpositive_coefficient_is_rejected(B):
    # a0 = 0.2 with y = -1/2 sign(psi_j) drives a below zero somewhere (Assumption A1)
    ctx = B.Context(0)
    ctx.mq_set_coefficient(0.2, 16)
    ctx.mq_set_levels([Level(16, 8, 16, 4, 8, 2)])
    with pytest.raises(B.MQError) as e:
        ctx.mq_eval_point(0, np.full(16, -0.5))
    assert e.value.status == B.MQ_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
def test_tiers_agree_and_match_oracle(B, prec):
    # every fine solve forced into the batched streaming tier (meshes 1/16 .. 1/64, including the
    # tier's single-CTA path for meshes up to 1/32) versus forced into the per-sample kernel
    levels = [Level(16, 8, 16, 4, 32, 3), Level(32, 8, 32, 6, 32, 3), Level(64, 16, 64, 8, 32, 3)]
    ctx_s, zs, ds = make_ctx(B, levels, seed=11, prec=prec)
    ctx_c, _, _ = make_ctx(B, levels, seed=11, prec=prec)
    ctx_s.mq_set_tier(2)
    ctx_c.mq_set_tier(4096)
    for l in range(3):
        k0, k1 = 5, 9
        ps_s, _ = ctx_s.mq_eval_level(l, k0, k1)
        ps_c, _ = ctx_c.mq_eval_level(l, k0, k1)
        assert np.all(np.abs(ps_s[..., 1:3] - ps_c[..., 1:3]) <= 1e-10 * np.abs(ps_c[..., 1:3]) + 1e-300)
        ref = mlqmc.level_samples(levels[l], levels[l - 1] if l else None, zs[l], ds[l], list(range(k0, k1)))
        _check_level(ps_s, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_smoothing_variants_agree(B, prec):
    # V(1,1) and V(2,2) precondition the same systems: the eigenvalues agree to the solver
    # tolerances, in both tiers (meshes 1/16 in the per-sample kernel, 1/64 streamed)
    levels = [Level(16, 8, 16, 4, 16, 2), Level(64, 16, 64, 8, 16, 2)]
    out = []
    for nu in (1, 2):
        ctx, zs, ds = make_ctx(B, levels, seed=5, prec=prec)
        ctx.mq_set_smoothing(nu)
        out.append([ctx.mq_eval_level(l, 2, 6)[0] for l in range(2)])
    for l in range(2):
        a, b = out[0][l], out[1][l]
        assert np.all(np.abs(a[..., :3] - b[..., :3]) <= 1e-10 * np.abs(b[..., :3]) + 1e-300)


def test_eval_levels_device_matches_level_by_level(B):
    # the concurrent multi-level call (one internal context, stream and host thread per level)
    # gives the per-level results, sums and estimate of the level-by-level calls
    levels = [Level(16, 8, 16, 4, 32, 2), Level(32, 8, 32, 6, 32, 2), Level(64, 16, 64, 8, 16, 2)]
    ctx_a, _, _ = make_ctx(B, levels, seed=9, prec=1)
    ctx_b, _, _ = make_ctx(B, levels, seed=9, prec=1)
    out_a = [torch.empty((lv.R, lv.N, 4), dtype=torch.float64, device="cuda") for lv in levels]
    sum_a = [torch.empty(lv.R, dtype=torch.float64, device="cuda") for lv in levels]
    # warm-up calls build the coefficient tables (each internal context builds its own), then
    # the compared calls
    ctx_a.mq_eval_levels_device([0, 1, 2], out_a, sum_a)
    for l, lv in enumerate(levels):
        ctx_b.mq_eval_level_device(l, 0, lv.N, None, None)
    ctx_a.mq_reset_sums()
    ctx_b.mq_reset_sums()
    ctx_a.mq_eval_levels_device([0, 1, 2], out_a, sum_a)
    for l, lv in enumerate(levels):
        out_b = torch.empty((lv.R, lv.N, 4), dtype=torch.float64, device="cuda")
        sum_b = torch.empty(lv.R, dtype=torch.float64, device="cuda")
        ctx_b.mq_eval_level_device(l, 0, lv.N, out_b, sum_b)
        assert torch.equal(out_a[l], out_b)
        assert torch.equal(sum_a[l], sum_b)
    ma, sa, _, _ = ctx_a.mq_estimate()
    mb, sb, _, _ = ctx_b.mq_estimate()
    assert ma == mb and sa == sb
    assert ctx_a.mq_get_launch_count() == ctx_b.mq_get_launch_count()
    # a second call reuses the internal contexts; a setter rebuilds them
    ctx_a.mq_eval_levels_device([2, 0], [out_a[2], out_a[0]], None)
    ctx_a.mq_set_tier(0)
    ctx_a.mq_eval_levels_device([1], [out_a[1]], None)
    with pytest.raises(B.MQError) as e:
        ctx_a.mq_eval_levels_device([1, 1], None, None)
    assert e.value.status == B.MQ_EINVAL


def _problem1_ctx(B, prec):
    # the paper's first test problem: psi_j = j^-p sin(j pi x1) sin((j+1) pi x2), p = 4/3
    wl = WORKLOADS["paper_p1_h8_64"]
    ctx = B.Context(0)
    ctx.mq_set_coefficient(wl.a0, max(lv.s for lv in wl.levels), wl.family, wl.decay)
    ctx.mq_set_levels(wl.levels)
    zs = [lattice.cbc(lv.N, lv.s, wl.decay) for lv in wl.levels]
    ds = shifts(wl.seed, wl.levels)
    for l in range(len(wl.levels)):
        ctx.mq_set_lattice(l, zs[l])
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    return wl, ctx, zs, ds


@pytest.mark.parametrize("prec", [0, 1])
def test_paper_problem1_family_matches_oracle(B, prec):
    # the FP64 path runs the fine solves of mesh 1/64 in the per-sample kernel with its workspace
    # in a global scratch of back-to-back slabs (a slab size off 16-byte alignment once let one
    # block's fine solve overwrite the next block's coarse eigenvector here)
    wl, ctx, zs, ds = _problem1_ctx(B, prec)
    # centroid coefficients (FP64 GEMM, or the tensor-core split on the mixed path)
    Y = random_points(31, 6, 64)
    da = torch.empty((6, 2 * 16 * 16), dtype=torch.float64, device="cuda")
    ctx.mq_coefficients_device(16, 64, torch.from_numpy(Y).cuda(), 6, 64, da)
    got = da.cpu().numpy()
    for b in range(6):
        assert np.abs(got[b] - fem.coefficient(16, Y[b], wl.a0, wl.decay, family=1)).max() < 1e-14
    # the direct level 0 and two two-grid levels, several shifts and points
    for l, (k0, k1) in [(0, (0, 4)), (1, (5, 8)), (3, (0, 2))]:
        lv, pv = wl.levels[l], (wl.levels[l - 1] if l else None)
        ps, _ = ctx.mq_eval_level(l, k0, k1)
        ref = mlqmc.level_samples(lv, pv, zs[l], ds[l], list(range(k0, k1)), wl.a0, wl.decay, wl.family)
        _check_level(ps, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_iteration_caps_report_noconvergence(B, prec):
    # the error path of the solvers, forced on the host side by iteration caps: the call returns
    # MQ_ENOCONV, the per-sample flags and the statistics say which samples, and the outputs are
    # still written.  Per-sample tier (mesh 1/16) and streaming tier (mesh 1/64).
    levels = [Level(16, 8, 16, 4, 16, 2), Level(64, 16, 64, 8, 16, 2)]
    for l in range(2):
        ctx, zs, ds = make_ctx(B, levels, seed=3, prec=prec)
        ctx.mq_set_tier(32 if l else 0)
        ctx.mq_set_solver_options(0.0, 1, 1)  # one MINRES iteration, one refinement step
        with pytest.raises(B.MQNoConvergence) as e:
            ctx.mq_eval_level(l, 0, 4)
        assert e.value.status == B.MQ_ENOCONV
        st = ctx.mq_get_stats()
        assert st["noconv"] > 0 and st["samples"] == 2 * 4
        assert st["fine_iters_max"] <= 1
        d_ps = torch.full((2, 4, 4), float("nan"), dtype=torch.float64, device="cuda")
        with pytest.raises(B.MQNoConvergence):
            ctx.mq_eval_level_device(l, 0, 4, d_ps, None)
        assert torch.isfinite(d_ps).all()  # outputs written despite the caps
        ctx.close()
    # the coarse eigensolver cap: one LOBPCG iteration cannot reach the eigen-residual target
    ctx, _, _ = make_ctx(B, levels[:1], seed=3, prec=prec)
    ctx.mq_set_eig_options(0.0, 1)
    with pytest.raises(B.MQNoConvergence):
        ctx.mq_eval_level(0, 0, 4)
    st = ctx.mq_get_stats()
    assert st["noconv"] == st["samples"] == 8 and st["coarse_iters_max"] == 1
    # lifting the caps again restores convergence and the oracle's values
    ctx.mq_set_eig_options(0.0, 0)
    ps, _ = ctx.mq_eval_level(0, 0, 4)
    assert ctx.mq_get_stats()["noconv"] == 0
    ref = mlqmc.level_samples(levels[0], None, lattice.cbc(16, 16), shifts(3, levels)[0], list(range(4)))
    _check_level(ps, ref)
    ctx.close()


def test_autotuner_keeps_results_and_caches_its_choice(B, tmp_path):
    # the tuner times the candidate configurations of a level on a probe, applies the fastest and
    # stores it; the results stay those of the default configuration to the solver tolerances,
    # and the probes leave the estimator state untouched
    levels = [Level(16, 8, 16, 4, 32, 2), Level(32, 8, 32, 6, 32, 2), Level(64, 16, 64, 8, 16, 2)]
    ctx, zs, ds = make_ctx(B, levels, seed=13, prec=1)
    ref = [ctx.mq_eval_level(l, 0, 8)[0] for l in range(3)]
    before = [ctx.mq_get_sums(l) for l in range(3)]
    cache = str(tmp_path / "tune.txt")
    choices = [ctx.mq_autotune_level(l, 8, cache) for l in range(3)]
    for (sa, na), (sb, nb) in zip(before, [ctx.mq_get_sums(l) for l in range(3)]):
        assert na == nb and np.array_equal(sa, sb)
    for l, ch in enumerate(choices):
        assert ch["from_cache"] == 0 and ch["tried"] >= 6 and ch["ms"] > 0
        assert ch["threads"] in (64, 128, 256) and ch["nu"] in (1, 2)
    # meshes 1/16 .. 1/64 can run in either tier: both were timed
    assert all(ch["tier"] in (0, 1) and ch["tried"] == 12 for ch in choices)
    for l in range(3):
        got, _ = ctx.mq_eval_level(l, 0, 8)
        assert np.all(np.abs(got[..., :3] - ref[l][..., :3]) <= 1e-10 * np.abs(ref[l][..., :3]) + 1e-300)
    # a second context reads the choices from the cache without timing
    ctx2, _, _ = make_ctx(B, levels, seed=13, prec=1)
    for l in range(3):
        ch = ctx2.mq_autotune_level(l, 8, cache)
        assert ch["from_cache"] == 1 and (ch["tier"], ch["threads"], ch["nu"]) == (
            choices[l]["tier"], choices[l]["threads"], choices[l]["nu"])
    ctx.close()
    ctx2.close()
