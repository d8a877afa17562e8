"""Pins for the oracle's lattice rules, CBC construction (Sec. 2.5) and estimator
(Algorithm 2, eq. sample_var, eq. tg-mlqmc)."""
import math

import numpy as np
import pytest

from oracle import lattice, mlqmc
from synthetic_inputs import Level


@pytest.mark.parametrize("N", [8, 64, 256, 1024])
def test_first_component_is_one(N):
    assert lattice.cbc(N, 3)[0] == 1


@pytest.mark.parametrize("N", [4, 16, 128])
def test_one_dimensional_error_closed_form(N):
    # sum_k B2(k/N) = 1/(6N), so e^2 = gamma_1/(6 N^2) for z = 1
    assert lattice.cbc_error2([1], N, [1.0]) == pytest.approx(1.0 / (6 * N * N), rel=1e-12)
    assert lattice.cbc_error2([1], N, [0.25]) == pytest.approx(0.25 / (6 * N * N), rel=1e-12)


@pytest.mark.parametrize("N,s", [(16, 4), (32, 3), (64, 4)])
def test_cbc_is_componentwise_argmin(N, s):
    gamma = [(j + 1) ** -2.0 for j in range(s)]
    z = lattice.cbc(N, s)
    for j in range(1, s):
        cands = [c for c in range(1, N // 2 + 1) if math.gcd(c, N) == 1]
        errs = [lattice.cbc_error2(list(z[:j]) + [c], N, gamma[: j + 1]) for c in cands]
        best = min(errs)
        assert lattice.cbc_error2(list(z[: j + 1]), N, gamma[: j + 1]) <= best + 1e-12
        # tie rule: no smaller candidate reaches the minimum
        first = next(c for c, e in zip(cands, errs) if e <= best + 1e-12)
        assert z[j] == first


def test_lattice_dual_exactness():
    # (1/N) sum_k exp(2 pi i m.(t_k + Delta)) = exp(2 pi i m.Delta) if m.z = 0 mod N, else 0
    N, s = 64, 3
    z = lattice.cbc(N, s)
    rng = np.random.default_rng(5)
    delta = rng.random(s)
    Y = lattice.points(z, N, delta, np.arange(N)) + 0.5
    for m in [(1, 0, 0), (0, 1, 1), (2, -1, 3), (int(z[1]), -1, 0), (5, 7, -2), (N, 0, 0)]:
        m = np.array(m)
        val = np.exp(2j * np.pi * (Y @ m)).mean()
        if int(m @ z) % N == 0:
            assert abs(val - np.exp(2j * np.pi * (m @ delta))) < 1e-12
        else:
            assert abs(val) < 1e-12


def test_lattice_integrates_low_order_trig_product_exactly():
    # prod_j (1 + alpha_j cos(2 pi m_j x_j)) has integral 1; exact when no nonzero m with
    # |m_j| <= 1 lies in the dual lattice
    N, s = 128, 3
    z = lattice.cbc(N, s)
    import itertools
    dual_free = all(int(np.dot(m, z)) % N != 0
                    for m in itertools.product((-1, 0, 1), repeat=s) if any(m))
    assert dual_free
    Y = lattice.points(z, N, np.array([0.1, 0.7, 0.33]), np.arange(N)) + 0.5
    f = np.prod(1 + np.array([0.5, 0.3, 0.2]) * np.cos(2 * np.pi * Y), axis=1)
    assert abs(f.mean() - 1.0) < 1e-13
    # and a rule that is not dual-free misses: z = (1, 1, 1) has m = (1, -1, 0) in its dual
    Y = lattice.points(np.array([1, 1, 1]), N, np.array([0.1, 0.7, 0.33]), np.arange(N)) + 0.5
    f = np.prod(1 + np.array([0.5, 0.3, 0.2]) * np.cos(2 * np.pi * Y), axis=1)
    assert abs(f.mean() - 1.0) > 1e-3


def test_points_range_and_origin():
    z = np.array([1, 3, 5])
    Y = lattice.points(z, 16, np.zeros(3), np.arange(16))
    assert np.all(Y >= -0.5) and np.all(Y < 0.5)
    assert np.all(Y[0] == -0.5)
    Y = lattice.points(z, 16, np.array([0.99, 0.5, 0.0]), [3])
    assert np.allclose(Y[0], [np.mod(3 / 16 + 0.99, 1) - 0.5, np.mod(9 / 16 + 0.5, 1) - 0.5, 15 / 16 - 0.5])


def test_estimator_worked_example():
    # two levels, two shifts: Q^(r)_0 = (1, 3), Q^(r)_1 = (0.5, 0.25)
    est, se, qhat, vhat = mlqmc.estimate([[1.0, 3.0], [0.5, 0.25]])
    assert qhat == [2.0, 0.375]
    assert vhat == [1.0, 0.015625]
    assert est == 2.375
    assert se == pytest.approx(np.sqrt(1.015625))


def test_estimator_needs_two_shifts():
    with pytest.raises(ValueError):
        mlqmc.estimate([[1.0]])


def test_shift_means():
    d = np.array([[1.0, 2.0, 3.0, 4.0], [0.0, 0.0, 0.0, 8.0]])
    assert np.allclose(mlqmc.shift_means(d, 4), [2.5, 2.0])


def test_sample_level_difference_uses_one_coarse_pair():
    from oracle import twogrid
    lv = Level(32, 8, 8, 3, 16, 2)
    pv = Level(16, 8, 4, 2, 16, 2)
    y = np.array([0.2, -0.1, 0.3, 0.05, -0.4, 0.1, 0.2, -0.2])
    lam_H, lam_l, lam_p, d = mlqmc.sample_level(lv, pv, y)
    lH, uH = twogrid.coarse_pair(8, y[:3])
    assert lam_H == lH
    assert lam_l == twogrid.twogrid_update(32, y[:8], lH, uH, 8)
    assert lam_p == twogrid.twogrid_update(16, y[:4], lH, uH, 8)
    assert d == lam_l - lam_p
    # level 0: lambda^{-1} = 0
    assert mlqmc.sample_level(pv, None, y)[3] == mlqmc.sample_level(pv, None, y)[1]


# ---- embedded lattice rules and the shared-shift reuse scheme (Sec. 2.5; Sec. 4.3 after Alg. 2)

@pytest.mark.parametrize("m,s", [(3, 3), (5, 4), (7, 5)])
def test_embedded_cbc_with_one_size_is_the_fixed_size_cbc(m, s):
    # one N: the worst ratio orders the candidates as the error itself, over the same candidates
    assert np.array_equal(lattice.embedded_cbc(m, m, s), lattice.cbc(1 << m, s))


def test_embedded_cbc_brute_force():
    # every component re-derived with the plain double-loop error formula: the smallest candidate
    # whose worst ratio over N = 2, 4, 8, 16 is (within 1e-12) the minimum
    m_min, m_max, s = 1, 4, 4
    gamma = [(j + 1) ** -2.0 for j in range(s)]
    z = lattice.embedded_cbc(m_min, m_max, s)
    cands = list(range(1, (1 << m_max) // 2, 2))
    for j in range(s):
        worst = []
        for c in cands:
            ratios = []
            for m in range(m_min, m_max + 1):
                N = 1 << m
                errs = [lattice.cbc_error2(list(z[:j]) + [cc], N, gamma[: j + 1]) for cc in cands]
                ratios.append(lattice.cbc_error2(list(z[:j]) + [c], N, gamma[: j + 1]) / min(errs))
            worst.append(max(ratios))
        best = min(worst)
        assert z[j] == next(c for c, w in zip(cands, worst) if w <= best + 1e-12)


def test_embedded_points_are_nested_rules():
    # the first 2^m points in radical-inverse order are the 2^m-point rule, for every m
    m_max, s = 6, 3
    z = lattice.embedded_cbc(2, m_max, s)
    delta = np.array([0.3, 0.71, 0.05])
    for m in range(0, m_max + 1):
        N = 1 << m
        emb = lattice.embedded_points(z, m_max, delta, np.arange(N))
        rule = lattice.points(z, N, delta, np.arange(N))
        key = lambda P: sorted(map(tuple, np.round(P, 12)))
        assert key(emb) == key(rule)
    assert np.array_equal(np.sort(lattice.bit_reverse(np.arange(64), 6)), np.arange(64))
    assert lattice.bit_reverse(1, 6) == 32 and lattice.bit_reverse(3, 6) == 48


def test_shared_samples_equal_algorithm_2_recomputed():
    # reusing the level-0 eigenpair and the level below's value gives exactly what Algorithm 2
    # computes from scratch at the same point with H_l = h_0 and S_l = s_0
    levels = [Level(8, 8, 4, 4, 16, 2), Level(16, 8, 8, 4, 8, 2), Level(32, 8, 16, 4, 4, 2)]
    z = lattice.embedded_cbc(2, 4, 16)
    delta = np.random.default_rng(0).random(16)
    ks = [0, 1, 3, 5, 9]
    out = mlqmc.shared_samples(levels, z, 4, delta, ks)
    Y = lattice.embedded_points(z, 4, delta, ks)
    for i, k in enumerate(ks):
        for l, lv in enumerate(levels):
            if k >= lv.N:
                assert np.all(np.isnan(out[l, i]))
                continue
            ref = mlqmc.sample_level(lv, levels[l - 1] if l else None, Y[i])
            assert np.array_equal(out[l, i], np.array(ref))


def test_shared_shift_estimate():
    # per-shift totals 1.0+0.1, 2.0-0.1, 3.0+0.3: mean 2.1, sample variance of the mean
    q = np.array([[1.0, 2.0, 3.0], [0.1, -0.1, 0.3]])
    m, se, qhat, vhat = mlqmc.estimate_shared(q)
    tot = np.array([1.1, 1.9, 3.3])
    assert m == pytest.approx(2.1, rel=1e-15)
    assert se == pytest.approx(math.sqrt(((tot - 2.1) ** 2).sum() / 6.0), rel=1e-14)
    assert qhat[0] == pytest.approx(2.0) and qhat[1] == pytest.approx(0.1)
    # one level: the same as the independent-level estimate
    m1, se1, _, _ = mlqmc.estimate_shared(q[:1])
    m2, se2, _, _ = mlqmc.estimate([q[0]])
    assert m1 == pytest.approx(m2, rel=1e-15) and se1 == pytest.approx(se2, rel=1e-14)
    with pytest.raises(ValueError):
        mlqmc.estimate_shared(q[:, :1])


# ---- the adaptive algorithm (Sec. 4.2, Giles-Waterhouse choice of N_l and L)

@pytest.mark.parametrize("bdecay", [4.0, 2.0])
def test_adaptive_decisions_follow_the_closed_form(bdecay):
    # a synthetic level whose differences are b_l + a_l w_r at point 0 and b_l elsewhere: after N
    # points Q^(r)_l = b_l + a_l w_r / N, so Vhat_l(N) = (a_l / N)^2 S_w and Qhat_l = b_l + a_l wbar / N
    # in closed form; the greedy rule is re-derived from those formulas and compared
    R = 4
    w = np.array([1.0, -1.0, 2.0, 0.0])
    wbar, Sw = w.mean(), ((w.mean() - w) ** 2).sum() / (R * (R - 1))
    a = [2.0 ** -l for l in range(5)]
    b = [bdecay ** -l for l in range(5)]  # bdecay 2: the bias test fails until level 4
    cost = [4.0 ** l for l in range(5)]
    eps, alpha, n_init = 0.05, 2.0, 2

    def evaluate(l, k0, k1):
        d = np.full((R, k1 - k0), b[l])
        if k0 == 0 and k1 > 0:
            d[:, 0] += a[l] * w
        return d

    res = mlqmc.adaptive(evaluate, cost, R, eps, alpha, n_init)
    # re-derivation
    N, hist = [n_init] * 3, [(0, 2), (1, 2), (2, 2)]
    V = lambda l: (a[l] / N[l]) ** 2 * Sw
    Q = lambda l: b[l] + a[l] * wbar / N[l]
    while True:
        while sum(V(l) for l in range(len(N))) > eps ** 2 / 2:
            sc = [V(l) / (cost[l] * N[l]) for l in range(len(N))]
            l = sc.index(max(sc))
            N[l] *= 2
            hist.append((l, N[l]))
        L = len(N) - 1
        if max(abs(Q(L)), abs(Q(L - 1)) / 4.0) <= 3.0 * eps / math.sqrt(2.0):
            break
        N.append(n_init)
        hist.append((L + 1, n_init))
    assert res["history"] == hist and res["N"] == N and res["converged"]
    assert res["L"] == len(N) - 1 == (2 if bdecay == 4.0 else 4)
    assert res["mean"] == pytest.approx(sum(Q(l) for l in range(len(N))), rel=1e-13)
    assert res["std_err"] == pytest.approx(math.sqrt(sum(V(l) for l in range(len(N)))), rel=1e-12)
    # a cap on the points per level that blocks every doubling ends the run unconverged
    capped = mlqmc.adaptive(evaluate, cost, R, 1e-6, alpha, n_init, n_max=[4] * 5)
    assert not capped["converged"] and all(n <= 4 for n in capped["N"])
