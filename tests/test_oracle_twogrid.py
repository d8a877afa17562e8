"""Pins for the oracle's interpolation and two-grid-truncation step (Algorithm 1, Lemma 3.1,
Theorem 3.1)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, twogrid
from synthetic_inputs import random_points, random_vectors


def _coarse_constant_fine_coeff(n_c, n_f, a_c):
    """Fine per-triangle coefficient equal to that of the coarse triangle containing it."""
    c = fem.centroids(n_f)
    H = 1.0 / n_c
    ci = np.floor(c[:, 0] / H).astype(int)
    cj = np.floor(c[:, 1] / H).astype(int)
    lower = (c[:, 0] - ci * H) > (c[:, 1] - cj * H)
    t = np.where(lower, 0, 1) * n_c * n_c + cj * n_c + ci
    return a_c[t]


@pytest.mark.parametrize("n_c,n_f", [(2, 4), (4, 8), (4, 16), (8, 32)])
def test_interpolation_preserves_energy_and_mass(n_c, n_f):
    # V_H is a subspace of V_h: for a coefficient constant on coarse triangles the fine forms
    # restricted to interpolated coarse functions equal the coarse forms
    rng = np.random.default_rng(n_f)
    a_c = 0.3 + rng.random(2 * n_c * n_c)
    a_f = _coarse_constant_fine_coeff(n_c, n_f, a_c)
    A_c, M_c = fem.assemble(n_c, a_c)
    A_f, M_f = fem.assemble(n_f, a_f)
    P = twogrid.interpolation_matrix(n_c, n_f)
    for v in random_vectors(n_c, 3, (n_c - 1) ** 2):
        pv = P @ v
        assert abs(pv @ (A_f @ pv) - v @ (A_c @ v)) < 1e-12 * (v @ (A_c @ v))
        assert abs(pv @ (M_f @ pv) - v @ (M_c @ v)) < 1e-12 * (v @ (M_c @ v))
    # Galerkin identity P^T A_h P = A_H holds entry by entry
    assert abs(P.T @ A_f @ P - A_c).max() < 1e-12


def test_interpolation_injects_coarse_nodes():
    n_c, n_f = 4, 16
    v = random_vectors(1, 1, (n_c - 1) ** 2)[0]
    pv = twogrid.interpolate(v, n_c, n_f).reshape(n_f - 1, n_f - 1)
    r = n_f // n_c
    assert np.allclose(pv[r - 1::r, r - 1::r], v.reshape(n_c - 1, n_c - 1), atol=1e-15)


def test_degenerate_two_grid_returns_coarse_eigenvalue():
    y = random_points(2, 1, 8)[0]
    lam_fine = twogrid.fine_eigenvalue(16, y)
    assert twogrid.twogrid(16, 8, 16, 8, y) == pytest.approx(lam_fine, rel=1e-13)


def test_two_grid_matches_dense_solve():
    n_c, n_f, S, s = 4, 16, 3, 8
    y = random_points(4, 1, s)[0]
    lam_H, u_H = twogrid.coarse_pair(n_c, y[:S])
    lam = twogrid.twogrid_update(n_f, y[:s], lam_H, u_H, n_c)
    A, M = fem.assemble(n_f, fem.coefficient(n_f, y[:s]))
    Ad, Md = A.toarray(), M.toarray()
    P = twogrid.interpolation_matrix(n_c, n_f).toarray()
    w = np.linalg.solve(Ad - lam_H * Md, Md @ (P @ u_H))
    assert lam == pytest.approx((w @ Ad @ w) / (w @ Md @ w), rel=1e-12)


def test_two_grid_bounded_below_by_fine_eigenvalue():
    # a Rayleigh quotient is never below the smallest eigenvalue (min-max)
    for seed in range(3):
        y = random_points(20 + seed, 1, 16)[0]
        lam_h = twogrid.fine_eigenvalue(32, y)
        lam_tg = twogrid.twogrid(32, 16, 8, 4, y)
        assert lam_tg >= lam_h - 1e-12 * lam_h


def test_rq_difference_identity():
    # Lemma 3.1 with B = A_s (eigenpair (lambda, u)) and B~ = A_s' (s' < s), any w
    n = 16
    y = random_points(31, 1, 16)[0]
    A_s, M = fem.assemble(n, fem.coefficient(n, y))
    A_t, _ = fem.assemble(n, fem.coefficient(n, y[:5]))
    lam, u = twogrid.smallest_eigpair(A_s, M)
    for w in random_vectors(32, 3, (n - 1) ** 2):
        w = u + 0.3 * w / np.linalg.norm(w)
        lhs = (w @ (A_t @ w)) / (w @ (M @ w)) - lam
        e = u - w
        rhs = ((e @ (A_t @ e)) - lam * (e @ (M @ e))
               + (u @ (A_s @ (u - 2 * w))) - (u @ (A_t @ (u - 2 * w)))) / (w @ (M @ w))
        assert abs(lhs - rhs) < 1e-11 * lam


def test_two_grid_rate_in_coarse_mesh():
    # Theorem 3.1 with S = s and h fixed: lambda^h - lambda_h behaves like H^8; the build
    # requires at least H^4 (a factor 16 per halving of H)
    n_f = 64
    y = np.array([0.4, -0.3])
    lam_h = twogrid.fine_eigenvalue(n_f, y)
    gaps = [twogrid.twogrid(n_f, 2, n_c, 2, y) - lam_h for n_c in (4, 8, 16)]
    assert all(g > 0 for g in gaps)
    ratios = [gaps[i] / gaps[i + 1] for i in range(2)]
    assert min(ratios) > 16.0
    assert ratios[0] > 100.0  # close to 2^8 before rounding enters


def test_coarse_eigenvalue_error_is_order_H2():
    n_f = 64
    y = np.array([0.4, -0.3])
    lam_h = twogrid.fine_eigenvalue(n_f, y)
    d = [twogrid.coarse_pair(n_c, y)[0] - lam_h for n_c in (8, 16, 32)]
    assert all(x > 0 for x in d)
    # lambda_H - lambda_h = C (H^2 - h^2) to leading order: ratios 63/15 and 15/3
    assert d[0] / d[1] == pytest.approx(63 / 15, rel=0.03)
    assert d[1] / d[2] == pytest.approx(15 / 3, rel=0.03)
