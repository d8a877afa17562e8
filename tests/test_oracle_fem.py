"""Pins for the oracle's P1 finite elements (Sec. 2.3) against closed forms and invariants."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, twogrid
from synthetic_inputs import random_cell_coefficients, random_points


def laplacian_5pt(n):
    m = n - 1
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_constant_stiffness_is_five_point_laplacian(n):
    # textbook: P1 on a right-isosceles mesh with a = 1 is the 4/-1 five-point stencil
    A, _ = fem.assemble(n)
    assert abs(A - laplacian_5pt(n)).max() < 1e-13


@pytest.mark.parametrize("n,p,q", [(8, 1, 1), (8, 3, 2), (16, 5, 7), (16, 15, 1)])
def test_stiffness_on_sine_modes(n, p, q):
    # discrete sine modes are exact eigenvectors of the constant stencil
    A, _ = fem.assemble(n)
    i = np.arange(1, n)
    v = np.outer(np.sin(q * np.pi * i / n), np.sin(p * np.pi * i / n)).ravel()  # row j, column i
    mu = 4 - 2 * np.cos(p * np.pi / n) - 2 * np.cos(q * np.pi / n)
    assert np.allclose(A @ v, mu * v, atol=1e-12)


def _edge_form(n, a_t):
    """Weighted five-point form derived by hand from the cotangent formula: on a right-isosceles
    triangle only the two legs carry a weight a_T/2; the hypotenuse carries none."""
    low = a_t[: n * n].reshape(n, n)  # [j, i]
    up = a_t[n * n:].reshape(n, n)
    m = n - 1
    A = np.zeros((m * m, m * m))

    def k(i, j):
        return (j - 1) * m + (i - 1) if (1 <= i <= m and 1 <= j <= m) else -1

    def add(p, q, w):
        if p >= 0:
            A[p, p] += w
        if q >= 0:
            A[q, q] += w
        if p >= 0 and q >= 0:
            A[p, q] -= w
            A[q, p] -= w

    for j in range(0, n + 1):
        for i in range(0, n):
            # horizontal edge (i,j)-(i+1,j): lower triangle of cell (i,j), upper of cell (i,j-1)
            w = 0.0
            if j < n:
                w += 0.5 * low[j, i]
            if j > 0:
                w += 0.5 * up[j - 1, i]
            add(k(i, j), k(i + 1, j), w)
    for j in range(0, n):
        for i in range(0, n + 1):
            # vertical edge (i,j)-(i,j+1): upper triangle of cell (i,j), lower of cell (i-1,j)
            w = 0.0
            if i < n:
                w += 0.5 * up[j, i]
            if i > 0:
                w += 0.5 * low[j, i - 1]
            add(k(i, j), k(i, j + 1), w)
    return A


@pytest.mark.parametrize("n", [4, 8])
def test_variable_stiffness_matches_cotangent_edge_form(n):
    a = random_cell_coefficients(11, 1, n)[0].ravel()
    A, _ = fem.assemble(n, a)
    assert np.abs(A.toarray() - _edge_form(n, a)).max() < 1e-12


@pytest.mark.parametrize("n", [4, 8, 16])
def test_mass_seven_point_form(n):
    # consistent P1 mass: h^2/2 on the diagonal, h^2/12 along the six mesh edges (E W N S NE SW)
    _, M = fem.assemble(n)
    h2 = 1.0 / n ** 2
    m = n - 1
    ref = np.zeros((m * m, m * m))
    for j in range(1, n):
        for i in range(1, n):
            p = (j - 1) * m + (i - 1)
            ref[p, p] = h2 / 2
            for di, dj in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)]:
                ii, jj = i + di, j + dj
                if 1 <= ii <= m and 1 <= jj <= m:
                    ref[p, (jj - 1) * m + (ii - 1)] = h2 / 12
    assert np.abs(M.toarray() - ref).max() < 1e-15


@pytest.mark.parametrize("n", [2, 4, 8])
def test_mass_and_energy_exact_on_linear_functions(n):
    # with all nodes kept, P1 integrates u^2 exactly and a|grad u|^2 element by element
    alpha, beta, gamma = 0.7, -1.3, 2.1
    a = random_cell_coefficients(5, 1, n)[0].ravel()
    A, M = fem.assemble(n, a, with_boundary=True)
    coords, _, _ = fem.mesh(n)
    u = alpha + beta * coords[:, 0] + gamma * coords[:, 1]
    int_u2 = alpha ** 2 + beta ** 2 / 3 + gamma ** 2 / 3 + alpha * beta + alpha * gamma + beta * gamma / 2
    assert abs(u @ (M @ u) - int_u2) < 1e-13
    # every triangle has area h^2 / 2 and the same gradient (beta, gamma)
    assert abs(u @ (A @ u) - (beta ** 2 + gamma ** 2) * a.mean()) < 1e-12


def test_psi_pair_order():
    pairs = fem.psi_pairs(200)
    keys = [(k1 * k1 + k2 * k2, k1) for k1, k2 in pairs]
    assert keys == sorted(keys) and len(set(pairs)) == 200
    top = keys[-1][0]
    # complete: every pair with a smaller squared norm than the last one is present
    for k1 in range(1, 40):
        for k2 in range(1, 40):
            if k1 * k1 + k2 * k2 < top:
                assert (k1, k2) in pairs
    assert pairs[:4] == [(1, 1), (1, 2), (2, 1), (2, 2)]


def test_centroids_inside_their_triangles():
    n = 8
    c = fem.centroids(n).reshape(2, n, n, 2)
    h = 1.0 / n
    for p in range(2):
        for j in range(n):
            for i in range(n):
                x, y = c[p, j, i] / h - np.array([i, j])
                assert 0 < x < 1 and 0 < y < 1
                assert (x > y) if p == 0 else (x < y)
    assert np.allclose(c.reshape(-1, 2).mean(axis=0), 0.5)


def test_coefficient_zero_parameter_and_bounds():
    n = 16
    assert np.allclose(fem.coefficient(n, np.zeros(16), a0=1.3), 1.3)
    # |a - a0| <= 1/2 sum_j j^-2 < pi^2/12 for y in [-1/2, 1/2)^s
    y = random_points(3, 4, 64)
    for yy in y:
        a = fem.coefficient(n, yy)
        assert np.all(np.abs(a - 1.0) <= 0.5 * sum(j ** -2.0 for j in range(1, 65)) + 1e-15)
    # extreme parameter y = -1/2 sign(psi_j): a_min > 1 - pi^2/12 > 0
    assert fem.coefficient(n, -0.5 * np.ones(64)).min() > 1 - np.pi ** 2 / 12


def test_coefficient_integral_converges():
    # centroid rule: sum_T area_T psi_j(c_T) -> closed-form integral of psi_j over the square
    n = 64
    Psi = fem.psi_matrix(n, 6)
    area = 0.5 / n ** 2
    for j, (k1, k2) in enumerate(fem.psi_pairs(6), start=1):
        exact = j ** -2.0 * (1 - np.cos(np.pi * k1)) / (np.pi * k1) * (1 - np.cos(np.pi * k2)) / (np.pi * k2)
        assert abs(area * Psi[:, j - 1].sum() - exact) < 2e-3 * j ** -2.0 + 1e-15


def test_constant_coefficient_eigenvalue_converges_to_2pi2():
    lam = [twogrid.fine_eigenvalue(n, np.zeros(0)) for n in (8, 16, 32, 64)]
    err = np.array(lam) - 2 * np.pi ** 2
    assert np.all(err > 0) and np.all(np.diff(err) < 0)  # conforming FE converge from above
    ratios = err[:-1] / err[1:]
    assert abs(ratios[-1] - 4.0) < 0.05  # O(h^2), eq. fe_lam_u


def test_dense_and_sparse_eigensolvers_agree():
    n = 32
    y = random_points(7, 1, 16)[0]
    a = fem.coefficient(n, y)
    A, M = fem.assemble(n, a)
    lam_d, u_d = twogrid.smallest_eigpair(A, M)
    import scipy.sparse.linalg as spla
    w, V = spla.eigsh(A.tocsc(), k=1, M=M.tocsc(), sigma=0.0, which="LM", tol=1e-14)
    assert abs(lam_d - w[0]) < 1e-11 * lam_d
    v = V[:, 0] / np.sqrt(V[:, 0] @ (M @ V[:, 0]))
    assert min(np.abs(u_d - v).max(), np.abs(u_d + v).max()) < 1e-8


def test_homogeneity_and_monotonicity():
    n = 16
    y = random_points(9, 1, 16)[0]
    a = fem.coefficient(n, y)
    A, M = fem.assemble(n, a)
    lam = twogrid.smallest_eigpair(A, M)[0]
    lam3 = twogrid.smallest_eigpair(fem.assemble(n, 3.0 * a)[0], M)[0]
    assert abs(lam3 - 3 * lam) < 1e-12 * lam3
    bump = a.copy()
    bump[::7] += 0.1
    lam_b = twogrid.smallest_eigpair(fem.assemble(n, bump)[0], M)[0]
    assert lam_b > lam
    assert twogrid.smallest_eigpair(fem.assemble(n, a - 0.05)[0], M)[0] < lam


def test_smallest_eigenvector_positive():
    n = 16
    y = random_points(13, 1, 16)[0]
    lam, u = twogrid.coarse_pair(n, y)
    assert np.all(u > 0)
    _, M = fem.assemble(n)
    assert abs(u @ (M @ u) - 1) < 1e-13


def test_coefficient_large_mesh_path_matches_matrix_path():
    # the term-by-term evaluation used on large meshes equals the Psi-matrix product
    n, s = 256, 300
    y = random_points(17, 1, s)[0]
    a_terms = fem.coefficient(n, y)  # 2 n^2 s > 2^25: term by term
    a_matrix = 1.0 + fem._psi_matrix(n, s, 2.0) @ y
    assert np.abs(a_terms - a_matrix).max() < 1e-13


# ---- the paper's first test problem (Sec. 5): psi_j = j^-p sin(j pi x1) sin((j+1) pi x2)
def test_family1_pairs():
    assert fem.psi_pairs(5, family=1) == [(1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    with pytest.raises(ValueError):
        fem.psi_pairs(3, family=7)


@pytest.mark.parametrize("j", [1, 2, 5])
def test_family1_term_has_wave_numbers_j_and_j_plus_1(j):
    # centroid rule of psi_j * sin(j pi x1) sin((j+1) pi x2): with equal wave numbers in each
    # direction the moment is j^-p / 4 (the rule is exact for these products: the centroids sit
    # symmetrically in every cell); with the wave numbers swapped the integrand's integral is zero
    # and the rule's value vanishes as the mesh is refined
    p = 4.0 / 3.0
    sw = []
    for n in (32, 64):
        c = fem.centroids(n)
        area = 0.5 / n ** 2
        Psi = fem.psi_matrix(n, j, p, family=1)[:, j - 1]
        probe = np.sin(j * np.pi * c[:, 0]) * np.sin((j + 1) * np.pi * c[:, 1])
        swapped = np.sin((j + 1) * np.pi * c[:, 0]) * np.sin(j * np.pi * c[:, 1])
        assert abs(area * Psi @ probe - j ** (-p) / 4) < 1e-14
        sw.append(abs(area * Psi @ swapped))
    assert sw[1] < 1e-8 * j ** (-p) and sw[1] < sw[0] / 4


def test_family1_coefficient_bound_and_positivity():
    p, a0, n, s = 4.0 / 3.0, np.pi / np.sqrt(2.0), 16, 64
    bound = 0.5 * sum(j ** (-p) for j in range(1, s + 1))
    for yy in random_points(21, 4, s):
        a = fem.coefficient(n, yy, a0, p, family=1)
        assert np.all(np.abs(a - a0) <= bound + 1e-14)
        assert a.min() > 0
    # the extreme parameter y = -1/2 sign(psi_j) stays positive for a0 = pi / sqrt(2)
    assert a0 - bound > 0.7


def test_family1_two_grid_between_fine_and_coarse_eigenvalues():
    p, a0 = 4.0 / 3.0, np.pi / np.sqrt(2.0)
    y = random_points(23, 1, 64)[0]
    lam_h = twogrid.fine_eigenvalue(32, y, a0, p, family=1)
    lam_H = twogrid.coarse_pair(8, y[:8], a0, p, family=1)[0]
    lam_tg = twogrid.twogrid(32, 64, 8, 8, y, a0, p, family=1)
    # the two-grid value is a Rayleigh quotient (>= lambda_h) and far closer to lambda_h than the
    # coarse eigenvalue is
    assert lam_tg >= lam_h - 1e-12 * lam_h
    assert abs(lam_tg - lam_h) < 0.1 * abs(lam_H - lam_h)


def test_large_coefficient_path_is_correctly_summed():
    # above 2^25 table entries the coefficient adds its terms one by one with compensated
    # summation: on sampled triangles it equals math.fsum (the correctly rounded sum) of the terms
    import math

    n, s = 256, 1024
    y = random_points(77, 1, s)[0]
    a = fem.coefficient(n, y)
    c = fem.centroids(n)
    pairs = fem.psi_pairs(s)
    for t in (0, 777, 65535, 2 * n * n - 1):
        terms = [1.0] + [y[j] * (j + 1) ** -2.0 * np.sin(np.pi * k1 * c[t, 0]) * np.sin(np.pi * k2 * c[t, 1])
                         for j, (k1, k2) in enumerate(pairs)]
        assert abs(a[t] - math.fsum(terms)) <= np.finfo(float).eps * abs(a[t])
