"""Pins of the oracle's second test problem (Sec. 5, domain with four islands) and of the
eigenfunction functional (Sec. 1 and Sec. 4.3: the estimator of E[G(u)] for a linear functional G).

Each check compares with something fixed independently of the code under test: the island
geometry (area 1/4, boundaries on the mesh lines of width 1/8), closed-form L2 norms and
orthogonality of the term families on their regions, an element-by-element quadrature of the
reaction matrix, the exact shift of the spectrum by a constant reaction, Rayleigh-quotient bounds,
and the integral 8 / pi^2 of the normalised Dirichlet ground state of the Laplacian.
"""
import numpy as np
import pytest

from oracle import fem, mlqmc, twogrid
from synthetic_inputs import Level, random_points


def _areas(n):
    return np.full(2 * n * n, 0.5 / (n * n))


def test_islands_area_and_alignment():
    # D_f is four squares of side 1/4: area 1/4.  On meshes of width 1/8 and finer every triangle
    # lies entirely inside or entirely outside (all three vertices agree with the centroid, up to
    # vertices on the island boundary, which belong to both closures).
    for n in (8, 16, 64):
        inside = fem.in_islands(fem.centroids(n))
        assert _areas(n)[inside].sum() == pytest.approx(0.25, abs=1e-14)
        coords, tris, _ = fem.mesh(n)
        v = coords[tris]  # [nt, 3, 2]
        strictly_in = lambda x: (((x > 0.125) & (x < 0.375)) | ((x > 0.625) & (x < 0.875)))  # noqa: E731
        # no triangle has a vertex strictly inside an island while its centroid is outside, or a
        # vertex strictly outside (not on a closure) while its centroid is inside
        vin = strictly_in(v[..., 0]) & strictly_in(v[..., 1])
        vclosed = fem.in_islands(v)
        assert not np.any(vin.any(axis=1) & ~inside)
        assert not np.any((~vclosed).any(axis=1) & inside)


def test_zeroth_terms_and_their_scaling():
    # y = 0: a = 0.01 on D_f and 0.011 off it, b = 2 and 0.3; integrals over D in closed form
    n = 32
    s2 = np.pi / np.sqrt(2.0)
    for decays, fa_in, fa_out, fb_in, fb_out in [
        ((2.0, 2.0, 2.0, 2.0), 1, 1, 1, 1),
        ((4 / 3, 2.0, 4 / 3, 2.0), s2, 1, s2, 1),  # the left case of the paper's Problem 2 figure
        ((2.0, 4 / 3, 3.0, 1.5), 1, s2, 1, s2),
    ]:
        a, b = fem.problem2_coefficients(n, np.zeros(6), decays)
        w = _areas(n)
        assert (w * a).sum() == pytest.approx(0.25 * 0.01 * fa_in + 0.75 * 0.011 * fa_out, rel=1e-13)
        assert (w * b).sum() == pytest.approx(0.25 * 2.0 * fb_in + 0.75 * 0.3 * fb_out, rel=1e-13)
        assert set(np.round(a, 12)) == {round(0.01 * fa_in, 12), round(0.011 * fa_out, 12)}


def test_term_families_norms_and_orthogonality():
    # The discrete L2 Gram matrix of the terms (centroid rule) tends to the continuous one with
    # O(h^2): odd j (k = (j+1)/2) live on D_f with norm^2 sigma^2 k^{-2p} / 16, even j (k = j/2) live
    # off D_f with norm^2 sigma'^2 k^{-2p'} * 3/16; distinct terms are orthogonal (the frequencies
    # 8k pi, 8(k+1) pi are multiples of the island width's reciprocal 4, so the sines complete whole
    # half-periods on every island).
    s = 8
    decays = (4 / 3, 2.0, 1.5, 3.0)
    pa, pa2, pb, pb2 = decays
    expect_a = np.zeros(s)
    expect_b = np.zeros(s)
    for j in range(1, s + 1):
        if j % 2:
            k = (j + 1) // 2
            expect_a[j - 1] = 0.01 ** 2 * k ** (-2 * pa) / 16
            expect_b[j - 1] = 2.0 ** 2 * k ** (-2 * pb) / 16
        else:
            k = j // 2
            expect_a[j - 1] = 0.011 ** 2 * k ** (-2 * pa2) * 3 / 16
            expect_b[j - 1] = 0.3 ** 2 * k ** (-2 * pb2) * 3 / 16
    errs = []
    for n in (64, 128):
        _, Pa, _, Pb = fem.problem2_terms(n, s, decays)
        w = _areas(n)[:, None]
        Ga = Pa.T @ (w * Pa)
        Gb = Pb.T @ (w * Pb)
        errs.append(max(np.max(np.abs(np.diag(Ga) / expect_a - 1)), np.max(np.abs(np.diag(Gb) / expect_b - 1))))
        off = Ga - np.diag(np.diag(Ga))
        assert np.max(np.abs(off)) <= 2e-2 * np.max(expect_a)
        offb = Gb - np.diag(np.diag(Gb))
        assert np.max(np.abs(offb)) <= 2e-2 * np.max(expect_b)
    assert errs[1] < 0.05 and errs[0] / errs[1] > 3.0  # second order in h


def test_reaction_matrix_by_quadrature():
    # B_ij = integral of b phi_i phi_j, b constant per triangle, by the three-edge-midpoint rule
    # (exact for quadratics) element by element, on all nodes
    n = 4
    rng = np.random.default_rng(3)
    b_t = 0.1 + rng.random(2 * n * n)
    _, _, B = fem.assemble(n, np.ones(2 * n * n), with_boundary=True, b_t=b_t)
    coords, tris, _ = fem.mesh(n)
    N = coords.shape[0]
    ref = np.zeros((N, N))
    mids = [(0, 1), (1, 2), (0, 2)]
    for t, tri in enumerate(tris):
        area = 0.5 / (n * n)
        for (m0, m1) in mids:
            phi = np.zeros(3)
            phi[m0] = phi[m1] = 0.5
            for a in range(3):
                for c in range(3):
                    ref[tri[a], tri[c]] += b_t[t] * area / 3 * phi[a] * phi[c]
    assert np.allclose(B.toarray(), ref, rtol=0, atol=1e-15)
    # and 1^T B 1 = integral of b
    assert B.sum() == pytest.approx((_areas(n) * b_t).sum(), rel=1e-14)


def test_constant_reaction_shifts_the_spectrum():
    n = 16
    rng = np.random.default_rng(4)
    a_t = 0.5 + rng.random(2 * n * n)
    A, M, B = fem.assemble(n, a_t, b_t=np.full(2 * n * n, 0.7))
    assert abs(B - 0.7 * M).max() <= 1e-16
    lam0, _ = twogrid.smallest_eigpair(A, M)
    lam1, _ = twogrid.smallest_eigpair((A + B).tocsr(), M)
    assert lam1 == pytest.approx(lam0 + 0.7, rel=1e-12)


def test_problem2_eigenvalue_within_reaction_bounds():
    # B - b_min M and b_max M - B are sums of nonnegative multiples of element masses, so
    # lambda(A) + b_min <= lambda(A + B) <= lambda(A) + b_max
    n = 16
    y = random_points(8, 1, 12)[0]
    for decays in (2.0, (4 / 3, 2.0, 4 / 3, 2.0)):
        a, b = fem.problem2_coefficients(n, y, decays)
        assert a.min() > 0 and b.min() > 0
        A, M, B = fem.assemble(n, a, b_t=b)
        lamA, _ = twogrid.smallest_eigpair(A, M)
        lam = twogrid.fine_eigenvalue(n, y, decay=decays, family=2)
        assert lamA + b.min() - 1e-12 <= lam <= lamA + b.max() + 1e-12
        lam2, _ = twogrid.smallest_eigpair((A + B).tocsr(), M)
        assert lam == pytest.approx(lam2, rel=1e-13)


def test_integral_of_p1_functions():
    # the integral of a P1 hat function of an interior node is h^2 (six triangles of area h^2/2,
    # a third each); of the interpolant of x(1-x)y(1-y) it converges to 1/36 with O(h^2)
    n = 8
    for k in (0, 10, 48):
        u = np.zeros((n - 1) ** 2)
        u[k] = 1.0
        assert fem.integral(n, u) == pytest.approx(1.0 / n ** 2, rel=1e-14)
    errs = []
    for n in (16, 32):
        x = np.arange(1, n) / n
        X, Y = np.meshgrid(x, x, indexing="xy")
        u = (X * (1 - X) * Y * (1 - Y)).ravel()
        errs.append(abs(fem.integral(n, u) - 1.0 / 36))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


def test_functional_of_the_laplacian_ground_state():
    # a = 1: u = 2 sin(pi x1) sin(pi x2) has ||u||_L2 = 1 and integral 8 / pi^2; the FE value
    # converges with O(h^2), independently of the scaling and sign of the discrete vector
    errs = []
    for n in (16, 32, 64):
        lam, u = twogrid.smallest_eigpair(fem.stiffness(n, np.ones(2 * n * n)), fem.mass(n))
        g = twogrid.functional(n, u)
        assert twogrid.functional(n, -3.5 * u) == pytest.approx(g, rel=1e-14)
        errs.append(abs(g - 8 / np.pi ** 2))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_twogrid_functional_converges_in_the_coarse_mesh():
    # G of the two-grid eigenfunction approximation tends to G of the fine eigenfunction as H -> h
    # (Algorithm 1: the approximation error is a power of H); for both test problems
    n = 32
    for fam, decay, a0, s in ((1, 2.0, 1.0, 8), (2, (4 / 3, 2.0, 4 / 3, 2.0), 1.0, 8)):
        y = random_points(9, 1, s)[0]
        _, u = twogrid.smallest_eigpair(fem.operator(n, y, a0, decay, fam), fem.mass(n))
        g_fine = twogrid.functional(n, u)
        errs = []
        for H in (8, 16):
            lvl = Level(n, H, s, s, 1, 1)
            g = mlqmc.sample_level(lvl, None, y, a0, decay, fam, qoi="functional")[1]
            errs.append(abs(g - g_fine))
        assert errs[1] < errs[0] / 3.0, (fam, errs)


def test_functional_level_values():
    # direct level: G(u_H) of the coarse eigenvector; level differences as for eigenvalues
    y = random_points(10, 1, 8)[0]
    lv0 = Level(8, 8, 8, 8, 1, 1)
    lv1 = Level(16, 8, 8, 8, 1, 1)
    dec = (4 / 3, 2.0, 4 / 3, 2.0)
    q0 = mlqmc.sample_level(lv0, None, y, 1.0, dec, 2, qoi="functional")
    lam_H, u_H = twogrid.coarse_pair(8, y, 1.0, dec, 2)
    assert q0[0] == lam_H and q0[1] == pytest.approx(twogrid.functional(8, u_H), rel=1e-14) and q0[3] == q0[1]
    q1 = mlqmc.sample_level(lv1, lv0, y, 1.0, dec, 2, qoi="functional")
    assert q1[2] == q0[1] and q1[3] == q1[1] - q1[2]
    # the eigenvalue of the same sample is the default quantity
    e1 = mlqmc.sample_level(lv1, lv0, y, 1.0, dec, 2)
    assert e1[0] == lam_H and e1[1] > lam_H * 0.5
