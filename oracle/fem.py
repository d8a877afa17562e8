"""P1 finite elements on the uniform triangulation of D = (0,1)^2 (Sec. 2.3).

Test infrastructure only (see ``oracle/__init__.py``).

Mesh reading (the paper only says "uniform triangular meshes"): the unit
square is cut into n x n squares of side h = 1/n and each square is split by
its south-west to north-east diagonal.  Cell (i, j) = [ih,(i+1)h] x [jh,(j+1)h]
holds the lower triangle {(i,j), (i+1,j), (i+1,j+1)} and the upper triangle
{(i,j), (i+1,j+1), (i,j+1)}.  Homogeneous Dirichlet conditions: only the
(n-1)^2 interior nodes are unknowns, numbered row by row,
k = (j-1)(n-1) + (i-1).

The coefficient is constant on each triangle, equal to a at the centroid
(one-point rule); the mass matrix is the exact consistent P1 mass (c = 1).
Matrices are assembled by an explicit loop over elements from the vertex
coordinates: nothing here assumes the stencil that results.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


_MESH_CACHE: dict = {}


def mesh(n: int):
    """Return (coords [(n+1)^2, 2], triangles [2n^2, 3] vertex ids, interior map).

    Node id = j*(n+1) + i.  Triangle t = p*n*n + j*n + i with p = 0 for the lower and
    p = 1 for the upper triangle of cell (i, j).  ``interior[id]`` is the unknown
    number of a node, or -1 on the boundary.  (Cached per mesh.)
    """
    if n in _MESH_CACHE:
        return _MESH_CACHE[n]
    h = 1.0 / n
    idx = np.arange(n + 1)
    I, J = np.meshgrid(idx, idx, indexing="xy")  # I[j, i] = i
    coords = np.stack([I.ravel() * h, J.ravel() * h], axis=1)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # cell (i, j) at [j, i]

    def nid(i, j):
        return j * (n + 1) + i

    low = np.stack([nid(ii, jj), nid(ii + 1, jj), nid(ii + 1, jj + 1)], axis=-1)
    up = np.stack([nid(ii, jj), nid(ii + 1, jj + 1), nid(ii, jj + 1)], axis=-1)
    tris = np.concatenate([low.reshape(-1, 3), up.reshape(-1, 3)], axis=0).astype(np.int64)

    interior = -np.ones((n + 1) * (n + 1), dtype=np.int64)
    jj, ii = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    interior[nid(ii, jj).ravel()] = ((jj - 1) * (n - 1) + (ii - 1)).ravel()
    _MESH_CACHE[n] = (coords, tris, interior)
    return coords, tris, interior


def centroids(n: int) -> np.ndarray:
    """Centroids of all 2 n^2 triangles, as the mean of the three vertices."""
    coords, tris, _ = mesh(n)
    return coords[tris].mean(axis=1)


# ---------------------------------------------------------------------------------------------
# The second test problem of Sec. 5 (domain with four interior islands): family 2.
#   D_f = four squares [1/8,3/8]^2, [5/8,7/8]^2, [1/8,3/8] x [5/8,7/8], [5/8,7/8] x [1/8,3/8]
#   a0 = 0.01 on D_f, 0.011 elsewhere;  b0 = 2 on D_f, 0.3 elsewhere;
#   term j: odd j -> k = (j+1)/2, supported on D_f:   a_j = 0.01 w_k(p_a),   b_j = 2 w_k(p_b);
#           even j -> k = j/2, supported off D_f:      a_j = 0.011 w_k(p_a'), b_j = 0.3 w_k(p_b');
#   w_k(q; x) = k^-q sin(8 k pi x1) sin(8 (k+1) pi x2) on its region, 0 on the other.
# A zeroth term is scaled by pi / sqrt(2) when a decay below 2 belongs to it.  Reading: each
# decay belongs to the part of the zeroth term on its own region (p_a to a0 on D_f, p_a' to a0 off
# D_f, p_b and p_b' likewise for b0), the part whose positivity its terms put at risk.  A triangle
# belongs to D_f when its centroid does (the meshes of width 1/8 and finer resolve the islands).

SIG_A_IN, SIG_A_OUT, SIG_B_IN, SIG_B_OUT = 0.01, 0.011, 2.0, 0.3


def in_islands(x: np.ndarray) -> np.ndarray:
    """Whether each point x [.., 2] lies in the four closed islands D_f."""
    def band(t):
        return ((t >= 0.125) & (t <= 0.375)) | ((t >= 0.625) & (t <= 0.875))
    return band(x[..., 0]) & band(x[..., 1])


def problem2_decays(decay):
    """(p_a, p_a', p_b, p_b') from one decay or a sequence of four."""
    d = np.atleast_1d(np.asarray(decay, dtype=np.float64))
    if d.size == 1:
        d = np.repeat(d, 4)
    if d.size != 4:
        raise ValueError("the second test problem takes one decay or four")
    return tuple(float(v) for v in d)


def problem2_terms(n: int, s: int, decay=2.0):
    """(a0_t, Psi_a [nT, s], b0_t, Psi_b [nT, s]) at the triangle centroids of mesh 1/n;
    ``decay`` is (p_a, p_a', p_b, p_b') or one value for all four."""
    pa, pa2, pb, pb2 = problem2_decays(decay)
    c = centroids(n)
    inside = in_islands(c)
    sc = lambda p: np.pi / np.sqrt(2.0) if p < 2.0 else 1.0  # noqa: E731
    a0 = np.where(inside, SIG_A_IN * sc(pa), SIG_A_OUT * sc(pa2))
    b0 = np.where(inside, SIG_B_IN * sc(pb), SIG_B_OUT * sc(pb2))
    Pa = np.zeros((c.shape[0], s))
    Pb = np.zeros((c.shape[0], s))
    for j in range(1, s + 1):
        odd = j % 2 == 1
        k = (j + 1) // 2 if odd else j // 2
        shape = np.sin(8 * k * np.pi * c[:, 0]) * np.sin(8 * (k + 1) * np.pi * c[:, 1])
        region = inside if odd else ~inside
        qa, qb = (pa, pb) if odd else (pa2, pb2)
        Pa[:, j - 1] = np.where(region, (SIG_A_IN if odd else SIG_A_OUT) * k ** (-qa) * shape, 0.0)
        Pb[:, j - 1] = np.where(region, (SIG_B_IN if odd else SIG_B_OUT) * k ** (-qb) * shape, 0.0)
    return a0, Pa, b0, Pb


def problem2_coefficients(n: int, y: np.ndarray, decay=2.0):
    """(a_t, b_t) = (a0 + sum_j y_j a_j, b0 + sum_j y_j b_j) at the centroids (s = len(y))."""
    y = np.asarray(y, dtype=np.float64)
    a0, Pa, b0, Pb = problem2_terms(n, y.size, decay)
    return a0 + Pa @ y, b0 + Pb @ y


def psi_pairs(s: int, family: int = 0):
    """Frequency pairs (k1, k2) of the first s terms of a coefficient family.

    family 0 (the synthetic workload family): all pairs with k1, k2 >= 1 ordered by
    k1^2 + k2^2, ties broken by smaller k1.  family 1 (the paper's first test problem, Sec. 5):
    psi_j uses sin(j pi x1) sin((j+1) pi x2), i.e. (k1, k2) = (j, j+1).
    """
    if family == 1:
        return [(j, j + 1) for j in range(1, s + 1)]
    if family != 0:
        raise ValueError(f"unknown coefficient family {family}")
    K = int(np.ceil(2.0 * np.sqrt(max(s, 1)))) + 2
    pairs = [(k1, k2) for k1 in range(1, K + 1) for k2 in range(1, K + 1)]
    pairs.sort(key=lambda p: (p[0] ** 2 + p[1] ** 2, p[0]))
    return pairs[:s]


_PSI_CACHE: dict = {}


def psi_matrix(n: int, s: int, decay: float = 2.0, family: int = 0) -> np.ndarray:
    """Psi[t, j-1] = psi_j(c_t) = j^-decay sin(pi k1_j x1) sin(pi k2_j x2) at triangle centroids
    (cached per mesh, truncation, decay and family; callers must not modify the result)."""
    key = (n, s, decay, family)
    if key not in _PSI_CACHE:
        _PSI_CACHE[key] = _psi_matrix(n, s, decay, family)
    return _PSI_CACHE[key]


def _psi_matrix(n: int, s: int, decay: float, family: int = 0) -> np.ndarray:
    c = centroids(n)
    out = np.zeros((c.shape[0], s))
    for j, (k1, k2) in enumerate(psi_pairs(s, family), start=1):
        out[:, j - 1] = j ** (-decay) * np.sin(np.pi * k1 * c[:, 0]) * np.sin(np.pi * k2 * c[:, 1])
    return out


def coefficient(n: int, y: np.ndarray, a0: float = 1.0, decay: float = 2.0, family: int = 0) -> np.ndarray:
    """a(c_t, y) = a0 + sum_{j<=s} y_j psi_j(c_t) for every triangle t (eq. coeff, eq. coeff_s).

    The truncation dimension is len(y): terms beyond it are zero.  Small meshes use the cached
    Psi matrix; large ones add the terms one by one (same formula, no s x 2n^2 matrix in memory)
    with compensated (Neumaier) summation, so their rounding error stays near one unit of the
    result however many terms there are.
    """
    y = np.asarray(y, dtype=np.float64)
    if y.size == 0:
        return np.full(2 * n * n, float(a0))
    if y.size * 2 * n * n <= (1 << 25):
        return a0 + psi_matrix(n, y.size, decay, family) @ y
    c = centroids(n)
    a = np.full(c.shape[0], float(a0))
    # sin(pi k x) only depends on k and on the 2n distinct centroid abscissae (ordinates)
    xs, xi = np.unique(c[:, 0], return_inverse=True)
    ys, yi = np.unique(c[:, 1], return_inverse=True)
    comp = np.zeros_like(a)
    for j, (k1, k2) in enumerate(psi_pairs(y.size, family), start=1):
        term = y[j - 1] * j ** (-decay) * np.sin(np.pi * k1 * xs)[xi] * np.sin(np.pi * k2 * ys)[yi]
        t = a + term
        # the low-order part lost by the addition, whichever operand is larger
        comp += np.where(np.abs(a) >= np.abs(term), (a - t) + term, (term - t) + a)
        a = t
    return a + comp


_ELEMENT_CACHE: dict = {}


def _element_entries(n: int, with_boundary: bool):
    """Element loop over all triangles: for every local (a, b) pair whose two nodes are
    unknowns, record (row, col, triangle, K_ab for a = 1, M_ab).  The geometric part does
    not depend on the coefficient, so it is cached per mesh.  The per-element matrices are
    computed for all triangles at once: the stiffness for a = 1 is area * G G^T with G the
    physical gradients of the three hat functions (reference gradients times the inverse of the
    triangle's edge matrix), the consistent mass (area / 12) (1 + delta_ab)."""
    key = (n, with_boundary)
    if key in _ELEMENT_CACHE:
        return _ELEMENT_CACHE[key]
    coords, tris, interior = mesh(n)
    p = coords[tris]  # [nt, 3, 2]
    Bm = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]], axis=2)  # columns: edge vectors
    area = 0.5 * np.abs(np.linalg.det(Bm))
    ref_grad = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    G = np.einsum("ak,tkd->tad", ref_grad, np.linalg.inv(Bm))  # physical gradients
    K = area[:, None, None] * np.einsum("tad,tbd->tab", G, G)
    Mloc = (area[:, None, None] / 12.0) * (np.ones((3, 3)) + np.eye(3))[None]
    nt = tris.shape[0]
    ga = np.repeat(tris, 3, axis=1).reshape(nt, 3, 3)  # [t, a, b] -> node of a
    gb = np.tile(tris, (1, 3)).reshape(nt, 3, 3)  # [t, a, b] -> node of b
    ra = ga if with_boundary else interior[ga]
    cb = gb if with_boundary else interior[gb]
    keep = (ra >= 0) & (cb >= 0)
    tt = np.broadcast_to(np.arange(nt)[:, None, None], (nt, 3, 3))
    ent = (ra[keep], cb[keep], tt[keep], K[keep], Mloc[keep])
    _ELEMENT_CACHE[key] = ent
    return ent


def assemble(n: int, a_t: np.ndarray | None = None, with_boundary: bool = False, b_t: np.ndarray | None = None):
    """Stiffness A = sum_T a_T K_T and mass M = sum_T M_T over the elements (Sec. 2.3); with
    ``b_t`` also the reaction matrix B = sum_T b_T M_T of the term b u (the coefficient b
    constant on each triangle, equal to its centroid value), returned third.

    Returns sparse CSR matrices over the interior unknowns, or over all (n+1)^2
    nodes when ``with_boundary`` is set (used by exactness tests).
    """
    nt = 2 * n * n
    if a_t is None:
        a_t = np.ones(nt)
    a_t = np.asarray(a_t, dtype=np.float64).ravel()
    assert a_t.size == nt
    rows, cols, tt, kv, mv = _element_entries(n, with_boundary)
    size = (n + 1) ** 2 if with_boundary else (n - 1) ** 2
    A = sp.coo_matrix((a_t[tt] * kv, (rows, cols)), shape=(size, size)).tocsr()
    M = sp.coo_matrix((mv, (rows, cols)), shape=(size, size)).tocsr()
    A.sum_duplicates()
    M.sum_duplicates()
    if b_t is None:
        return A, M
    b_t = np.asarray(b_t, dtype=np.float64).ravel()
    assert b_t.size == nt
    Bm = sp.coo_matrix((b_t[tt] * mv, (rows, cols)), shape=(size, size)).tocsr()
    Bm.sum_duplicates()
    return A, M, Bm


_MASS_CACHE: dict = {}


def mass(n: int):
    """The y-independent mass matrix (built once per mesh, Sec. 4.2)."""
    if n not in _MASS_CACHE:
        _MASS_CACHE[n] = assemble(n, np.ones(2 * n * n))[1]
    return _MASS_CACHE[n]


def stiffness(n: int, a_t: np.ndarray):
    return assemble(n, a_t)[0]


def operator(n: int, y: np.ndarray, a0: float = 1.0, decay=2.0, family: int = 0):
    """The y-dependent matrix of the eigenproblem on mesh 1/n: the stiffness A(y), plus the
    reaction matrix B(y) for the second test problem (family 2)."""
    if family == 2:
        a_t, b_t = problem2_coefficients(n, y, decay)
        A, _, Bm = assemble(n, a_t, b_t=b_t)
        return (A + Bm).tocsr()
    return stiffness(n, coefficient(n, y, a0, decay, family))


def integral(n: int, u: np.ndarray) -> float:
    """The integral over D of the P1 function with interior nodal values u (zero on the boundary):
    the sum over the triangles of the area times the mean of the three vertex values (exact for a
    linear function on a triangle)."""
    coords, tris, interior = mesh(n)
    full = np.zeros(coords.shape[0])
    full[interior >= 0] = u[interior[interior >= 0]]
    area = 0.5 / (n * n)
    return float(area * full[tris].mean(axis=1).sum())
