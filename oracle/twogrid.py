"""Exact eigenpairs, nested-mesh interpolation and the two-grid-truncation step.

Test infrastructure only (see ``oracle/__init__.py``).

Algorithm 1 (two-grid-truncation method), for a parameter y, coarse mesh H with
truncation S and fine mesh h with truncation s:

1. (lambda_H, u_H): smallest eigenpair of A_H(y_S) u = lambda M_H u, ||u||_M = 1.
2. Solve A_h(y_s) w - lambda_H M_h w = M_h P u_H (eq. 2grid_source), with P the P1
   nodal interpolation from V_H into V_h ("linear interpolation is sufficient").
3. Normalise w in the M-norm.
4. lambda^h = A_h(y_s)(w, w) (eq. RQ_update).

The inner problems are solved exactly: dense LAPACK ``eigh`` on small coarse
meshes, sparse shift-invert ``eigsh`` on larger ones, and sparse direct LU for
the shifted system.  When H = h and S = s the shifted matrix is singular
(lambda_H is an exact eigenvalue of it); the step then returns lambda_H, the
value its limit takes.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import fem

DENSE_MAX = 961  # dense generalised eigh up to 31 x 31 interior nodes


def smallest_eigpair(A, M):
    """Smallest eigenpair of A u = lambda M u, normalised so that u^T M u = 1 and sum(u) > 0."""
    n = A.shape[0]
    if n <= DENSE_MAX:
        w, V = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, 0])
        u = V[:, 0].copy()
    else:
        w, V = spla.eigsh(A.tocsc(), k=1, M=M.tocsc(), sigma=0.0, which="LM", tol=1e-14)
        u = V[:, 0].copy()
    u /= np.sqrt(u @ (M @ u))
    if u.sum() < 0:
        u = -u
    # the Rayleigh quotient of the computed vector: second-order accurate in the vector
    # error, so it is not limited by the eps * lambda_max error of the dense reduction
    lam = float(u @ (A @ u)) / float(u @ (M @ u))
    return lam, u


_P_CACHE: dict = {}


def interpolation_matrix(n_coarse: int, n_fine: int):
    """P1 nodal interpolation V_H -> V_h as a sparse matrix [fine interior x coarse interior].

    For every fine node x the coarse triangle that contains it is located, the
    barycentric coordinates of x in it are found by solving the 2 x 2 affine
    system of that triangle, and the weights of its three vertices are recorded
    (vertices on the boundary carry the value zero and are dropped).
    """
    key = (n_coarse, n_fine)
    if key in _P_CACHE:
        return _P_CACHE[key]
    import scipy.sparse as sp
    assert n_fine % n_coarse == 0
    coords_c, tris_c, interior_c = fem.mesh(n_coarse)
    H = 1.0 / n_coarse
    jj, ii = np.meshgrid(np.arange(1, n_fine), np.arange(1, n_fine), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    x = np.stack([ii / n_fine, jj / n_fine], axis=1)
    ci = np.minimum(np.floor(x[:, 0] / H).astype(np.int64), n_coarse - 1)
    cj = np.minimum(np.floor(x[:, 1] / H).astype(np.int64), n_coarse - 1)
    lower = (x[:, 0] - ci * H) >= (x[:, 1] - cj * H)
    t = np.where(lower, 0, 1) * n_coarse * n_coarse + cj * n_coarse + ci
    verts = tris_c[t]  # [nf, 3]
    p = coords_c[verts]  # [nf, 3, 2]
    Bm = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]], axis=2)  # columns: edge vectors
    l12 = np.linalg.solve(Bm, (x - p[:, 0])[:, :, None])[:, :, 0]
    bary = np.stack([1.0 - l12.sum(axis=1), l12[:, 0], l12[:, 1]], axis=1)
    rows = np.repeat(np.arange(x.shape[0]), 3)
    cols = interior_c[verts.ravel()]
    vals = bary.ravel()
    keep = cols >= 0
    P = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])),
                      shape=(x.shape[0], (n_coarse - 1) ** 2)).tocsr()
    _P_CACHE[key] = P
    return P


def interpolate(u_coarse: np.ndarray, n_coarse: int, n_fine: int) -> np.ndarray:
    """The fine-mesh nodal values of the coarse P1 function u_coarse."""
    return interpolation_matrix(n_coarse, n_fine) @ u_coarse


def coarse_pair(n_coarse: int, y_coarse: np.ndarray, a0: float = 1.0, decay=2.0, family: int = 0):
    """Step 1 of Algorithm 1: the smallest eigenpair on the coarse mesh with S terms."""
    return smallest_eigpair(fem.operator(n_coarse, y_coarse, a0, decay, family), fem.mass(n_coarse))


def twogrid_update(n_fine: int, y_fine: np.ndarray, lam_H: float, u_H: np.ndarray, n_coarse: int,
                   a0: float = 1.0, decay=2.0, return_vector: bool = False, family: int = 0):
    """Steps 2-4 of Algorithm 1 for a given coarse pair: one shifted solve and a Rayleigh quotient."""
    A = fem.operator(n_fine, y_fine, a0, decay, family)
    M = fem.mass(n_fine)
    if n_fine == n_coarse:
        Pu = u_H.copy()
    else:
        Pu = interpolation_matrix(n_coarse, n_fine) @ u_H
    b = M @ Pu
    K = (A - lam_H * M).tocsc()
    w = spla.splu(K).solve(b)
    # sanity check of the direct solve: its backward error grows with the conditioning of the
    # nearly singular shifted matrix (about 1e-8 relative on the 1/512 mesh)
    res = np.linalg.norm(b - K @ w) / np.linalg.norm(b)
    if not np.isfinite(res) or res > 1e-6:
        raise RuntimeError(f"shifted solve failed: relative residual {res:.3e}")
    w = w / np.sqrt(w @ (M @ w))  # step 3
    lam = float(w @ (A @ w))  # step 4
    return (lam, w) if return_vector else lam


def twogrid(n_fine: int, s: int, n_coarse: int, S: int, y: np.ndarray, a0: float = 1.0,
            decay=2.0, family: int = 0) -> float:
    """Algorithm 1 for one parameter vector y (len(y) >= s >= S).  Degenerate H = h, S = s:
    the coarse eigenvalue itself."""
    lam_H, u_H = coarse_pair(n_coarse, y[:S], a0, decay, family)
    if n_fine == n_coarse and s == S:
        return lam_H
    return twogrid_update(n_fine, y[:s], lam_H, u_H, n_coarse, a0, decay, family=family)


def fine_eigenvalue(n: int, y: np.ndarray, a0: float = 1.0, decay=2.0, family: int = 0) -> float:
    """lambda_{h,s}(y): the smallest FE eigenvalue on mesh 1/n with s = len(y) terms."""
    return smallest_eigpair(fem.operator(n, y, a0, decay, family), fem.mass(n))[0]


def functional(n: int, u: np.ndarray) -> float:
    """G(u) for the linear functional G(v) = integral of v over D, with u scaled to ||u||_{L2} = 1
    and the sign that makes the integral positive (Sec. 1: the eigenfunction is made unique by its
    normalisation and a consistent sign, and each approximation u_l likewise):
    |integral of u| / sqrt(u^T M u)."""
    return abs(fem.integral(n, u)) / float(np.sqrt(u @ (fem.mass(n) @ u)))
