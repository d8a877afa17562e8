"""Per-sample level differences and the two-grid MLQMC estimator (Sec. 4.3).

Test infrastructure only (see ``oracle/__init__.py``).

Algorithm 2, for level l with fine mesh h_l, truncation s_l, coarse mesh H_l
and coarse truncation S_l, shift Delta^(r) and lattice point k:

* y = {k z_l / N_l + Delta^(r)} - 1/2 (eq. t_kl, eq. rqmc), k = 0..N_l-1.
* the coarse pair (lambda_H, u_H) on (H_l, S_l) (step 6);
* lambda^l by the two-grid update on (h_l, s_l) (eq. 2grid_src_ell,
  eq. 2grid_update_ell);
* for l > 0, lambda^{l-1} by the two-grid update on (h_{l-1}, s_{l-1}) from the
  SAME coarse pair (steps 10-14); lambda^{-1} = 0;
* Q^(r)_l = (1/N_l) sum_k (lambda^l - lambda^{l-1}) (steps 15-16),
  Qhat_l = mean over r, Qhat^ML = sum_l Qhat_l (eq. tg-mlqmc), and the
  sample-variance error estimate of eq. sample_var per level, added over
  the independent levels (eq. ml-var).

A level whose coarse mesh and truncation equal its fine ones (H_l = h_l,
S_l = s_l) is a direct eigensolve: lambda^l = lambda_{h_l, s_l}.
"""
from __future__ import annotations

import numpy as np

from . import lattice, twogrid


QOIS = ("eigenvalue", "functional")


def _update(n_fine, y, lam_H, u_H, n_coarse, a0, decay, family, qoi):
    """The quantity of interest of the two-grid update on mesh n_fine: lambda^h, or G(u^h) of its
    eigenfunction approximation (Algorithm 1 steps 2-4; G as in ``twogrid.functional``)."""
    if qoi == "eigenvalue":
        return twogrid.twogrid_update(n_fine, y, lam_H, u_H, n_coarse, a0, decay, family=family)
    _, w = twogrid.twogrid_update(n_fine, y, lam_H, u_H, n_coarse, a0, decay, return_vector=True, family=family)
    return twogrid.functional(n_fine, w)


def sample_level(level, prev, y, a0: float = 1.0, decay=2.0, family: int = 0, qoi: str = "eigenvalue"):
    """(lambda_H, Q^l, Q^{l-1}, difference) for one parameter vector y (len >= s_l), where Q is the
    eigenvalue (qoi "eigenvalue") or G(u) of the eigenfunction (qoi "functional"; Sec. 4.3: the same
    estimator for a linear functional of u).

    ``level`` and ``prev`` carry n_fine, n_coarse, s, S (``prev`` is None on level 0).
    """
    assert qoi in QOIS
    lam_H, u_H = twogrid.coarse_pair(level.n_coarse, y[: level.S], a0, decay, family)
    q_H = lam_H if qoi == "eigenvalue" else twogrid.functional(level.n_coarse, u_H)
    if level.n_fine == level.n_coarse and level.s == level.S:
        q_l = q_H
    else:
        q_l = _update(level.n_fine, y[: level.s], lam_H, u_H, level.n_coarse, a0, decay, family, qoi)
    if prev is None:
        return lam_H, q_l, 0.0, q_l
    if prev.n_fine == level.n_coarse and prev.s == level.S:
        q_p = q_H
    else:
        q_p = _update(prev.n_fine, y[: prev.s], lam_H, u_H, level.n_coarse, a0, decay, family, qoi)
    return lam_H, q_l, q_p, q_l - q_p


def level_samples(level, prev, z, delta, ks, a0: float = 1.0, decay=2.0, family: int = 0,
                  qoi: str = "eigenvalue") -> np.ndarray:
    """Per-sample results [R, len(ks), 4] = (lambda_H, Q^l, Q^{l-1}, diff) at lattice indices ks
    for every shift row of ``delta`` [R, s_l] (Q as in ``sample_level``)."""
    delta = np.atleast_2d(delta)
    out = np.zeros((delta.shape[0], len(ks), 4))
    for r in range(delta.shape[0]):
        Y = lattice.points(z, level.N, delta[r], ks)
        for i in range(len(ks)):
            out[r, i] = sample_level(level, prev, Y[i], a0, decay, family, qoi)
    return out


def shift_means(diffs: np.ndarray, N: int) -> np.ndarray:
    """Q^(r)_l = (1/N_l) sum_k diff[r, k] for each shift r (Algorithm 2, steps 15-16)."""
    return np.asarray(diffs).sum(axis=1) / N


def estimate(level_shift_means):
    """Shift-averaged MLQMC estimate and its standard error.

    ``level_shift_means[l]`` holds Q^(r)_l for r = 1..R.  Returns (Qhat^ML, SE, Qhat_l[], Vhat_l[])
    with Vhat_l = sum_r (Qhat_l - Q^(r)_l)^2 / (R (R - 1)) (eq. sample_var) and
    SE = sqrt(sum_l Vhat_l) (eq. ml-var).
    """
    qhat, vhat = [], []
    for q in level_shift_means:
        q = np.asarray(q, dtype=np.float64)
        R = q.size
        if R < 2:
            raise ValueError("the sample-variance estimate needs R >= 2 shifts")
        m = q.sum() / R
        qhat.append(m)
        vhat.append(((m - q) ** 2).sum() / (R * (R - 1)))
    return float(sum(qhat)), float(np.sqrt(sum(vhat))), qhat, vhat


# ---------------------------------------------------------------------------------------------
# Shared shifts, nested points and reuse across levels (Sec. 4.3, the paragraphs after Algorithm
# 2).  Every level uses the same random shifts (drawn once with s_L components; level l uses the
# first s_l of them) and the same embedded lattice rule in radical-inverse order, so point k of
# level l is point k of level 0 in the first s_0 components and point k of level l-1 in the first
# s_{l-1}.  With H_l = h_0 and S_l = s_0 on every level l >= 1, the coarse pair of level l at
# point k is the level-0 (direct) eigenpair at point k, and lambda^{l-1} at point k is the value
# level l-1 computed there: steps 6-8 and 12-14 of Algorithm 2 are skipped and only the fine
# two-grid update (h_l, s_l) remains per level.

def shared_samples(levels, z, m_max: int, delta_row, ks, a0: float = 1.0, decay=2.0,
                   family: int = 0, qoi: str = "eigenvalue") -> np.ndarray:
    """Per-sample results [L+1, len(ks), 4] = (lambda_H, Q^l, Q^{l-1}, diff) of the reuse
    scheme for one shift row (length >= s_L) at embedded-rule indices ks; entries of levels whose
    N_l <= k are NaN.  Level 0 must be direct (n_coarse = n_fine, S = s); levels l >= 1 must have
    n_coarse = n_fine of level 0 and S = s_0."""
    lv0 = levels[0]
    assert lv0.n_fine == lv0.n_coarse and lv0.S == lv0.s
    for lv in levels[1:]:
        assert lv.n_coarse == lv0.n_fine and lv.S == lv0.s
    out = np.full((len(levels), len(ks), 4), np.nan)
    s_max = max(lv.s for lv in levels)
    Y = lattice.embedded_points(z[:s_max], m_max, np.asarray(delta_row)[:s_max], ks)
    for i, k in enumerate(ks):
        y = Y[i]
        lam0, u0 = twogrid.coarse_pair(lv0.n_fine, y[: lv0.s], a0, decay, family)
        q0 = lam0 if qoi == "eigenvalue" else twogrid.functional(lv0.n_fine, u0)
        out[0, i] = (lam0, q0, 0.0, q0)
        prev = q0
        for l in range(1, len(levels)):
            lv = levels[l]
            if k >= lv.N:
                break
            q = _update(lv.n_fine, y[: lv.s], lam0, u0, lv0.n_fine, a0, decay, family, qoi)
            out[l, i] = (lam0, q, prev, q - prev)
            prev = q
    return out


def estimate_shared(level_shift_means):
    """Estimate and standard error with shared shifts.  The levels are no longer independent, but
    the per-shift totals Q^(r) = sum_l Q^(r)_l are (one independent shift each): the estimate is
    their mean and its variance is estimated by their sample variance (eq. sample_var applied to
    the totals).  Returns (Qhat^ML, SE, Qhat_l[], Vhat_l[]) with the per-level values of eq.
    sample_var for information."""
    q = np.asarray(level_shift_means, dtype=np.float64)  # [L+1, R]
    R = q.shape[1]
    if R < 2:
        raise ValueError("the sample-variance estimate needs R >= 2 shifts")
    tot = q.sum(axis=0)
    m = tot.sum() / R
    var = ((m - tot) ** 2).sum() / (R * (R - 1))
    _, _, qhat, vhat = estimate(q)
    return float(m), float(np.sqrt(var)), qhat, vhat


# ---------------------------------------------------------------------------------------------
# Adaptive choice of the point counts and the number of levels (Sec. 4.2: the adaptive algorithm
# the paper takes from Giles & Waterhouse for multilevel QMC).  Reading used here:
#   1. start with levels 0..2, each with n_init points (an embedded rule, so a level's points can
#      be doubled by evaluating the next n of them);
#   2. while the sum of the level variances (eq. sample_var) exceeds eps^2 / 2: double the points
#      of the level with the largest Vhat_l / (C_l N_l) -- the largest variance per unit of the cost
#      of doubling it (C_l: cost per sample) -- among the levels that can still double (ties: the
#      lowest level); stop unconverged when none can;
#   3. bias test with weak order alpha (the level differences shrink like 2^(-alpha l)):
#      max(|Qhat_L|, |Qhat_{L-1}| / 2^alpha) <= (2^alpha - 1) eps / sqrt(2) ends the run; otherwise
#      add level L + 1 with n_init points and return to 2 (unconverged when no level is left).
# Estimate: sum_l Qhat_l with SE = sqrt(sum_l Vhat_l) (independent shifts per level).

def adaptive(evaluate, cost, R: int, eps: float, alpha: float = 2.0, n_init: int = 8, n_max=None,
             L_max: int = None):
    """Runs the adaptive algorithm.  evaluate(l, k0, k1) returns the level differences [R, k1 - k0]
    of level l at points k0 .. k1 - 1; cost[l] is the cost per sample of level l; n_max[l] the
    points level l can have (default unbounded); L_max the last level available (default
    len(cost) - 1).  Returns a dict with L, N (points per level), mean, std_err, level_mean,
    level_var, converged, and the history of (level, new N) doublings and level additions."""
    L_max = len(cost) - 1 if L_max is None else L_max
    n_max = n_max or [1 << 62] * (L_max + 1)
    sums, N, history = [], [], []

    def add(l, n_new):
        if l == len(N):
            sums.append(np.zeros(R))
            N.append(0)
        d = np.asarray(evaluate(l, N[l], n_new), dtype=np.float64)
        sums[l] = sums[l] + d.sum(axis=1)
        N[l] = n_new
        history.append((l, n_new))

    def level_stats():
        means, vars_ = [], []
        for l in range(len(N)):
            q = sums[l] / N[l]
            m = q.sum() / R
            means.append(m)
            vars_.append(((m - q) ** 2).sum() / (R * (R - 1)))
        return means, vars_

    for l in range(min(3, L_max + 1)):
        add(l, n_init)
    converged = False
    while True:
        means, vars_ = level_stats()
        stuck = False
        while sum(vars_) > eps * eps / 2.0:
            score = [vars_[l] / (cost[l] * N[l]) if 2 * N[l] <= n_max[l] else -1.0 for l in range(len(N))]
            best = max(score)
            if best < 0.0:
                stuck = True
                break
            l = score.index(best)
            add(l, 2 * N[l])
            means, vars_ = level_stats()
        if stuck:
            break
        L = len(N) - 1
        if L >= 2:
            bias = max(abs(means[L]), abs(means[L - 1]) / 2.0 ** alpha)
            if bias <= (2.0 ** alpha - 1.0) * eps / np.sqrt(2.0):
                converged = True
                break
        if L >= L_max:
            break
        add(L + 1, n_init)
    means, vars_ = level_stats()
    return {"L": len(N) - 1, "N": list(N), "mean": float(sum(means)), "std_err": float(np.sqrt(sum(vars_))),
            "level_mean": means, "level_var": vars_, "converged": converged, "history": history}
