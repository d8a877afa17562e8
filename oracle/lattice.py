"""Randomly shifted rank-1 lattice rules and CBC generating vectors (Sec. 2.5).

Test infrastructure only (see ``oracle/__init__.py``).

* Points: t_k = {k z / N}, shifted y_k = {t_k + Delta} - 1/2 (eq. rqmc, eq. t_kl),
  for k = 0, ..., N-1.
* CBC: the component-by-component construction for the shift-averaged
  worst-case error in the unanchored weighted Sobolev space of eq. W-norm with
  product weights gamma_u = prod_{j in u} gamma_j.  Its squared error for a
  generating vector z is

      e^2(z) = -1 + (1/N) sum_{k=0}^{N-1} prod_j (1 + gamma_j B2({k z_j / N})),

  with B2(x) = x^2 - x + 1/6 the Bernoulli polynomial of degree 2.  Component j
  takes the candidate z in [1, N/2] with gcd(z, N) = 1 that minimises e^2 given
  the earlier components; candidates within an absolute 1e-12 of the minimum
  count as tied and the smallest of them is taken.  (e^2 is a difference of
  order-one sums, so rounding alone separates candidates that tie exactly, such
  as every candidate for the first component, by up to ~1e-15; the tie window
  absorbs that.)
"""
from __future__ import annotations

import math

import numpy as np


def bernoulli2(x: np.ndarray) -> np.ndarray:
    return x * x - x + 1.0 / 6.0


def cbc_error2(z, N: int, gamma) -> float:
    """Shift-averaged squared worst-case error e^2(z) written out as a plain double loop."""
    total = 0.0
    for k in range(N):
        prod = 1.0
        for j, zj in enumerate(z):
            prod *= 1.0 + gamma[j] * bernoulli2(((k * zj) % N) / N)
        total += prod
    return -1.0 + total / N


def cbc(N: int, s: int, decay: float = 2.0, tie_atol: float = 1e-12) -> np.ndarray:
    """Generating vector z (length s) by CBC with product weights gamma_j = j^-decay."""
    gamma = np.array([(j + 1) ** (-decay) for j in range(s)])
    k = np.arange(N, dtype=np.int64)
    cands = np.array([c for c in range(1, N // 2 + 1) if math.gcd(c, N) == 1] or [1], dtype=np.int64)
    prod = np.ones(N)  # prod over chosen components of (1 + gamma_j B2({k z_j / N}))
    z = []
    step = max(1, (1 << 22) // N)  # candidates per block, bounds the [cand, k] work array
    for j in range(s):
        e2 = np.empty(cands.size)
        for c0 in range(0, cands.size, step):
            frac = ((np.outer(cands[c0:c0 + step], k)) % N) / N  # [cand, k]
            e2[c0:c0 + step] = -1.0 + np.mean(prod[None, :] * (1.0 + gamma[j] * bernoulli2(frac)), axis=1)
        best = e2.min()
        pick = int(cands[np.nonzero(e2 <= best + tie_atol)[0][0]])
        z.append(pick)
        prod = prod * (1.0 + gamma[j] * bernoulli2(((k * pick) % N) / N))
    return np.array(z, dtype=np.int64)


def points(z, N: int, delta, k) -> np.ndarray:
    """Shifted lattice points y_k = {k z / N + Delta} - 1/2 in [-1/2, 1/2)^s (eq. rqmc).

    ``k`` may be an int or an array of indices; the result has shape [len(k), s].
    """
    z = np.asarray(z, dtype=np.int64)
    delta = np.asarray(delta, dtype=np.float64)
    kk = np.atleast_1d(np.asarray(k, dtype=np.int64))
    t = ((kk[:, None] * z[None, :]) % N) / N  # {k z / N}
    return np.mod(t + delta[None, :], 1.0) - 0.5


# ---------------------------------------------------------------------------------------------
# Embedded lattice rules (Sec. 2.5): one generating vector that works for every N = 2^m with
# m_min <= m <= m_max, and whose point sets are nested.
#
# The paper cites the embedded construction without stating its error criterion.  Reading used
# here: component by component, every odd candidate c in [1, 2^(m_max - 1)) is scored for every m
# by the ratio of the squared shift-averaged worst-case error of the 2^m-point rule with c
# appended, e^2_{2^m}(z_1, ..., z_{j-1}, c), to the smallest such error over the candidates
# (the best that component j could do for that N alone, given the earlier components); the
# candidate with the smallest worst ratio over m is taken.  Odd candidates are exactly those
# coprime to every power of two, and c and 2^m - c give the same point set, so they cover every
# distinct choice.  The errors are formed as means of the excess P_k - 1 of the running products
# (no cancellation against the constant 1), and ratios within a relative 1e-6 of the minimum count
# as tied (the rounding of e^2 at the largest N stays some orders below that); the smallest tied
# candidate wins.
#
# Point order: the radical inverse in base 2.  Point k (0 <= k < 2^m_max) is
#     x_k = {rev(k) z / 2^m_max + Delta} - 1/2,
# with rev(k) the m_max-bit reversal of k.  The first 2^m points are then exactly the 2^m-point
# rule {i z / 2^m}, i < 2^m (in another order), so a level that uses N = 2^m points evaluates a
# prefix of the sequence, and doubling N adds the next 2^m points.

EMBEDDED_TIE_RTOL = 1e-6


def embedded_cbc(m_min: int, m_max: int, s: int, decay: float = 2.0) -> np.ndarray:
    """Generating vector z (length s) of an embedded lattice rule for N = 2^m_min ... 2^m_max."""
    assert 0 <= m_min <= m_max
    gamma = np.array([(j + 1) ** (-decay) for j in range(s)])
    Nmax = 1 << m_max
    cands = np.arange(1, max(2, Nmax // 2), 2, dtype=np.int64)
    ms = list(range(m_min, m_max + 1))
    excess = {m: np.zeros(1 << m) for m in ms}  # prod over chosen components minus one, per N = 2^m
    z = []
    for j in range(s):
        worst = np.zeros(cands.size)
        for m in ms:
            N = 1 << m
            k = np.arange(N, dtype=np.int64)
            q = excess[m]
            e2 = np.empty(cands.size)
            step = max(1, (1 << 22) // N)
            for c0 in range(0, cands.size, step):
                a = gamma[j] * bernoulli2((np.outer(cands[c0:c0 + step], k) % N) / N)
                # e^2 = mean_k prod_j (1 + gamma_j B2) - 1 = mean_k [q + a (1 + q)]
                e2[c0:c0 + step] = np.mean(q[None, :] + a * (1.0 + q[None, :]), axis=1)
            worst = np.maximum(worst, e2 / e2.min())
        best = worst.min()
        pick = int(cands[np.nonzero(worst <= best * (1.0 + EMBEDDED_TIE_RTOL))[0][0]])
        z.append(pick)
        for m in ms:
            N = 1 << m
            k = np.arange(N, dtype=np.int64)
            a = gamma[j] * bernoulli2(((k * pick) % N) / N)
            excess[m] = excess[m] + a * (1.0 + excess[m])
    return np.array(z, dtype=np.int64)


def bit_reverse(k, bits: int):
    """The `bits`-bit reversal of the integers in k."""
    k = np.asarray(k, dtype=np.int64)
    out = np.zeros_like(k)
    for b in range(bits):
        out |= ((k >> b) & 1) << (bits - 1 - b)
    return out


def embedded_points(z, m_max: int, delta, k) -> np.ndarray:
    """Shifted points of the embedded rule in radical-inverse order, [len(k), s]:
    x_k = {rev(k) z / 2^m_max + Delta} - 1/2."""
    kk = np.atleast_1d(np.asarray(k, dtype=np.int64))
    return points(z, 1 << m_max, delta, bit_reverse(kk, m_max))
