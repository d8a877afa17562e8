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
