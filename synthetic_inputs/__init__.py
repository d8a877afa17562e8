"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: only the workload table (mesh
widths, truncation dimensions, point counts, shift counts, seeds) and seeded
random draws.  Everything the method computes from these inputs (lattice
generating vectors, lattice points, coefficients, eigenpairs) is implemented
separately on each side.

Random shifts (Sec. 2.5, randomly shifted rank-1 lattice rules): the paper does
not name a generator.  The shifts are drawn with
``numpy.random.default_rng(seed).random((R, s_l))``, level by level for
l = 0..L in order, and passed to both sides as inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass(frozen=True)
class Level:
    """One MLQMC level: fine mesh 1/n_fine, coarse mesh 1/n_coarse, truncations s and S,
    N lattice points and R shifts.  n_coarse == n_fine with S == s marks a direct
    (non-two-grid) eigensolve on that level."""

    n_fine: int
    n_coarse: int
    s: int
    S: int
    N: int
    R: int


@dataclass(frozen=True)
class Workload:
    name: str
    levels: List[Level]
    seed: int
    precision: str  # "fp64" or "mixed"
    tol: float  # relative tolerance on each per-sample eigenvalue versus the oracle
    a0: float = 1.0
    decay: float = 2.0
    family: int = 0  # 0: the workload sine family; 1, 2: the paper's first and second test problems (Sec. 5)
    notes: str = ""
    extra: dict = field(default_factory=dict)
    decays: tuple = ()  # family 2: the term decays (p_a, p_a', p_b, p_b'); `decay` then weights the lattice

    @property
    def samples(self) -> int:
        return sum(lv.N * lv.R for lv in self.levels)

    @property
    def coef_decay(self):
        """The decay argument of the coefficient: the four decays of family 2, else ``decay``."""
        return self.decays if self.family == 2 else self.decay


def _ceil_sqrt(s: int) -> int:
    r = int(np.floor(np.sqrt(s)))
    while r * r < s:
        r += 1
    return r


# The workloads.  Coarse truncation S = ceil(sqrt(s)) (Sec. 4.3);
# coarse meshes as read for each workload.
WORKLOADS = {
    # single level, FP64: h = 1/16 (225 dofs), H = 1/8, s = 16, S = 4, N = 256, R = 8, seed 0
    "qmc_h16_s16": Workload(
        "qmc_h16_s16",
        [Level(16, 8, 16, 4, 256, 8)],
        seed=0, precision="fp64", tol=1e-10,
    ),
    # 4-level MLQMC, FP64: h = 1/16..1/128, H = 1/8,1/8,1/16,1/16, s = 16..128
    "mlqmc4_h16_128": Workload(
        "mlqmc4_h16_128",
        [
            Level(16, 8, 16, _ceil_sqrt(16), 4096, 16),
            Level(32, 8, 32, _ceil_sqrt(32), 2048, 16),
            Level(64, 16, 64, _ceil_sqrt(64), 1024, 16),
            Level(128, 16, 128, _ceil_sqrt(128), 512, 16),
        ],
        seed=1, precision="fp64", tol=1e-10,
    ),
    # single level h = 1/512, H = 1/32, s = 256, S = 16, 64 points x 16 shifts
    "single_h512_s256": Workload(
        "single_h512_s256",
        [Level(512, 32, 256, 16, 64, 16)],
        seed=2, precision="mixed", tol=1e-10,
    ),
    # 6-level MLQMC h = 1/32..1/1024, level 0 direct (H = h0 = 1/32, S = s0)
    "mlqmc6_h32_1024": Workload(
        "mlqmc6_h32_1024",
        [Level(32, 32, 32, 32, 16384, 16)]
        + [Level(32 << l, 32, 32 << l, _ceil_sqrt(32 << l), 16384 >> l, 16) for l in range(1, 6)],
        seed=3, precision="mixed", tol=1e-10,
    ),
    # the paper's first test problem (Sec. 5): psi_j = j^-p sin(j pi x1) sin((j+1) pi x2) with
    # p = 4/3 and a0 = pi / sqrt(2), s = 64 terms, S = 8, H = 1/8, h_l = 2^-(l+3) (level 0 direct),
    # R = 8 shifts; point counts halve level by level
    "paper_p1_h8_64": Workload(
        "paper_p1_h8_64",
        [Level(8, 8, 64, 64, 2048, 8)] + [Level(8 << l, 8, 64, _ceil_sqrt(64), 2048 >> l, 8) for l in range(1, 4)],
        seed=5, precision="mixed", tol=1e-10, a0=float(np.pi / np.sqrt(2.0)), decay=4.0 / 3.0, family=1,
    ),
    # the paper's second test problem (Sec. 5: four islands, parametric reaction term) with decays
    # p_a = p_b = 4/3 on the islands and p_a' = p_b' = 2 off them (the left case of the paper's
    # figure), s = 64 terms, S = 8, H = 1/8, h_l = 2^-(l+3) (level 0 direct; every mesh resolves the
    # islands), R = 8 shifts, point counts halving level by level; lattice weights j^-(4/3)
    "paper_p2_h8_64": Workload(
        "paper_p2_h8_64",
        [Level(8, 8, 64, 64, 2048, 8)] + [Level(8 << l, 8, 64, _ceil_sqrt(64), 2048 >> l, 8) for l in range(1, 4)],
        seed=7, precision="mixed", tol=1e-10, decay=4.0 / 3.0, family=2, decays=(4.0 / 3.0, 2.0, 4.0 / 3.0, 2.0),
    ),
    # shared shifts and nested points with reuse (Sec. 4.3, after Algorithm 2): h_l = 1/16 .. 1/128,
    # s_l = 16 .. 128, level 0 direct on (h_0, s_0) = (1/16, 16); every level l >= 1 takes its coarse
    # pair from level 0 (H_l = h_0, S_l = s_0); one embedded lattice rule for N = 2^9 .. 2^12 in
    # radical-inverse order; one set of 16 shifts drawn with s_L = 128 components
    "shared_mlqmc4_h16_128": Workload(
        "shared_mlqmc4_h16_128",
        [Level(16, 16, 16, 16, 4096, 16)] + [Level(16 << l, 16, 16 << l, 16, 4096 >> l, 16) for l in range(1, 4)],
        seed=6, precision="mixed", tol=1e-10, extra={"shared": True, "m_min": 9, "m_max": 12},
    ),
    # h = 1/1024 (1,046,529 dofs), H = 1/64, s = 1024, S = 32, 32 points x 16 shifts
    "stress_h1024_s1024": Workload(
        "stress_h1024_s1024",
        [Level(1024, 64, 1024, 32, 32, 16)],
        seed=4, precision="mixed", tol=1e-10,
    ),
}


def shifts(seed: int, levels: List[Level]) -> List[np.ndarray]:
    """Random shifts Delta_l in [0,1)^{R x s_l}, drawn level by level from one generator."""
    rng = np.random.default_rng(seed)
    return [rng.random((lv.R, lv.s)) for lv in levels]


def shifts_for_rank(seed: int, levels: List[Level], rank: int, world: int) -> List[np.ndarray]:
    """The shifts of one rank when `world` processes share one workload: R * world shifts per level
    drawn as in ``shifts`` (level by level from one generator), rank i taking rows
    [i R, (i + 1) R).  With world = 1 these are the workload's own shifts."""
    rng = np.random.default_rng(seed)
    return [rng.random((lv.R * world, lv.s))[rank * lv.R:(rank + 1) * lv.R] for lv in levels]


def shared_shifts(seed: int, levels: List[Level], rank: int = 0, world: int = 1) -> List[np.ndarray]:
    """One set of shifts Delta in [0,1)^{R x s_L} for every level (the reuse scheme): level l takes
    the first s_l components.  With `world` processes, R * world shifts are drawn and rank i takes
    rows [i R, (i + 1) R)."""
    rng = np.random.default_rng(seed)
    R = levels[0].R
    full = rng.random((R * world, max(lv.s for lv in levels)))[rank * R:(rank + 1) * R]
    return [full[:, : lv.s].copy() for lv in levels]


def random_points(seed: int, count: int, s: int) -> np.ndarray:
    """Uniform parameter vectors y in [-1/2, 1/2)^s for single-point tests."""
    rng = np.random.default_rng(seed)
    return rng.random((count, s)) - 0.5


def random_vectors(seed: int, count: int, n: int) -> np.ndarray:
    """Standard normal test vectors (operator-apply tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, n))


def random_cell_coefficients(seed: int, count: int, n: int, lo: float = 0.2, hi: float = 1.8) -> np.ndarray:
    """Per-triangle coefficients in [lo, hi): layout [count][2][n][n] (lower / upper triangle
    of cell (i, j) at [.][0][j][i] / [.][1][j][i])."""
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((count, 2, n, n))
