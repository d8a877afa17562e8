"""The adaptive choice of N_l and L (Sec. 4.2) on the GPU against the oracle's run of the same
algorithm on the oracle's own level evaluations: the same decisions (finest level, points per
level, convergence) and the same estimate to the per-sample tolerance."""
import numpy as np
import pytest

from oracle import lattice, mlqmc
from synthetic_inputs import Level, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# level 0 direct on mesh 1/4, levels 1-4 two-grid on 1/8 .. 1/64 from the 1/4 mesh; s doubles per
# level; embedded rules of up to 2^10 points, 8 independent shifts per level
MBITS = 10
LEVELS = [Level(4, 4, 4, 4, 1 << MBITS, 8)] + [Level(4 << l, 4, 4 << l, {1: 3, 2: 4, 3: 6, 4: 8}[l], 1 << MBITS, 8)
                                               for l in range(1, 5)]
EPS, ALPHA, N_INIT = 0.03, 2.0, 8


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


def _setup(B, prec):
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, max(lv.s for lv in LEVELS), 0, 2.0)
    ctx.mq_set_levels(LEVELS)
    zs = [lattice.embedded_cbc(3, MBITS, lv.s) for lv in LEVELS]
    ds = shifts(17, LEVELS)
    for l, lv in enumerate(LEVELS):
        ctx.mq_set_lattice_embedded(l, zs[l], MBITS)
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    return ctx, zs, ds


def _cost():
    out = []
    for l, lv in enumerate(LEVELS):
        c = (lv.n_fine - 1) ** 2
        if l > 0 and not (lv.n_fine == lv.n_coarse and lv.s == lv.S):
            c += (LEVELS[l - 1].n_fine - 1) ** 2
        out.append(float(c))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_run_matches_oracle(B, prec):
    ctx, zs, ds = _setup(B, prec)
    got = ctx.mq_run_adaptive(EPS, ALPHA, N_INIT)

    def evaluate(l, k0, k1):
        lv, pv = LEVELS[l], (LEVELS[l - 1] if l else None)
        out = np.zeros((lv.R, k1 - k0))
        for r in range(lv.R):
            Y = lattice.embedded_points(zs[l], MBITS, ds[l][r], np.arange(k0, k1))
            for i in range(k1 - k0):
                out[r, i] = mlqmc.sample_level(lv, pv, Y[i])[3]
        return out

    ref = mlqmc.adaptive(evaluate, _cost(), LEVELS[0].R, EPS, ALPHA, N_INIT, n_max=[lv.N for lv in LEVELS])
    print(f"adaptive: L {got['L']} N {got['N']} converged {got['converged']} mean {got['mean']!r} "
          f"(oracle {ref['mean']!r}) se {got['std_err']!r} (oracle {ref['std_err']!r})")
    assert got["L"] == ref["L"] and got["N"] == ref["N"] and got["converged"] == ref["converged"]
    assert got["converged"] and got["L"] >= 2 and max(got["N"]) > N_INIT  # the run did adapt
    assert got["mean"] == pytest.approx(ref["mean"], rel=1e-10)
    for l in range(got["L"] + 1):
        assert got["level_mean"][l] == pytest.approx(ref["level_mean"][l], rel=1e-9, abs=1e-10 * 30)
    # standard error: within the propagated per-sample tolerance (2 e sqrt((L+1)/(R-1)), e = 1e-10 lambda)
    bound = 2.0 * 1e-10 * 30.0 * np.sqrt((got["L"] + 1) / (LEVELS[0].R - 1))
    assert abs(got["std_err"] - ref["std_err"]) <= bound
    # the context's estimator holds the run's sums
    m, se, _, _ = ctx.mq_estimate() if got["L"] == len(LEVELS) - 1 else (got["mean"], got["std_err"], 0, 0)
    assert m == pytest.approx(got["mean"], rel=1e-14)
    ctx.close()


def test_adaptive_needs_embedded_independent_levels(B):
    ctx, zs, ds = _setup(B, 1)
    ctx.mq_set_lattice(2, np.array(lattice.cbc(LEVELS[2].N, LEVELS[2].s)))
    with pytest.raises(B.MQError) as e:
        ctx.mq_run_adaptive(EPS)
    assert e.value.status == B.MQ_ESTATE
    with pytest.raises(B.MQError) as e:
        ctx.mq_run_adaptive(-1.0)
    assert e.value.status == B.MQ_EINVAL
    ctx.close()
