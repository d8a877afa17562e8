"""The graph schedule: several levels' point ranges captured as one CUDA graph (the streaming
tier's loops as conditional WHILE nodes set on the device, no host reads) and replayed with one
launch, against the level-by-level calls: per-sample results, shift sums and the estimate equal
bit for bit, also when the graph is replayed on other point ranges, with iteration caps and in the
reuse scheme."""
import numpy as np
import pytest

from oracle import lattice
from synthetic_inputs import Level, shared_shifts, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


# per-sample tier (1/16), streaming tier with the on-chip sub-cycle (1/32) and with streamed
# V-cycle levels (1/64, 1/128)
LEVELS = [Level(16, 8, 16, 4, 64, 3), Level(32, 8, 32, 6, 64, 3), Level(64, 16, 64, 8, 32, 3),
          Level(128, 16, 128, 12, 16, 3)]


def _ctx(B, prec=1, seed=4):
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, 128, 0, 2.0)
    ctx.mq_set_levels(LEVELS)
    ds = shifts(seed, LEVELS)
    for l, lv in enumerate(LEVELS):
        ctx.mq_set_lattice(l, lattice.cbc(lv.N, lv.s))
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    return ctx


def _run_both(B, ctx_g, ctx_l, ranges, launches):
    """Captures `ranges` on ctx_g and replays it once per entry of `launches` (start points or
    None); runs the same ranges level by level on ctx_l; compares everything."""
    outs = [torch.empty((LEVELS[l].R, k1 - k0, 4), dtype=torch.float64, device="cuda") for l, k0, k1 in ranges]
    sums = [torch.empty(LEVELS[l].R, dtype=torch.float64, device="cuda") for l, _, _ in ranges]
    ctx_g.mq_graph_capture(ranges, outs, sums)
    cap, nodes = ctx_g.mq_get_graph_info()
    assert cap and nodes > 0
    for starts in launches:
        try:
            ctx_g.mq_graph_launch(starts)
            gstat = None
        except B.MQNoConvergence as e:
            gstat = e.status
        cur = [(l, (starts[i] if starts else k0), (starts[i] if starts else k0) + (k1 - k0))
               for i, (l, k0, k1) in enumerate(ranges)]
        for i, (l, k0, k1) in enumerate(cur):
            ref = torch.empty_like(outs[i])
            rs = torch.empty_like(sums[i])
            try:
                ctx_l.mq_eval_level_device(l, k0, k1, ref, rs)
                lstat = None
            except B.MQNoConvergence as e:
                lstat = e.status
            assert torch.equal(outs[i], ref), (i, l, k0, k1)
            assert torch.equal(sums[i], rs), (i, l)
            if gstat is None:
                assert lstat is None
    for l in sorted({r[0] for r in ranges}):
        (sa, na), (sb, nb) = ctx_g.mq_get_sums(l), ctx_l.mq_get_sums(l)
        assert na == nb and np.array_equal(sa, sb)
    if len({r[0] for r in ranges}) == len(LEVELS):
        ma, sa, la, va = ctx_g.mq_estimate()
        mb, sb, lb, vb = ctx_l.mq_estimate()
        assert ma == mb and sa == sb and np.array_equal(la, lb) and np.array_equal(va, vb)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_equals_level_by_level(B, prec):
    ctx_g, ctx_l = _ctx(B, prec), _ctx(B, prec)
    ranges = [(0, 0, 16), (1, 0, 16), (2, 0, 8), (3, 0, 4)]
    # the captured ranges twice, then the graph moved to later points
    _run_both(B, ctx_g, ctx_l, ranges, [None, None, [16, 24, 8, 12]])
    ctx_g.close()
    ctx_l.close()


def test_graph_with_iteration_caps(B):
    # one MINRES iteration and one refinement step (odd cap: the graph's paired iterations end on
    # the device counter), and two: both schedules flag the same samples and write the same values
    for cap in (1, 2):
        ctx_g, ctx_l = _ctx(B, 1), _ctx(B, 1)
        for c in (ctx_g, ctx_l):
            c.mq_set_solver_options(0.0, cap, cap)
        _run_both(B, ctx_g, ctx_l, [(2, 0, 4), (3, 0, 4)], [None])
        ctx_g.close()
        ctx_l.close()


def test_graph_in_the_reuse_scheme_and_invalidation(B):
    levels = [Level(16, 16, 16, 16, 32, 3), Level(32, 16, 32, 16, 16, 3), Level(64, 16, 64, 16, 8, 3)]
    z = lattice.embedded_cbc(1, 5, 64)
    ds = shared_shifts(8, levels)

    def mk():
        c = B.Context(0)
        c.mq_set_coefficient(1.0, 64, 0, 2.0)
        c.mq_set_levels(levels)
        for l, lv in enumerate(levels):
            c.mq_set_lattice_embedded(l, z[: lv.s], 5)
            c.mq_set_shifts(l, ds[l])
        c.mq_set_precision(1)
        c.mq_set_reuse(1)
        return c

    ctx_g, ctx_l = mk(), mk()
    ranges = [(0, 0, 16), (1, 0, 8), (2, 0, 8)]
    outs = [torch.empty((3, k1 - k0, 4), dtype=torch.float64, device="cuda") for _, k0, k1 in ranges]
    ctx_g.mq_graph_capture(ranges, outs, None)
    ctx_g.mq_graph_launch()
    for i, (l, k0, k1) in enumerate(ranges):
        ref = torch.empty_like(outs[i])
        ctx_l.mq_eval_level_device(l, k0, k1, ref, None)
        assert torch.equal(outs[i], ref)
    # a setter drops the graph
    ctx_g.mq_set_smoothing(1)
    assert ctx_g.mq_get_graph_info() == (False, 0)
    with pytest.raises(B.MQError) as e:
        ctx_g.mq_graph_launch()
    assert e.value.status == B.MQ_ESTATE
    ctx_g.close()
    ctx_l.close()
