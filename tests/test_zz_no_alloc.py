"""The allocation-free entry point against the regular one.

mq_twogrid_samples_noalloc serves callers that may not allocate device memory (code running
under someone else's graph capture, plugins with a fixed memory pool, real-time services): it
keeps the per-block workspace in a fixed array inside the library and takes every input and
output from the caller.  Here it must give the same per-sample results as mq_eval_level for the
same samples, on two calls in a row (the second call finds the first call's leftovers in the
shared array).  The file is named to be collected last.
"""
import numpy as np
import pytest

from synthetic_inputs import Level, shifts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2103_03407_gb300 import binding, build

    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    return binding


GEOMETRIES = [
    # a level whose workspace does not fit in shared memory: 1/64 fine mesh, 1/32 previous fine
    # mesh, 1/16 coarse mesh
    [Level(32, 16, 32, 6, 64, 2), Level(64, 16, 64, 8, 64, 2)],
    # the previous fine mesh is the coarse mesh itself (a longer truncation on the same mesh): a
    # nearly singular shifted system, solved with an FP64 inner solve in both precisions
    [Level(16, 8, 16, 4, 64, 2), Level(32, 16, 32, 6, 64, 2)],
]


@pytest.mark.parametrize("geom", range(len(GEOMETRIES)))
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_regular_entry_point(B, prec, geom):
    levels = GEOMETRIES[geom]
    lv, pv = levels[1], levels[0]
    nf, nc, npv = lv.n_fine, lv.n_coarse, pv.n_fine
    ctx = B.Context(0)
    ctx.mq_set_coefficient(1.0, 64, 0, 2.0)
    ctx.mq_set_levels(levels)
    ds = shifts(7, levels)
    for l, L in enumerate(levels):
        ctx.mq_set_lattice(l, B.mq_cbc_lattice(L.N, L.s))
        ctx.mq_set_shifts(l, ds[l])
    ctx.mq_set_precision(prec)
    k0, k1 = 3, 15
    npts = k1 - k0
    ref, _ = ctx.mq_eval_level(1, k0, k1)  # regular entry point: [R][npts][4]

    # the same samples' coefficients, evaluated with the regular building blocks
    nb = lv.R * npts
    dY = torch.empty((lv.R, npts, lv.s), dtype=torch.float64, device="cuda")
    ctx.mq_lattice_points_device(1, k0, k1, dY)
    a_c = torch.empty((nb, 2 * nc * nc), dtype=torch.float64, device="cuda")
    a_f = torch.empty((nb, 2 * nf * nf), dtype=torch.float64, device="cuda")
    a_p = torch.empty((nb, 2 * npv * npv), dtype=torch.float64, device="cuda")
    ctx.mq_coefficients_device(nc, lv.S, dY, nb, lv.s, a_c)
    ctx.mq_coefficients_device(nf, lv.s, dY, nb, lv.s, a_f)
    ctx.mq_coefficients_device(npv, pv.s, dY, nb, lv.s, a_p)

    for call in range(2):
        out = torch.full((nb, 4), float("nan"), dtype=torch.float64, device="cuda")
        stat = torch.full((nb, 4), -1, dtype=torch.int32, device="cuda")
        outer = torch.zeros((nb, 2), dtype=torch.int32, device="cuda")
        B.mq_twogrid_samples_noalloc(nf, nc, npv, prec, nb, a_f, a_c, a_p, out, stat, outer)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(lv.R, npts, 4)
        assert np.all(stat.cpu().numpy()[:, 3] == 0), f"call {call}: flags set"
        assert np.all(np.abs(got[..., 0] - ref[..., 0]) <= 1e-12 * np.abs(ref[..., 0])), f"call {call}"
        for c in (1, 2):
            assert np.all(np.abs(got[..., c] - ref[..., c]) <= 1e-10 * np.abs(ref[..., c])), f"call {call}"
        assert np.all(np.abs(got[..., 3] - ref[..., 3]) <= 2e-10 * np.abs(ref[..., 1])), f"call {call}"
    ctx.close()


def test_noalloc_rejects_workspace_beyond_the_fixed_array(B):
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(B.MQError) as e:
        # one block's workspace on a 1/4096 mesh is far above the fixed 32 MiB array
        B.mq_twogrid_samples_noalloc(4096, 64, 0, 1, 1, dummy, dummy, None, dummy, st, st)
    assert e.value.status == B.MQ_EINVAL
