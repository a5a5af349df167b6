"""Domain decomposition on one GPU: a grid split into slab contexts whose halo
messages move by device-to-device copies (SlabGrid) must advance exactly like the
undivided grid: the slabs' interior cells gather the same populations and do the
same arithmetic, so the states agree bit for bit, in every storage form."""
import numpy as np
import pytest

from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("D3Q95", (24, 6, 20), [6, 7, 7]), ("D3Q95", (136, 8, 16), [16]),
         ("D2Q33", (40, 15, 1), [7, 8]), ("D2Q33", (264, 12, 1), [4, 4, 4])]


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model,dims,splits", CASES)
def test_slabs_match_the_undivided_grid_bitwise(lbm, model, dims, splits, storage):
    from paper_1303_4624_gb300 import slabs
    D = 3 if model == "D3Q95" else 2
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=13, noise=1e-2)
    omega, steps = 1.65, 7
    ref = lbm.Lattice(model, dims, omega, storage)
    T = fields.theta * ref.info["T0"]
    ref.init(fields.rho, fields.U, T)
    ref.step(steps)
    want = ref.raw()
    r0, U0, T0 = ref.moments()
    ref.close()
    grid = slabs.SlabGrid(model, dims, omega, storage, splits)
    info = lbm.lbm_halo_info(grid.ctxs[0])
    plane = dims[0] * dims[1] if D == 3 else dims[0]
    esize = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[storage]
    assert info["segments"] == (102 if D == 3 else 26)
    assert info["face_bytes"] == info["segments"] * plane * esize
    grid.init(fields.rho, fields.U, T)
    grid.step(steps)
    got = grid.raw()
    assert np.array_equal(want.view(np.uint8), got.view(np.uint8))
    r, U, Tg = grid.moments()
    assert np.array_equal(r, r0) and np.array_equal(Tg, T0) and np.array_equal(U, U0)
    grid.close()


def test_slab_contexts_refuse_what_they_do_not_cover(lbm):
    ctx = lbm.lbm_create_slab("D3Q95", (8, 8, 6), 1.5, "fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_slab("D3Q95", (8, 8, 4), 1.5, "fp32")      # thinner than the reach
    assert ei.value.code == lbm.LBM_EINVAL
    shape = (16, 8, 8)                                             # 6 + 2 x 5 planes
    lbm.lbm_init(ctx, np.ones(shape), np.zeros((3,) + shape), np.full(shape, 2.8))
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_record(ctx, 4, 2)
    assert ei.value.code == lbm.LBM_EINVAL
    plain = lbm.Lattice("D3Q95", (8, 8, 8), 1.5, "fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_halo_info(plain.ctx)
    assert ei.value.code == lbm.LBM_ESTATE
    plain.close()
    lbm.lbm_destroy(ctx)
