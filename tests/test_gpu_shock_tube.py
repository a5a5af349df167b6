"""The paper's shock tube on the GPU: fixed-state end planes (lbm_set_fixed_ends)."""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import riemann
from oracle.model import get_model
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu


def tube_fields(D, dims, axis, lo, hi):
    shape = dims[::-1]
    idx = np.indices(shape)[2 - axis]            # coordinate along the tube axis
    n = dims[axis]
    rho = np.where(idx < n // 2, lo[0], hi[0]).astype(float)
    T = np.where(idx < n // 2, lo[-1], hi[-1]).astype(float)
    return rho, np.zeros((D,) + shape), T


@pytest.mark.parametrize("model,dims,axis", [("D3Q95", (3, 2, 240), 2), ("D2Q33", (200, 3, 1), 0)])
def test_fixed_ends_match_oracle_fp64(lbm, model, dims, axis):
    mdl = get_model(model)
    D, T0 = mdl.D, mdl.T0
    lo = [4.0] + [0.0] * D + [T0]
    hi = [1.0] + [0.0] * D + [1.1 * T0]
    rho, U, T = tube_fields(D, dims, axis, lo, hi)
    width = mdl.reach
    S = olbm.init_populations(mdl, rho, U, T)
    ends = (axis, width, (lo[0], np.array(lo[1:1 + D]), lo[-1]), (hi[0], np.array(hi[1:1 + D]), hi[-1]))
    S = olbm.run(mdl, S, 1.5, 30, ends)
    lat = lbm.Lattice(model, dims, 1.5, "fp64")
    lat.init(rho, U, T)
    lbm.lbm_set_fixed_ends(lat.ctx, axis, width, lo, hi)
    lat.step(30)
    compare(mdl, S, lat, 1e-12)


def test_paper_tube_11x11x800_plateaus(lbm):
    """Full geometry of the paper (11 x 11 x 800, D3Q95, omega 1.5, rho = p = 4 | 1,
    theta = 1, end planes C_L / C_R), FP32: both plateaus within 0.5 % of the exact
    Riemann solution after 150 steps."""
    mdl = get_model("D3Q95")
    T0, dims, steps = mdl.T0, (11, 11, 800), 150
    lo, hi = [4.0, 0.0, 0.0, 0.0, T0], [1.0, 0.0, 0.0, 0.0, T0]
    rho, U, T = tube_fields(3, dims, 2, lo, hi)
    lat = lbm.Lattice("D3Q95", dims, 1.5, "fp32")
    lat.init(rho, U, T)
    lbm.lbm_set_fixed_ends(lat.ctx, 2, 5, lo, hi)
    lat.step(steps)
    r, _, Tn = lat.moments()
    r = r[:, 5, 5]
    th = Tn[:, 5, 5] / T0
    st = riemann.star_state(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, 5.0 / 3.0)
    ws = riemann.wave_speeds(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, 5.0 / 3.0)
    zc = np.arange(800) + 0.5 - 400

    def central(a, b):
        L = b - a
        return (zc > a + 0.3 * L) & (zc < b - 0.3 * L)

    mL = central(ws["left_tail"] * steps, ws["contact"] * steps)
    mR = central(ws["contact"] * steps, ws["right"] * steps)
    assert abs(r[mL].mean() / st.rho_L - 1) < 5e-3 and abs(r[mR].mean() / st.rho_R - 1) < 5e-3
    assert abs(th[mL].mean() / (st.p / st.rho_L / T0) - 1) < 5e-3
    assert abs(th[mR].mean() / (st.p / st.rho_R / T0) - 1) < 5e-3
    assert np.allclose(r[:5], 4.0, rtol=1e-6) and np.allclose(r[-5:], 1.0, rtol=1e-6)


def test_fixed_ends_argument_errors(lbm):
    lat = lbm.Lattice("D3Q95", (8, 8, 40), 1.5, "fp32")
    st = [1.0, 0.0, 0.0, 0.0, lat.info["T0"]]
    for axis, width in [(2, 4), (3, 5), (0, 5)]:       # below the reach, bad axis, > N/2
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_set_fixed_ends(lat.ctx, axis, width, st, st)
        assert ei.value.code == lbm.LBM_EINVAL
    lbm.lbm_set_fixed_ends(lat.ctx, 2, 5, st, st)
    lat.init(np.ones((40, 8, 8)), np.zeros((3, 40, 8, 8)), np.full((40, 8, 8), lat.info["T0"]))
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_record(lat.ctx, 4, 2)
    assert ei.value.code == lbm.LBM_EINVAL
    lbm.lbm_set_fixed_ends(lat.ctx, 2, 0)
    lbm.lbm_record(lat.ctx, 4, 2)
