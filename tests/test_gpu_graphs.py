"""lbm_step through CUDA-graph replays against direct launches: the same kernels
on the same buffers, so the states must agree bit for bit, including runs that
start from either ping-pong buffer, a change of omega (recapture), the fixed end
planes and the launch count the context reports."""
import numpy as np
import pytest

from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def pair(lbm, model, dims, storage, graph_steps):
    mdl = get_model(model)
    D = mdl.D
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=11)
    lats = []
    for gs in (0, graph_steps):
        lat = lbm.Lattice(model, dims, 1.7, storage)
        lbm.lbm_set_graph_steps(lat.ctx, gs)
        lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
        lats.append(lat)
    return lats


def same(a, b):
    return np.array_equal(a.raw().view(np.uint8), b.raw().view(np.uint8))


@pytest.mark.parametrize("model,dims,storage", [("D3Q95", (40, 6, 5), "fp32"),
                                                ("D3Q95", (40, 6, 5), "fp16"),
                                                ("D3Q95", (24, 5, 4), "fp64"),
                                                ("D2Q33", (64, 4, 1), "fp32")])
def test_graph_replays_match_direct_launches(lbm, model, dims, storage):
    direct, graph = pair(lbm, model, dims, storage, 4)
    for n in (1, 11, 9, 8, 3, 17):        # odd counts change the starting buffer
        direct.step(n)
        graph.step(n)
        assert same(direct, graph), n
    assert lbm.lbm_steps_done(direct.ctx) == lbm.lbm_steps_done(graph.ctx) == 49
    assert lbm.lbm_launch_count(direct.ctx) == lbm.lbm_launch_count(graph.ctx)
    direct.close()
    graph.close()


def test_graph_recaptured_after_omega_change(lbm):
    direct, graph = pair(lbm, "D3Q95", (40, 6, 5), "fp32", 6)
    for lat in (direct, graph):
        lat.step(13)
        lbm.lbm_set_omega(lat.ctx, 1.2)
        lat.step(25)
    assert same(direct, graph)
    direct.close()
    graph.close()


def test_graph_with_fixed_end_planes(lbm):
    direct, graph = pair(lbm, "D3Q95", (6, 5, 40), "fp32", 4)
    mdl = get_model("D3Q95")
    lo = [4.0, 0.0, 0.0, 0.0, 1.0 * mdl.T0]
    hi = [1.0, 0.0, 0.0, 0.0, 1.0 * mdl.T0]
    for lat in (direct, graph):
        lbm.lbm_set_fixed_ends(lat.ctx, 2, 5, lo, hi)
        lat.step(21)
    assert same(direct, graph)
    assert lbm.lbm_launch_count(direct.ctx) == lbm.lbm_launch_count(graph.ctx)
    direct.close()
    graph.close()


def test_graph_steps_argument_errors(lbm):
    lat = lbm.Lattice("D3Q95", (8, 8, 8), 1.0, "fp32")
    for bad in (3, -2, 5000):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_set_graph_steps(lat.ctx, bad)
        assert ei.value.code == lbm.LBM_EINVAL
    lbm.lbm_set_graph_steps(lat.ctx, 0)
    lbm.lbm_set_graph_steps(lat.ctx, 2)
    lat.close()
