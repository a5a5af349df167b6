"""lbm_audit_noalloc: the conservation audit without any device allocation.

It is for callers that cannot call cudaMalloc (their device memory belongs to
another allocator, or they cannot take the synchronisation an allocation may
cause).  The test calls it through the C ABI on a state held in a caller-owned
buffer, twice in a row on different states, and checks each result against the
allocating entry point lbm_audit of the same state: the two run the same kernels
(same source, same flags) with the same fixed reduction order, so the results
must agree bit for bit.  It also checks the property the entry point exists for:
once warmed up, a call leaves the device's free memory unchanged.  This file is
collected last so that a failure here stops a run only after every other test.
"""
import numpy as np
import pytest

from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _check_equal(a, ref):
    assert a[0] == ref["mass"] and a[4] == ref["energy"]
    assert np.array_equal(a[1:4], ref["momentum"])
    assert a[5] == ref["min_f_over_w"]
    assert a[6] == ref["nonfinite"] and a[7] == ref["cells"]


@pytest.mark.parametrize("model,dims,storage", [("D3Q95", (40, 12, 9), "fp32"),
                                                ("D2Q33", (96, 20, 1), "fp64"),
                                                ("D3Q95", (32, 16, 8), "fp16")])
def test_noalloc_audit_matches_lbm_audit_twice(lbm, model, dims, storage):
    torch = pytest.importorskip("torch")
    D = 3 if model == "D3Q95" else 2
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=11)
    lat = lbm.Lattice(model, dims, 1.6, storage)
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    Q = lat.info["Q"]
    esize = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[storage]
    h = torch.empty(Q * lat.cells * esize, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    lbm.lbm_audit_noalloc(model, storage, dims, h, out)   # warm-up: set-up, module load
    torch.cuda.synchronize()
    for _ in range(2):
        lat.step(3)
        lbm.lbm_get_raw(lat.ctx, h)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        lbm.lbm_audit_noalloc(model, storage, dims, h, out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        _check_equal(out.cpu().numpy(), lat.audit())


def test_noalloc_audit_rejects_grids_beyond_its_scratch(lbm):
    torch = pytest.importorskip("torch")
    h = torch.empty(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_audit_noalloc("D3Q95", "fp32", (256, 128, 128), h, out)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "at most" in str(ei.value)


def test_noalloc_audit_rejects_host_and_undersized_buffers(lbm):
    """Host memory and a buffer smaller than the grid's populations are refused on
    the host (LBM_EINVAL), before anything is launched."""
    torch = pytest.importorskip("torch")
    dims = (32, 16, 8)
    need = 95 * 32 * 16 * 8 * 4
    h = torch.zeros(need, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    cases = [(torch.zeros(need, dtype=torch.uint8), out),            # h on the host
             (h[: need - 4], out),                                   # h too small
             (h, torch.zeros(8, dtype=torch.float64))]               # out on the host
    for hh, oo in cases:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_audit_noalloc("D3Q95", "fp32", dims, hh, oo)
        assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(ValueError):
        lbm.lbm_audit_noalloc("D3Q95", "fp32", dims, h, out[:4])
