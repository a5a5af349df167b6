"""lbm_audit_noalloc: the conservation audit without any device allocation.

It is for callers that cannot call cudaMalloc (their device memory belongs to
another allocator, or they cannot take the synchronisation an allocation may
cause).  The test calls it through the C ABI on a state held in a caller-owned
buffer, twice in a row on different states, and checks each result against the
allocating entry point lbm_audit of the same state (FP64 audit tolerance
1e-12 relative; both run the same reduction in the same order).  This file is
collected last so that a failure here stops a run only after every other test.
"""
import numpy as np
import pytest

from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _check_close(a, ref):
    got = {"mass": a[0], "momentum": a[1:4], "energy": a[4], "min_f_over_w": a[5],
           "nonfinite": a[6], "cells": a[7]}
    assert abs(got["mass"] - ref["mass"]) <= 1e-12 * abs(ref["mass"])
    assert abs(got["energy"] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert np.max(np.abs(got["momentum"] - ref["momentum"])) <= 1e-12 * abs(ref["mass"])
    assert abs(got["min_f_over_w"] - ref["min_f_over_w"]) <= 1e-12
    assert got["nonfinite"] == ref["nonfinite"] and got["cells"] == ref["cells"]


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
    for _ in range(2):
        lat.step(3)
        lbm.lbm_get_raw(lat.ctx, h)
        lbm.lbm_audit_noalloc(model, storage, dims, h, out)
        torch.cuda.synchronize()
        _check_close(out.cpu().numpy(), lat.audit())


def test_noalloc_audit_rejects_grids_beyond_its_scratch(lbm):
    torch = pytest.importorskip("torch")
    h = torch.empty(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_audit_noalloc("D3Q95", "fp32", (256, 128, 128), h, out)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "at most" in str(ei.value)
