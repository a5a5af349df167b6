"""Moments and conservation audit of every storage form against the FP64 oracle.

Both sides see the same stored state: the populations the library holds are read
back as FP64 (f_i = w_i (1 + h_i), exact for every storage type) and handed to
the oracle's macroscopic fields and audit (Formula 1, n <= 2).

Bounds.  The FP64 form sums in FP64 (1e-13).  The FP32, FP16 and BF16 forms take
the collision's own sums: each +/- pair and each weight product is rounded to
FP32 (relative 2^-24 of the deviation terms, and the FP32-rounded weights shift
every product by up to 2^-24), the rho and E sums are compensated, and the
fields are formed in FP32; 2e-6 relative on rho and T and 2e-6 sqrt(T0) on U
covers that with a margin of about ten.  The audit totals carry the same
per-cell bound (2e-7 relative on mass and energy; momentum 2e-7 of the mass).
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = {"fp64": 1e-13, "fp32": 2e-6, "fp16": 2e-6, "bf16": 2e-6}
AUDIT_TOL = {"fp64": 1e-13, "fp32": 2e-7, "fp16": 2e-7, "bf16": 2e-7}

# The larger cases span more than a wave of 256-cell blocks (152 SMs x 4 resident)
# and end in a partial block.
CASES = [("D3Q95", (165, 6, 5), 82), ("D2Q33", (300, 7, 1), 150),
         ("D3Q95", (97, 63, 47), 48), ("D2Q33", (641, 299, 1), 320)]


def oracle_order(mdl, lat, f):
    pos = {tuple(v): j for j, v in enumerate(lat.info["e"].tolist())}
    return f[[pos[tuple(v)] for v in mdl.e.tolist()]]


def stepped_lattice(lbm, model, dims, cut, storage, steps=15):
    D = 2 if model == "D2Q33" else 3
    fields = W.riemann_planar(D, *dims, cut, (1.0, 1.0), (0.55, 0.7), seed=21)
    mdl = get_model(model)
    lat = lbm.Lattice(model, dims, 1.6, storage)
    lat.init(fields.rho, fields.U, fields.theta * mdl.T0)
    lat.step(steps)
    return mdl, lat


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model,dims,cut", CASES)
def test_moments_match_oracle(lbm, model, dims, cut, storage):
    mdl, lat = stepped_lattice(lbm, model, dims, cut, storage)
    f = oracle_order(mdl, lat, lat.populations())
    rho, U, T = lat.moments()
    r0, U0, T0 = olbm.macroscopic(mdl, f)
    tol = FIELD_TOL[storage]
    assert np.max(np.abs(rho - r0) / r0) <= tol
    assert np.max(np.abs(T - T0) / T0) <= tol
    assert np.max(np.abs(U - U0)) / np.sqrt(mdl.T0) <= tol
    lat.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model,dims,cut", CASES)
def test_audit_matches_oracle(lbm, model, dims, cut, storage):
    mdl, lat = stepped_lattice(lbm, model, dims, cut, storage)
    f = oracle_order(mdl, lat, lat.populations())
    a = lat.audit()
    o = olbm.audit(mdl, f)
    tol = AUDIT_TOL[storage]
    assert a["nonfinite"] == 0 and a["cells"] == int(np.prod(dims))
    assert abs(a["mass"] - o["mass"]) <= tol * o["mass"]
    assert abs(a["energy"] - o["energy"]) <= tol * o["energy"]
    mom = np.zeros(3)
    mom[:mdl.D] = o["momentum"]
    assert np.max(np.abs(a["momentum"] - mom)) <= tol * o["mass"]
    # the two sides solve the weights independently (agreeing to ~1e-14 relative)
    assert abs(a["min_f_over_w"] - o["min_f_over_w"]) <= 1e-12 * max(1.0, abs(o["min_f_over_w"]))
    # deterministic: a second audit of the same state is bitwise the same
    b = lat.audit()
    assert (a["mass"], a["energy"]) == (b["mass"], b["energy"])
    assert np.array_equal(a["momentum"], b["momentum"])
    lat.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_audit_counts_planted_nonfinite(lbm, storage):
    """NaN and Inf deviations planted through set_raw (two of them in one cell) are
    counted one by one, the audit reports LBM_EUNSTABLE, and the minimum of f / w
    is the planted -Inf (NaN never wins a minimum)."""
    dims = (40, 6, 5)
    mdl, lat = stepped_lattice(lbm, "D3Q95", dims, 20, storage, steps=3)
    h = lat.raw()
    if storage == "bf16":
        nan, inf, ninf = np.uint16(0x7FC0), np.uint16(0x7F80), np.uint16(0xFF80)
    else:
        nan, inf, ninf = h.dtype.type(np.nan), h.dtype.type(np.inf), h.dtype.type(-np.inf)
    spots = [(3, 0, 1, 7), (40, 2, 5, 39), (94, 4, 0, 0), (0, 1, 1, 1), (7, 1, 1, 1)]
    for k, s in enumerate(spots):
        h[s] = (nan, inf, ninf, nan, inf)[k]
    lat.set_raw(h)
    a = lat.audit()
    assert a["nonfinite"] == len(spots)
    assert a["status"] == lbm.LBM_EUNSTABLE
    assert a["cells"] == int(np.prod(dims))
    assert a["min_f_over_w"] == -np.inf
    lat.close()
