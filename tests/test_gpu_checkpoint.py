"""Checkpoint / resume (lbm_save, lbm_load) and failure detection in the time loop
(lbm_set_audit_every).  The failure is made on the host: a NaN planted in the
stored state through lbm_set_raw; nothing faults or waits on the device."""
import os

import numpy as np
import pytest

from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS = (40, 6, 5)


def lattice(lbm, storage, dims=DIMS, omega=1.7):
    fields = W.riemann_planar(3, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=4)
    lat = lbm.Lattice("D3Q95", dims, omega, storage)
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    return lat


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_save_load_resumes_bit_for_bit(lbm, storage, tmp_path):
    path = str(tmp_path / "state.lbm")
    a = lattice(lbm, storage)
    a.step(13)
    lbm.lbm_save(a.ctx, path)
    b = lbm.Lattice("D3Q95", DIMS, 1.0, storage)      # omega and steps come from the file
    lbm.lbm_load(b.ctx, path)
    assert lbm.lbm_steps_done(b.ctx) == 13
    a.step(9)
    b.step(9)
    assert np.array_equal(a.raw().view(np.uint8), b.raw().view(np.uint8))
    # the file is the header plus exactly the stored deviations
    h = a.raw()
    assert os.path.getsize(path) == 72 + h.nbytes
    a.close()
    b.close()


def test_load_rejects_mismatched_or_damaged_files(lbm, tmp_path):
    path = str(tmp_path / "state.lbm")
    a = lattice(lbm, "fp32")
    a.step(3)
    lbm.lbm_save(a.ctx, path)
    for ctx_args in (("D3Q95", (40, 6, 6), 1.7, "fp32"), ("D3Q95", DIMS, 1.7, "fp16")):
        other = lbm.Lattice(*ctx_args)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_load(other.ctx, path)
        assert ei.value.code == lbm.LBM_EINVAL
        other.close()
    raw = open(path, "rb").read()
    bad = str(tmp_path / "bad.lbm")
    open(bad, "wb").write(b"NOTSTATE" + raw[8:])
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_load(a.ctx, bad)
    assert ei.value.code == lbm.LBM_EINVAL
    # truncated (or over-long) files are refused and the live state stays as it was,
    # bit for bit, with its step count: a later step continues the original run
    before = a.raw()
    ref = lattice(lbm, "fp32")
    ref.step(3)
    for name, data in (("short.lbm", raw[:len(raw) // 2]), ("shorter.lbm", raw[:72 + 16]),
                       ("long.lbm", raw + b"\0" * 64)):
        p = str(tmp_path / name)
        open(p, "wb").write(data)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_load(a.ctx, p)
        assert ei.value.code == lbm.LBM_EIO
        assert lbm.lbm_steps_done(a.ctx) == 3
        assert np.array_equal(before.view(np.uint8), a.raw().view(np.uint8))
    a.step(4)
    ref.step(4)
    assert np.array_equal(ref.raw().view(np.uint8), a.raw().view(np.uint8))
    ref.close()
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_load(a.ctx, str(tmp_path / "missing.lbm"))
    assert ei.value.code == lbm.LBM_EIO
    fresh = lbm.Lattice("D3Q95", DIMS, 1.7, "fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_save(fresh.ctx, str(tmp_path / "never.lbm"))
    assert ei.value.code == lbm.LBM_ESTATE
    fresh.close()
    a.close()


def test_audit_every_stops_the_loop_on_non_finite_populations(lbm):
    a = lattice(lbm, "fp32")
    lbm.lbm_set_audit_every(a.ctx, 5)
    a.step(12)                                   # a finite run passes every audit
    assert lbm.lbm_steps_done(a.ctx) == 12
    h = a.raw()
    h[7, 2, 3, 20] = np.nan
    a.set_raw(h)                                 # resets the step count to 0
    with pytest.raises(lbm.LbmError) as ei:
        a.step(12)
    assert ei.value.code == lbm.LBM_EUNSTABLE
    assert lbm.lbm_steps_done(a.ctx) == 5          # stopped at the first audit
    assert a.audit()["nonfinite"] > 0
    lbm.lbm_set_audit_every(a.ctx, 0)
    a.step(2)                                    # no audit: the loop runs on
    assert lbm.lbm_steps_done(a.ctx) == 7
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_audit_every(a.ctx, -1)
    a.close()
