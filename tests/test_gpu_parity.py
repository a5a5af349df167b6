"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the parity targets): FP64 form 1e-12 relative, FP32 form 1e-5 relative,
streaming indices bit-exact.  rho and T are compared relative per cell, U
relative to the sound-speed scale sqrt(T0).  Populations are compared per
direction, normalised by that direction's largest magnitude; their bound is
the field tolerance times the largest sensitivity |d h_i / d theta| of the model's
outer shell (h_i = f_i / w_i - 1): the (4,4) shell of D2Q33 has |xi|^2 = 43 and
|dh/dtheta| up to about 100, the outermost D3Q95 shells about 15, so a
temperature difference at the tolerance moves those populations by that factor.
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
SENS = {"D2Q33": 100.0, "D3Q95": 20.0}


def run_both(lbm, model, storage, fields, omega, steps, dims, variant=0):
    mdl = get_model(model)
    T = fields.theta * mdl.T0
    S = olbm.init_populations(mdl, fields.rho, fields.U, T)
    S = olbm.run(mdl, S, omega, steps)
    lat = lbm.Lattice(model, dims, omega, storage)
    if variant:
        lbm.lbm_set_variant(lat.ctx, variant)
    info = lat.info
    lat.init(fields.rho, fields.U, fields.theta * info["T0"])
    lat.step(steps)
    return mdl, S, lat


def to_oracle_order(mdl, lat, f):
    """Reorder GPU populations [Q, ...] (library direction order) to the oracle's order."""
    pos = {tuple(v): j for j, v in enumerate(lat.info["e"].tolist())}
    perm = [pos[tuple(v)] for v in mdl.e.tolist()]
    return f[perm]


def compare(mdl, S, lat, tol):
    f = to_oracle_order(mdl, lat, lat.populations())
    Q = mdl.Q
    df = np.abs(f - S).reshape(Q, -1).max(axis=1) / np.abs(S).reshape(Q, -1).max(axis=1)
    rho, U, T = lat.moments()
    r0, U0, T0 = olbm.macroscopic(mdl, S)
    err = {
        "rho": float(np.max(np.abs(rho - r0) / r0)),
        "T": float(np.max(np.abs(T - T0) / T0)),
        "U": float(np.max(np.abs(U - U0)) / np.sqrt(mdl.T0)),
    }
    assert max(err.values()) <= tol, err
    assert float(df.max()) <= tol * SENS[mdl.name], (float(df.max()), err)
    err["f_per_direction"] = float(df.max())
    return err


def test_d2q33_fp64_riemann_256x8_200_steps(lbm):
    """The D2Q33 FP64 workload in full: 256 x 8, 200 steps, omega 1.5."""
    wl, fields = W.d2q33_riemann()
    mdl, S, lat = run_both(lbm, "D2Q33", "fp64", fields, wl.omega, wl.steps, wl.dims)
    compare(mdl, S, lat, TOL["fp64"])


@pytest.mark.parametrize("storage,tol", [("fp32", TOL["fp32"]), ("fp16", 1e-3), ("bf16", 1e-2)])
def test_d2q33_reduced_precision_forms(lbm, storage, tol):
    """The D2Q33 workload's states on 256 x 8, 100 steps, in the FP32 form (1e-5)
    and the FP16 / BF16 deviation forms (1e-3 / 1e-2, their storage rounding).
    D2Q33's weights span five decades (3.5e-6 to 0.16); the deviation storage
    h = f/w - 1 keeps every direction in the same range."""
    fields = W.riemann_planar(2, 256, 8, 1, 128, (1.0, 1.0), (0.5, 0.8), seed=2)
    mdl, S, lat = run_both(lbm, "D2Q33", storage, fields, 1.5, 100, (256, 8, 1))
    rho, U, T = lat.moments()
    r0, U0, T0 = olbm.macroscopic(mdl, S)
    err = max(np.max(np.abs(rho - r0) / r0), np.max(np.abs(T - T0) / T0),
              np.max(np.abs(U - U0)) / np.sqrt(mdl.T0))
    assert err <= tol, err
    a = lat.audit()
    assert a["nonfinite"] == 0


@pytest.mark.parametrize("variant", [1, 3])
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_d3q95_riemann_ragged_grid(lbm, storage, variant):
    """165 x 6 x 5: two x tiles of 128 threads plus a ragged tail, y/z smaller than the reach."""
    dims = (165, 6, 5)
    fields = W.riemann_planar(3, *dims, 82, (1.0, 1.0), (0.6, 0.75), seed=3)
    steps = 12 if storage == "fp64" else 40
    if storage == "fp64" and variant == 3:
        pytest.skip("the split kernel serves the FP32-arithmetic forms")
    mdl, S, lat = run_both(lbm, "D3Q95", storage, fields, 1.6, steps, dims, variant)
    compare(mdl, S, lat, TOL[storage])


@pytest.mark.parametrize("model,dims", [("D3Q95", (3, 2, 4)), ("D3Q95", (1, 1, 1)),
                                        ("D2Q33", (3, 2, 1)), ("D2Q33", (33, 1, 1))])
def test_grids_smaller_than_the_reach(lbm, model, dims):
    rng = np.random.default_rng(4)
    mdl = get_model(model)
    shape = dims[::-1]
    rho = 1.0 + 0.05 * rng.standard_normal(shape)
    U = 0.05 * rng.standard_normal((mdl.D,) + shape)
    theta = 1.0 + 0.05 * rng.standard_normal(shape)
    fields = W.Fields(rho, U, theta)
    mdl, S, lat = run_both(lbm, model, "fp64", fields, 1.3, 7, dims)
    compare(mdl, S, lat, TOL["fp64"])


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model", ["D2Q33", "D3Q95"])
def test_init_is_the_discrete_equilibrium(lbm, model, storage):
    mdl = get_model(model)
    dims = (40, 3, 2) if model == "D3Q95" else (40, 3, 1)
    rng = np.random.default_rng(5)
    shape = dims[::-1]
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, shape)
    U = 0.1 * rng.uniform(-1, 1, (mdl.D,) + shape)
    theta = 1.0 + 0.2 * rng.uniform(-1, 1, shape)
    lat = lbm.Lattice(model, dims, 1.0, storage)
    lat.init(rho, U, theta * lat.info["T0"])
    S = olbm.init_populations(mdl, rho, U, theta * mdl.T0)
    wv = mdl.w.reshape((-1, 1, 1, 1))
    h_ref = S / wv - 1.0
    dh = np.abs(to_oracle_order(mdl, lat, lat.populations()) - S) / wv
    # one round-to-nearest of h = f/w - 1 in the storage type: half an ulp relative,
    # or half the subnormal spacing (FP16 below 2^-14); plus the FP64 evaluation of
    # the degree-4 polynomial, whose terms reach ~500 on the outer D2Q33 shell
    u = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage]
    sub = {"fp64": 0.0, "fp32": 2.0 ** -150, "fp16": 2.0 ** -25, "bf16": 2.0 ** -134}[storage]
    assert np.all(dh <= u * np.abs(h_ref) * (1 + 1e-6) + sub + 1e-12)


def label_array(Q, shape, storage):
    """Integer labels exactly representable in the storage type."""
    n = int(np.prod(shape))
    cell = np.arange(n).reshape(shape)
    mod = {"fp64": 1 << 40, "fp32": 1 << 23, "fp16": 2039, "bf16": 251}[storage]
    lab = np.stack([(cell * 3 + 7 * i) % mod + 1 for i in range(Q)]).astype(np.float64)
    return lab


def as_storage(a, storage):
    if storage == "fp64":
        return a.astype(np.float64)
    if storage == "fp32":
        return a.astype(np.float32)
    if storage == "fp16":
        return a.astype(np.float16)
    # bf16: the top 16 bits of the FP32 pattern (exact for these small integers)
    return (a.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model,dims", [("D3Q95", (37, 6, 7)), ("D3Q95", (2, 3, 4)),
                                        ("D3Q95", (40, 6, 7)), ("D3Q95", (8, 3, 2)),
                                        ("D3Q95", (133, 4, 3)),
                                        ("D2Q33", (131, 5, 1)), ("D2Q33", (3, 2, 1)),
                                        ("D2Q33", (136, 5, 1)), ("D2Q33", (8, 2, 1))])
def test_streaming_is_a_bit_exact_permutation(lbm, model, dims, storage):
    """omega = 0: after n steps h_i(x) = h_i((x - n e_i) mod N) bit for bit, on grids
    smaller than the reach, ragged in x, and spanning several 128-cell blocks."""
    lat = lbm.Lattice(model, dims, 0.0, storage)
    Q = lat.info["Q"]
    e = lat.info["e"]
    shape = dims[::-1]
    lab = as_storage(label_array(Q, shape, storage), storage)
    lat.set_raw(lab)
    n = 3
    lat.step(n)
    got = lat.raw()
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for i in range(Q):
        ex, ey = int(e[i, 0]), int(e[i, 1])
        ez = int(e[i, 2]) if e.shape[1] == 3 else 0
        src = (((z - n * ez) % nz) * ny + (y - n * ey) % ny) * nx + (x - n * ex) % nx
        expect = lab[i].reshape(-1)[src]
        assert np.array_equal(got[i].view(np.uint8), expect.view(np.uint8)), i


def test_d3q95_fp32_full_size_128x64x64(lbm):
    """The D3Q95 FP32 workload at full size (128 x 64 x 64, omega 1.6) in the launch
    configuration the benchmark times: every population after 2 steps against the
    oracle, plus the FP64 conservation audit after 200 steps."""
    wl, fields = W.d3q95_riemann()
    mdl, S, lat = run_both(lbm, "D3Q95", "fp32", fields, wl.omega, 2, wl.dims)
    compare(mdl, S, lat, TOL["fp32"])
    a0 = olbm.audit(mdl, olbm.init_populations(mdl, fields.rho, fields.U, fields.theta * mdl.T0))
    lat.step(198)
    a1 = lat.audit()
    assert a1["nonfinite"] == 0 and a1["cells"] == wl.cells
    assert abs(a1["mass"] / a0["mass"] - 1) < 1e-5
    assert abs(a1["energy"] / a0["energy"] - 1) < 1e-5
    assert np.max(np.abs(a1["momentum"])) / a0["mass"] < 1e-6


def test_audit_matches_oracle(lbm):
    dims = (24, 5, 4)
    fields = W.riemann_planar(3, *dims, 12, (1.0, 1.0), (0.6, 0.75), seed=8)
    mdl, S, lat = run_both(lbm, "D3Q95", "fp64", fields, 1.6, 5, dims)
    a = lat.audit()
    o = olbm.audit(mdl, S)
    assert abs(a["mass"] - o["mass"]) < 1e-12 * o["mass"]
    assert abs(a["energy"] - o["energy"]) < 1e-12 * o["energy"]
    assert np.max(np.abs(a["momentum"] - o["momentum"])) < 1e-12 * o["mass"]
    assert abs(a["min_f_over_w"] - o["min_f_over_w"]) < 1e-12
    assert a["nonfinite"] == 0


def test_errors_are_reported_before_launch(lbm):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice("D3Q95", (8, 8, 8), 2.5, "fp32")
    assert ei.value.code == lbm.LBM_EINVAL
    lat = lbm.Lattice("D3Q95", (8, 8, 8), 1.0, "fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lat.step(1)
    assert ei.value.code == lbm.LBM_ESTATE
    with pytest.raises(lbm.LbmError) as ei:
        lat.set_raw(np.zeros(10, dtype=np.float32))
    assert ei.value.code == lbm.LBM_EINVAL
    rho = np.ones((8, 8, 8))
    with pytest.raises(lbm.LbmError) as ei:
        lat.init(-rho, np.zeros((3, 8, 8, 8)), rho)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_backward(lat.ctx, rho)
    assert ei.value.code == lbm.LBM_ESTATE
    n0 = lbm.lbm_launch_count(lat.ctx)
    lat.init(rho, np.zeros((3, 8, 8, 8)), rho * lat.info["T0"])
    lat.step(4)
    # the check of the host fields, the equilibrium, four steps
    assert lbm.lbm_launch_count(lat.ctx) == n0 + 6
    # each field's first bad value is named; U must be finite
    for bad, name in ((dict(rho=np.nan), "rho[5]"), (dict(T=0.0), "T[5]"), (dict(U=np.inf), "U")):
        r, U, T = rho.copy(), np.zeros((3, 8, 8, 8)), rho * lat.info["T0"]
        arr = {"rho": r, "U": U[1], "T": T}[list(bad)[0]]
        arr.reshape(-1)[5] = list(bad.values())[0]
        with pytest.raises(lbm.LbmError) as ei:
            lat.init(r, U, T)
        assert ei.value.code == lbm.LBM_EINVAL and name in str(ei.value)


def test_chunked_host_init(lbm):
    """Host fields on a grid of at least 2^20 cells are uploaded, checked and turned
    into their equilibrium in 8 chunks: the state equals the one made from the same
    fields on the device (bitwise), and a bad value in the last chunk is refused
    with the previous state left live."""
    import torch
    dims = (128, 96, 96)   # 1,179,648 cells
    shape = dims[::-1]
    rng = np.random.default_rng(9)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, shape)
    U = 0.05 * rng.uniform(-1, 1, (3,) + shape)
    lat = lbm.Lattice("D3Q95", dims, 1.6, "fp32")
    T = (1.0 + 0.05 * rng.uniform(-1, 1, shape)) * lat.info["T0"]
    dev = lbm.Lattice("D3Q95", dims, 1.6, "fp32")
    try:
        lat.init(rho, U, T)
        dev.init(torch.from_numpy(rho).cuda(), torch.from_numpy(U).cuda(), torch.from_numpy(T).cuda())
        assert np.array_equal(lat.raw().view(np.uint32), dev.raw().view(np.uint32))
        lat.step(3)
        before = lat.raw()
        bad = T.copy()
        bad.reshape(-1)[-7] = -1.0
        with pytest.raises(lbm.LbmError) as ei:
            lat.init(rho, U, bad)
        assert ei.value.code == lbm.LBM_EINVAL and "T[%d]" % (rho.size - 7) in str(ei.value)
        assert np.array_equal(lat.raw().view(np.uint32), before.view(np.uint32))
        assert lbm.lbm_steps_done(lat.ctx) == 3
        lat.step(1)
    finally:
        lat.close()
        dev.close()


def test_grid_and_argument_limits(lbm):
    """Empty, oversized and malformed grids and arguments are refused on the host
    (nothing is allocated or launched); zero steps is a no-op."""
    for model, dims in (("D3Q95", (0, 8, 8)), ("D3Q95", (8, -1, 8)), ("D3Q95", (8, 8, 70000)),
                        ("D3Q95", (65536, 65535, 2)),           # 2^33 cells: past the 2^31 limit
                        ("D2Q33", (8, 8, 2)), (7, (8, 8, 8))):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Lattice(model, dims, 1.0, "fp32")
        assert ei.value.code == lbm.LBM_EINVAL, (model, dims)
    for omega in (-0.1, 2.0, float("nan")):
        with pytest.raises(lbm.LbmError):
            lbm.Lattice("D3Q95", (8, 8, 8), omega, "fp32")
    lat = lbm.Lattice("D3Q95", (8, 8, 8), 1.0, "fp32")
    rho = np.ones((8, 8, 8))
    lat.init(rho, np.zeros((3, 8, 8, 8)), rho * lat.info["T0"])
    before = lat.raw()
    lat.step(0)
    assert lbm.lbm_steps_done(lat.ctx) == 0
    assert np.array_equal(before.view(np.uint8), lat.raw().view(np.uint8))
    with pytest.raises(lbm.LbmError):
        lat.step(-1)
    nan_rho = rho.copy()
    nan_rho[1, 2, 3] = np.nan
    with pytest.raises(lbm.LbmError) as ei:
        lat.init(nan_rho, np.zeros((3, 8, 8, 8)), rho)
    assert ei.value.code == lbm.LBM_EINVAL
    lat.close()


@pytest.mark.parametrize("omega", [1.0, 1.95])
def test_d3q95_fp64_full_relaxation_and_near_two(lbm, omega):
    """omega = 1 (every step lands on the equilibrium of the gathered moments) and
    omega close to the stability limit 2, against the oracle at the FP64 bar."""
    dims = (24, 6, 5)
    fields = W.riemann_planar(3, *dims, 12, (1.0, 1.0), (0.7, 0.85), seed=12)
    mdl, S, lat = run_both(lbm, "D3Q95", "fp64", fields, omega, 10, dims)
    compare(mdl, S, lat, TOL["fp64"])


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_tma_kernel_matches_oracle_with_ragged_chunk(lbm, storage):
    """136 x 6 x 5 with the TMA kernel: one full 128-cell chunk and a ragged 8-cell
    chunk per row, row segments wrapping at both row ends, y / z smaller than the reach."""
    dims = (136, 6, 5)
    fields = W.riemann_planar(3, *dims, 68, (1.0, 1.0), (0.6, 0.75), seed=6)
    steps = 12 if storage == "fp64" else 40
    mdl, S, lat = run_both(lbm, "D3Q95", storage, fields, 1.6, steps, dims, lbm.VARIANT_TMA)
    compare(mdl, S, lat, TOL[storage])


# Grids for the bitwise comparison of the kernel variants: ragged chunks, grids below
# the reach, and grids with many chunks per persistent TMA CTA (several trips round
# the stage ring, the output tile reused chunk after chunk).
VARIANT_GRIDS = [("D3Q95", (136, 6, 5)), ("D3Q95", (8, 3, 4)), ("D3Q95", (256, 64, 32)),
                 ("D2Q33", (264, 5, 1)), ("D2Q33", (16, 2, 1)), ("D2Q33", (2048, 400, 1))]


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("model,dims", VARIANT_GRIDS)
def test_kernel_variants_agree_bitwise(lbm, model, dims, storage):
    """Direct, TMA, split (FP32-arithmetic forms) and pair (FP16 / BF16, two cells
    per thread on paired FP32 instructions) kernels compute the same arithmetic in
    the same order: their states agree bit for bit."""
    mdl = get_model(model)
    rng = np.random.default_rng(7)
    shape = dims[::-1]
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, shape)
    U = 0.05 * rng.uniform(-1, 1, (mdl.D,) + shape)
    theta = 1.0 + 0.1 * rng.uniform(-1, 1, shape)
    out = []
    variants = [lbm.VARIANT_DIRECT, lbm.VARIANT_TMA]
    if storage != "fp64":
        variants.append(lbm.VARIANT_SPLIT)
    if storage in ("fp16", "bf16"):
        variants.append(lbm.VARIANT_PAIR)
    for variant in variants:
        lat = lbm.Lattice(model, dims, 1.7, storage)
        lbm.lbm_set_variant(lat.ctx, variant)
        lat.init(rho, U, theta * lat.info["T0"])
        lat.step(9)
        lbm.lbm_synchronize(lat.ctx)
        out.append(lat.raw())
        lat.close()
    for o in out[1:]:
        assert np.array_equal(out[0].view(np.uint8), o.view(np.uint8))


def test_tma_variant_needs_nx_multiple_of_8(lbm):
    lat = lbm.Lattice("D3Q95", (12, 4, 4), 1.0, "fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_set_variant(lat.ctx, lbm.VARIANT_TMA)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_test_stall(lat.ctx, 0, 10 ** 6)         # the hook needs the TMA variant
    assert ei.value.code == lbm.LBM_ESTATE
    lat.close()


@pytest.mark.parametrize("model,dims,storage", [("D3Q95", (256, 64, 32), "fp16"),
                                                ("D3Q95", (256, 64, 32), "fp32"),
                                                ("D2Q33", (2048, 64, 1), "fp16")])
def test_tma_bounded_wait_runs_out_and_reports(lbm, model, dims, storage):
    """Failure detection of the TMA kernel without a fault: the test hook makes the
    producer skip one chunk's copies, so that chunk's consumers wait for data that
    never comes; their wait gives up after 20 ms, the CTA stops (after waiting for
    its other copies in flight), and lbm_synchronize reports LBM_EDEVICE once.  The
    context stays usable: a fresh run on it matches the direct kernel bit for bit.
    D2Q33 FP16 covers the path with the shared-memory output tile and bulk stores,
    the D3Q95 forms the path that stores from the threads."""
    D = 3 if model == "D3Q95" else 2
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=9)
    lat = lbm.Lattice(model, dims, 1.6, storage)
    lbm.lbm_set_graph_steps(lat.ctx, 0)
    lbm.lbm_set_variant(lat.ctx, lbm.VARIANT_TMA)
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    lbm.lbm_test_stall(lat.ctx, 777, 20 * 10 ** 6)
    lat.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_synchronize(lat.ctx)
    assert ei.value.code == lbm.LBM_EDEVICE
    lbm.lbm_synchronize(lat.ctx)                       # reported once, then cleared
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    lat.step(5)
    lbm.lbm_synchronize(lat.ctx)
    got = lat.raw()
    lat.close()
    ref = lbm.Lattice(model, dims, 1.6, storage)
    lbm.lbm_set_variant(ref.ctx, lbm.VARIANT_DIRECT)
    ref.init(fields.rho, fields.U, fields.theta * ref.info["T0"])
    ref.step(5)
    assert np.array_equal(got.view(np.uint8), ref.raw().view(np.uint8))
    ref.close()


def test_pair_variant_needs_16_bit_storage_and_even_nx(lbm):
    for storage, dims in (("fp32", (16, 4, 4)), ("fp64", (16, 4, 4)), ("fp16", (15, 4, 4))):
        lat = lbm.Lattice("D3Q95", dims, 1.0, storage)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_set_variant(lat.ctx, lbm.VARIANT_PAIR)
        assert ei.value.code == lbm.LBM_EINVAL
        lat.close()
