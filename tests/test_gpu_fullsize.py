"""The full-size workloads in the benchmark's launch configuration, checked where the
oracle can follow them.

* 512 x 256 x 256 precision sweep (FP32, FP16, BF16), the same setup on 768 x 256 x
  256 in FP32 (too large for 32-bit element indices) and the 768 x 384 x 384 FP16
  oblique Riemann problem (default kernel and the two-cell kernel): after the state has developed under CUDA-graph replays,
  one more step is checked cell by cell on a seeded sample (random cells, the
  corners of the box and the planes next to the diaphragm and the periodic seam):
  the oracle collides the populations the GPU gathered (its stored state, decoded
  with the oracle's weights) and the GPU's stored result must match.  Bounds: FP32
  2e-5 (FP32 arithmetic of one step, ~1e-7 relative, times the outer shells'
  sensitivity to theta, with a margin of ten); FP16 / BF16 one storage rounding of
  the result, 2^-11 / 2^-8 relative, plus that.
* 128^3 adjoint workload (500 steps, checkpoint every 22): the loss mean(rho_N) is
  conserved, so its exact gradient is dL/drho_0 = 1/N, dL/dU_0 = dL/dT_0 = 0 and
  dL/domega = 0 at any size; the FP32 adjoint must reproduce that after the full
  reverse sweep.
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TORCH_DTYPE = {"fp32": "float32", "fp16": "float16", "bf16": "bfloat16"}
TOL = {"fp32": 2e-5, "fp16": 1e-3, "bf16": 8e-3}


def sample_cells(dims, n, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    xs = list(rng.integers(0, nx, n))
    ys = list(rng.integers(0, ny, n))
    zs = list(rng.integers(0, nz, n))
    for x in (0, 1, nx // 2 - 2, nx // 2 - 1, nx // 2, nx // 2 + 1, nx - 2, nx - 1):
        for y in (0, ny - 1):
            for z in (0, nz - 1):
                xs.append(x)
                ys.append(y)
                zs.append(z)
    return np.array(xs), np.array(ys), np.array(zs)


def check_sampled_step(lbm, wl, fields, storage, warm, nsample=4000, seed=3, variant=None):
    import torch
    mdl = get_model("D3Q95")
    Q = mdl.Q
    nx, ny, nz = wl.dims
    lat = lbm.Lattice("D3Q95", wl.dims, wl.omega, storage)
    lbm.lbm_set_graph_steps(lat.ctx, 32)
    if variant is not None:
        lbm.lbm_set_variant(lat.ctx, variant)
    lat.init(fields.rho, fields.U, fields.theta * lat.info["T0"])
    lat.step(warm)
    dt = getattr(torch, TORCH_DTYPE[storage])
    before = torch.empty((Q, nz, ny, nx), dtype=dt, device="cuda")
    lbm.lbm_get_raw(lat.ctx, before)
    lat.step(1)
    after = torch.empty_like(before)
    lbm.lbm_get_raw(lat.ctx, after)
    lbm.lbm_synchronize(lat.ctx)
    lat_e = lat.info["e"]
    lat.close()
    xs, ys, zs = sample_cells(wl.dims, nsample, seed)
    e = lat_e.astype(np.int64)
    idx = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (
        np.broadcast_to(np.arange(Q)[:, None], (Q, len(xs))),
        (zs[None, :] - e[:, 2:3]) % nz, (ys[None, :] - e[:, 1:2]) % ny, (xs[None, :] - e[:, 0:1]) % nx)]
    g_lib = before[idx[0], idx[1], idx[2], idx[3]].double().cpu().numpy()        # [Q, S]
    h_lib = after[:, torch.from_numpy(zs).cuda(), torch.from_numpy(ys).cuda(),
                  torch.from_numpy(xs).cuda()].double().cpu().numpy()
    del before, after
    torch.cuda.empty_cache()
    pos = {tuple(v): j for j, v in enumerate(lat_e.tolist())}
    perm = [pos[tuple(v)] for v in mdl.e.tolist()]                              # oracle order
    w = mdl.w[:, None]
    f_new = olbm.collide(mdl, w * (1.0 + g_lib[perm]), wl.omega)
    ref = f_new / w - 1.0
    err = np.abs(h_lib[perm] - ref) / (1.0 + np.abs(ref))
    return float(err.max())


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_precision_sweep_512x256x256_sampled_step(lbm, storage):
    wl, fields = W.d3q95_sweep(storage=storage)
    err = check_sampled_step(lbm, wl, fields, storage, warm=64)
    assert err <= TOL[storage], err


def test_fp32_wide_index_768x256x256_sampled_step(lbm):
    """Q ncell = 4.78e9 exceeds 32 bits: the FP32 direct kernel forms its element
    indices in 64 bits here (every smaller FP32 D3Q95 grid takes the 32-bit form)."""
    wl, fields = W.d3q95_sweep(768, 256, 256, storage="fp32")
    assert 95 * wl.cells > 2 ** 32
    err = check_sampled_step(lbm, wl, fields, "fp32", warm=8)
    assert err <= TOL["fp32"], err


@pytest.mark.parametrize("variant", ["auto", "pair"])
def test_oblique_768x384x384_fp16_sampled_step(lbm, variant):
    """variant "pair": the two-cell kernel with 64-bit element indices (Q ncell =
    1.08e10 exceeds 32 bits)."""
    wl, fields = W.d3q95_oblique()
    v = None if variant == "auto" else lbm.VARIANT_PAIR
    err = check_sampled_step(lbm, wl, fields, "fp16", warm=32, variant=v)
    assert err <= TOL["fp16"], err


def test_adjoint_128cubed_conserved_mass_gradient(lbm):
    """dL/drho_N = 1/N through 500 FP32 steps (checkpoint every 22) maps back to the
    exact dL/drho_0 = 1/N and zero U, T and omega gradients.  Bounds: the FP32
    reverse sweep's relative rounding over 500 steps (1e-4 of the 1/N scale), and
    for omega 1e-3 against the ~5 summed per-step terms |lambda (f^eq - g)|."""
    import torch
    wl, fields = W.d3q95_adjoint()
    N = wl.cells
    lat = lbm.Lattice(wl.model, wl.dims, wl.omega, "fp32")
    T0 = lat.info["T0"]
    lat.init(fields.rho, fields.U, fields.theta * T0)
    lbm.lbm_record(lat.ctx, wl.steps, 22)
    shape = fields.rho.shape
    g = torch.full(shape, 1.0 / N, dtype=torch.float64, device="cuda")
    dr = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dU = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    dT = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dom = lbm.lbm_backward(lat.ctx, g, dr, dU, dT)
    lat.close()
    assert float((dr * N - 1.0).abs().max()) <= 1e-4
    assert float(dU.abs().max()) * N * np.sqrt(T0) <= 1e-4
    assert float(dT.abs().max()) * N * T0 <= 1e-4
    assert abs(dom) <= 1e-3
