"""Parity of the adjoint kernels (lbm_record / lbm_backward) with the oracle's
exact discrete adjoint, finite differences, and the autograd wrapper."""
import numpy as np
import pytest

from oracle import lbm as olbm
from oracle.model import get_model

pytestmark = pytest.mark.gpu


def setup(model, dims, seed):
    mdl = get_model(model)
    rng = np.random.default_rng(seed)
    shape = dims[::-1]
    rho0 = 1.0 + 0.05 * rng.standard_normal(shape)
    U0 = 0.03 * rng.standard_normal((mdl.D,) + shape)
    T0 = mdl.T0 * (1.0 + 0.05 * rng.standard_normal(shape))
    c = rng.standard_normal(shape)
    return mdl, rho0, U0, T0, c


def gpu_grads(lbm, model, storage, dims, omega, n, k, rho0, U0, T0, c):
    lat = lbm.Lattice(model, dims, omega, storage)
    lat.init(rho0, U0, T0)
    lbm.lbm_record(lat.ctx, n, k)
    rhoN = np.zeros(dims[::-1])
    lbm.lbm_moments(lat.ctx, rhoN, None, None)
    dr, dU, dT = np.zeros_like(rho0), np.zeros_like(U0), np.zeros_like(T0)
    dom = lbm.lbm_backward(lat.ctx, np.ascontiguousarray(c), dr, dU, dT)
    return rhoN, dr, dU, dT, dom, lat


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, np.max(np.abs(b))))


@pytest.mark.parametrize("model,dims,n,k", [("D3Q95", (9, 4, 3), 6, 4), ("D2Q33", (10, 3, 1), 7, 3),
                                            ("D3Q95", (133, 3, 2), 5, 2),
                                            # every extent >= the reach: the one-correction wrap
                                            ("D3Q95", (11, 6, 5), 4, 2), ("D2Q33", (20, 6, 1), 5, 2)])
def test_fp64_adjoint_matches_oracle(lbm, model, dims, n, k):
    mdl, rho0, U0, T0, c = setup(model, dims, 1)
    rN, dr, dU, dT, dom, _ = gpu_grads(lbm, model, "fp64", dims, 1.6, n, k, rho0, U0, T0, c)
    orN, odr, odU, odT, odom = olbm.rollout_gradients(mdl, rho0, U0, T0, 1.6, n, c)
    assert rel(rN, orN) < 1e-12
    assert rel(dr, odr) < 1e-10
    assert rel(dU, odU) < 1e-10
    assert rel(dT, odT) < 1e-10
    assert abs(dom - odom) < 1e-10 * max(1.0, abs(odom))


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fp32_adjoint_matches_oracle(lbm, storage):
    """FP32 adjoint arithmetic against the FP64 discrete adjoint: 1e-4 relative.
    (With FP16 state storage the forward trajectory itself is rounded, so the
    bound there is the storage precision.)"""
    model, dims = "D3Q95", (40, 6, 5)
    mdl, rho0, U0, T0, c = setup(model, dims, 2)
    _, dr, dU, dT, dom, _ = gpu_grads(lbm, model, storage, dims, 1.6, 10, 3, rho0, U0, T0, c)
    _, odr, odU, odT, odom = olbm.rollout_gradients(mdl, rho0, U0, T0, 1.6, 10, c)
    tol = 1e-4 if storage == "fp32" else 5e-3
    assert rel(dr, odr) < tol
    assert rel(dU, odU) < tol
    assert rel(dT, odT) < tol
    assert abs(dom - odom) < tol * max(1.0, abs(odom))


def test_checkpoint_schedules_are_bitwise_identical(lbm):
    model, dims = "D3Q95", (12, 5, 4)
    _, rho0, U0, T0, c = setup(model, dims, 3)
    outs = [gpu_grads(lbm, model, "fp32", dims, 1.7, 9, k, rho0, U0, T0, c)[:5] for k in (1, 4, 9, 20)]
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(np.asarray(a), np.asarray(b))


def test_fp64_gradients_vs_central_differences_on_gpu(lbm):
    """Central differences of the GPU FP64 forward against the GPU adjoint."""
    model, dims = "D3Q95", (7, 3, 2)
    mdl, rho0, U0, T0, c = setup(model, dims, 4)
    n, om = 5, 1.5
    _, dr, dU, dT, dom, lat = gpu_grads(lbm, model, "fp64", dims, om, n, 2, rho0, U0, T0, c)

    def loss(r, U, T, o):
        lbm.lbm_set_omega(lat.ctx, o)
        lat.init(r, U, T)
        lat.step(n)
        rho, _, _ = lat.moments()
        return float((c * rho).sum())

    h = 1e-6
    k = (1, 2, 3)
    e = np.zeros_like(rho0)
    e[k] = h
    fd = (loss(rho0 + e, U0, T0, om) - loss(rho0 - e, U0, T0, om)) / (2 * h)
    assert abs(fd - dr[k]) < 1e-6 * max(1.0, abs(fd))
    eT = e * mdl.T0
    fd = (loss(rho0, U0, T0 + eT, om) - loss(rho0, U0, T0 - eT, om)) / (2 * h * mdl.T0)
    assert abs(fd - dT[k]) < 1e-6 * max(1.0, abs(fd))
    fd = (loss(rho0, U0, T0, om + h) - loss(rho0, U0, T0, om - h)) / (2 * h)
    assert abs(fd - dom) < 1e-6 * max(1.0, abs(fd))


def test_autograd_function(lbm):
    torch = pytest.importorskip("torch")
    from paper_1303_4624_gb300.autograd import rollout
    model, dims = "D3Q95", (16, 4, 3)
    mdl, rho0, U0, T0, c = setup(model, dims, 5)
    lat = lbm.Lattice(model, dims, 1.6, "fp64")
    dev = torch.device("cuda")
    r = torch.tensor(rho0, device=dev, requires_grad=True)
    U = torch.tensor(U0, device=dev, requires_grad=True)
    T = torch.tensor(T0, device=dev, requires_grad=True)
    om = torch.tensor(1.6, dtype=torch.float64, device=dev, requires_grad=True)
    target = torch.tensor(c, device=dev)
    rhoN = rollout(lat, r, U, T, om, 6, 3)
    loss = ((rhoN - target) ** 2).mean()
    loss.backward()
    g = 2.0 * (rhoN.detach().cpu().numpy() - c) / c.size
    _, odr, odU, odT, odom = olbm.rollout_gradients(mdl, rho0, U0, T0, 1.6, 6, g)
    assert rel(r.grad.cpu().numpy(), odr) < 1e-10
    assert rel(U.grad.cpu().numpy(), odU) < 1e-10
    assert rel(T.grad.cpu().numpy(), odT) < 1e-10
    assert abs(om.grad.item() - odom) < 1e-10 * max(1.0, abs(odom))


def min_recompute(n, free):
    """Fewest forward steps that reverse n steps with `free` extra stored states
    (store a state m steps on, reverse the rest with one slot fewer, then the first
    m; with no slot every state is recomputed from the start)."""
    cost = [[0] * (free + 1) for _ in range(n + 1)]
    for l in range(2, n + 1):
        cost[l][0] = l * (l - 1) // 2
        for f in range(1, free + 1):
            cost[l][f] = min(m + cost[l - m][f - 1] + cost[m][f] for m in range(1, l))
    return cost[n][free]


def test_optimal_recompute_counts():
    """The schedule's cost against hand counts: 300 steps with 7 stored states (S_0
    and 6 more) take 1035 recomputed steps (bisection 1191), with 6 states 1170
    (bisection 1249); no spare state is the triangular count."""
    assert min_recompute(300, 6) == 1035 and min_recompute(300, 5) == 1170
    assert min_recompute(11, 0) == 55 and min_recompute(2, 1) == 1 and min_recompute(1, 3) == 0


@pytest.mark.parametrize("max_states", [1, 2, 3, 16])
def test_bounded_schedule_matches_uniform_bitwise(lbm, max_states):
    """lbm_record_bounded stores at most max_states states and recomputes the rest;
    the gradients equal the uniform schedule's bit for bit (same kernels, same order)."""
    model, dims, n = "D3Q95", (12, 5, 4), 11
    _, rho0, U0, T0, c = setup(model, dims, 6)
    ref = gpu_grads(lbm, model, "fp32", dims, 1.7, n, 4, rho0, U0, T0, c)[:5]
    lat = lbm.Lattice(model, dims, 1.7, "fp32")
    lat.init(rho0, U0, T0)
    lbm.lbm_record_bounded(lat.ctx, n, max_states)
    rhoN = np.zeros(dims[::-1])
    lbm.lbm_moments(lat.ctx, rhoN, None, None)
    dr, dU, dT = np.zeros_like(rho0), np.zeros_like(U0), np.zeros_like(T0)
    before = lbm.lbm_launch_count(lat.ctx)
    dom = lbm.lbm_backward(lat.ctx, np.ascontiguousarray(c), dr, dU, dT)
    # launches: the optimal number of recomputed forward steps, n adjoint steps,
    # grad_init and the omega reduction
    assert lbm.lbm_launch_count(lat.ctx) - before == min_recompute(n, max_states - 1) + n + 2
    for a, b in zip((rhoN, dr, dU, dT, dom), ref):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    # afterwards the context holds the initial state
    r0, _, _ = lat.moments()
    assert np.allclose(r0, rho0, rtol=1e-6)
