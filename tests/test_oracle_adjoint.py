"""Pins of the oracle's discrete adjoint: a column-by-column complex-step
Jacobian of the collision, the dot-product identity, and central finite
differences of the whole rollout."""
import numpy as np
import pytest

from oracle import lbm
from oracle.model import get_model
from test_oracle_lbm import random_state


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_collision_adjoint_matches_full_jacobian(name):
    mdl = get_model(name)
    g = random_state(mdl, (1, 1, 3), 5).reshape(mdl.Q, -1)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(g.shape)
    omega = 1.4
    mu, dom = lbm.collide_adjoint(mdl, g, lam, omega)
    h = 1e-30
    shape = (mdl.Q, 1, 1, g.shape[1])
    for c in range(g.shape[1]):
        J = np.empty((mdl.Q, mdl.Q))
        for j in range(mdl.Q):
            gp = g.astype(np.complex128)
            gp[j, c] += 1j * h
            J[:, j] = lbm.collide(mdl, gp.reshape(shape), omega).reshape(mdl.Q, -1)[:, c].imag / h
        assert np.max(np.abs(J.T @ lam[:, c] - mu[:, c])) < 1e-12 * np.max(np.abs(mu[:, c]))
    # d C / d omega = f^eq - g
    e = 1e-7
    dC = (lbm.collide(mdl, g.reshape(shape), omega + e) - lbm.collide(mdl, g.reshape(shape), omega - e)) / (2 * e)
    assert np.allclose((lam * dC.reshape(mdl.Q, -1)).sum(0), dom, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_stream_adjoint_dot_product(name):
    mdl = get_model(name)
    rng = np.random.default_rng(3)
    shape = (mdl.Q,) + ((3, 4, 5) if mdl.D == 3 else (1, 4, 6))
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    assert abs(np.sum(lbm.stream(mdl, a) * b) - np.sum(a * lbm.stream_adjoint(mdl, b))) < 1e-12


@pytest.mark.parametrize("name,shape", [("D2Q33", (1, 3, 5)), ("D3Q95", (2, 3, 3))])
def test_rollout_gradients_vs_central_differences(name, shape):
    mdl = get_model(name)
    rng = np.random.default_rng(9)
    rho0 = 1.0 + 0.05 * rng.standard_normal(shape)
    U0 = 0.03 * rng.standard_normal((mdl.D,) + shape)
    T0 = mdl.T0 * (1.0 + 0.05 * rng.standard_normal(shape))
    c = rng.standard_normal(shape)          # linear loss L = sum c rho_N
    omega, n = 1.6, 4

    def loss(r, U, T, om):
        S = lbm.run(mdl, lbm.init_populations(mdl, r, U, T), om, n)
        return float((c * S.sum(axis=0)).sum())

    _, dr, dU, dT, dom = lbm.rollout_gradients(mdl, rho0, U0, T0, omega, n, c)
    h = 1e-6
    for k in [(0, 0, 0), (0, shape[1] - 1, shape[2] - 1)]:
        e = np.zeros(shape)
        e[k] = h
        fd = (loss(rho0 + e, U0, T0, omega) - loss(rho0 - e, U0, T0, omega)) / (2 * h)
        assert abs(fd - dr[k]) < 1e-7 * max(1.0, abs(fd))
        eU = np.zeros_like(U0)
        eU[(0,) + k] = h
        fd = (loss(rho0, U0 + eU, T0, omega) - loss(rho0, U0 - eU, T0, omega)) / (2 * h)
        assert abs(fd - dU[(0,) + k]) < 1e-7 * max(1.0, abs(fd))
        eT = e * mdl.T0
        fd = (loss(rho0, U0, T0 + eT, omega) - loss(rho0, U0, T0 - eT, omega)) / (2 * h * mdl.T0)
        assert abs(fd - dT[k]) < 1e-6 * max(1.0, abs(fd))
    fd = (loss(rho0, U0, T0, omega + h) - loss(rho0, U0, T0, omega - h)) / (2 * h)
    assert abs(fd - dom) < 1e-7 * max(1.0, abs(fd))
