"""Pins of oracle/equilibrium.py: Formula 1 (moments of the Maxwellian to order
m = 4), uniqueness of the degree-4 equilibrium, and the rest state."""
import itertools

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle.equilibrium import feq, moments_xi
from oracle.model import get_model

_Z, _WZ = hermegauss(8)
_WZ = _WZ / _WZ.sum()


def maxwell_moment(rho, u, theta, beta):
    """rho E[prod_k (u_k + sqrt(theta) z_k)^beta_k], z standard normal (exact by
    Gauss-Hermite quadrature since the integrand is a polynomial)."""
    out = rho
    for k, b in enumerate(beta):
        out *= np.sum(_WZ * (u[k] + np.sqrt(theta) * _Z) ** b)
    return out


def monomials(D, deg):
    return [a for a in itertools.product(range(deg + 1), repeat=D) if sum(a) <= deg]


def random_states(D, n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.4, 2.0, n)
    u = rng.uniform(-0.5, 0.5, (n, D))
    th = rng.uniform(0.6, 1.4, n)
    return rho, u, th


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_maxwellian_moments_through_order_4(name):
    """Formula 1 with m = 4: sum_i f_i^eq xi_i^beta equals the Maxwellian's for |beta| <= 4."""
    mdl = get_model(name)
    rho, u, th = random_states(mdl.D, 12, 11)
    f = feq(mdl, rho, u, th)
    xi = mdl.xi
    for a in monomials(mdl.D, 4):
        lat = (f * np.prod(xi ** np.array(a)[None, :], axis=1)[:, None]).sum(axis=0)
        ref = np.array([maxwell_moment(rho[c], u[c], th[c], a) for c in range(len(rho))])
        scale = np.maximum(1.0, np.abs(ref))
        assert np.max(np.abs(lat - ref) / scale) < 1e-13, a


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_order_5_is_not_matched(name):
    """The models are fourth order: some fifth moment differs for a moving, hot state."""
    mdl = get_model(name)
    rho, u, th = np.array([1.0]), np.array([[0.3] + [0.1] * (mdl.D - 1)]), np.array([1.3])
    f = feq(mdl, rho, u, th)
    xi = mdl.xi
    worst = 0.0
    for a in monomials(mdl.D, 5):
        if sum(a) != 5:
            continue
        lat = float((f[:, 0] * np.prod(xi ** np.array(a)[None, :], axis=1)).sum())
        worst = max(worst, abs(lat - maxwell_moment(1.0, u[0], 1.3, a)))
    assert worst > 1e-3


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_rest_state_is_the_weights(name):
    mdl = get_model(name)
    f = feq(mdl, np.array([1.0]), np.zeros((1, mdl.D)), np.array([1.0]))
    assert np.max(np.abs(f[:, 0] - mdl.w)) < 1e-16
    f2 = feq(mdl, np.array([2.5]), np.zeros((1, mdl.D)), np.array([1.0]))
    assert np.max(np.abs(f2[:, 0] - 2.5 * mdl.w)) < 1e-15


def feq_by_moment_matching(mdl, rho, u, theta):
    """Brute force: the degree-4 polynomial P with sum_i w_i P(xi_i) xi_i^beta equal
    to the Maxwellian moments for all |beta| <= 4, solved as a linear system."""
    xi = mdl.xi
    mons = monomials(mdl.D, 4)
    V = np.array([np.prod(xi ** np.array(a)[None, :], axis=1) for a in mons])   # [K, Q]
    A = (V * mdl.w[None, :]) @ V.T
    b = np.array([maxwell_moment(rho, u, theta, a) for a in mons])
    coef = np.linalg.solve(A, b)
    return mdl.w * (coef @ V)


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_matches_linear_solve_brute_force(name):
    mdl = get_model(name)
    rho, u, th = random_states(mdl.D, 6, 5)
    f = feq(mdl, rho, u, th)
    for c in range(len(rho)):
        ref = feq_by_moment_matching(mdl, rho[c], u[c], th[c])
        assert np.max(np.abs(f[:, c] - ref)) < 1e-13 * np.max(np.abs(ref)), c


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_moments_recover_the_fields(name):
    mdl = get_model(name)
    rho, u, th = random_states(mdl.D, 20, 7)
    r2, u2, t2 = moments_xi(mdl, feq(mdl, rho, u, th))
    assert np.max(np.abs(r2 - rho)) < 1e-14
    assert np.max(np.abs(u2 - u)) < 1e-14
    assert np.max(np.abs(t2 - th)) < 1e-14
