"""Fourth-order Hermite discrete equilibrium (oracle).

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline; never by the product path.

The paper (text around Formulas 1-2 and after Formula 8) asks for an m-th order
Hermite expansion f_HE^eq of the Maxwellian about the lattice's own weight
exp(-v^2), truncated at degree N = m = 4, and takes the discrete equilibrium as
f_i^eq = w_i P^(N)(v_i), with exp(-v_i^2) merged into w_i.  The paper does not
print P^(4); the reading used here is the standard tensor Hermite series
written in unit-variance variables xi = sqrt(2) v (weight exp(-xi^2/2)):

    f_i^eq = w_i * sum_{n=0}^{4} (1/n!) a^(n) : H^(n)(xi_i)

with H^(n) the Hermite tensors and a^(n) the Hermite coefficients of the
Maxwellian rho N(xi; u, theta I) (u = sqrt(2) * the paper's dimensionless u,
theta = T/T0), i.e. a^(n) are the moments of N(u, (theta-1) I).

Pinned (tests/test_oracle_equilibrium.py): the moments sum_i f_i^eq xi_i^(k)
equal the Maxwellian's to order 4 (Formula 1, computed by Gauss-Hermite
product quadrature) and differ at order 5; an independent per-cell linear solve
of the moment conditions gives the same populations (uniqueness of the
degree-4 polynomial on a quadrature exact to degree 9).
"""
from __future__ import annotations

import numpy as np


def hermite_tensors(xi: np.ndarray):
    """H^(0..4)(xi) for xi of shape [Q, D]; returns a list of arrays [Q, D^n]."""
    Q, D = xi.shape
    I = np.eye(D)
    H0 = np.ones(Q)
    H1 = xi.copy()
    xx = np.einsum("qa,qb->qab", xi, xi)
    H2 = xx - I[None]
    xxx = np.einsum("qab,qc->qabc", xx, xi)
    H3 = xxx - (np.einsum("qa,bc->qabc", xi, I)
                + np.einsum("qb,ac->qabc", xi, I)
                + np.einsum("qc,ab->qabc", xi, I))
    xxxx = np.einsum("qabc,qd->qabcd", xxx, xi)
    H4 = (xxxx
          - (np.einsum("qab,cd->qabcd", xx, I) + np.einsum("qac,bd->qabcd", xx, I)
             + np.einsum("qad,bc->qabcd", xx, I) + np.einsum("qbc,ad->qabcd", xx, I)
             + np.einsum("qbd,ac->qabcd", xx, I) + np.einsum("qcd,ab->qabcd", xx, I))
          + (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
             + np.einsum("ad,bc->abcd", I, I))[None])
    return [H0, H1, H2, H3, H4]


def maxwellian_hermite_coefficients(rho, u, theta):
    """a^(0..4) of rho N(u, theta I); rho, theta shape [C], u shape [C, D].

    With s = theta - 1, a^(n) are the moments of a Gaussian of mean u and
    covariance s I (Isserlis): every way of pairing indices into deltas
    contributes s^(#pairs) times u on the unpaired indices.
    """
    C, D = u.shape
    I = np.eye(D)
    s = theta - 1.0
    a0 = rho
    a1 = rho[:, None] * u
    uu = np.einsum("ca,cb->cab", u, u)
    a2 = rho[:, None, None] * (uu + s[:, None, None] * I[None])
    uuu = np.einsum("cab,cd->cabd", uu, u)
    a3 = rho[:, None, None, None] * (
        uuu + s[:, None, None, None] * (np.einsum("ca,bd->cabd", u, I)
                                        + np.einsum("cb,ad->cabd", u, I)
                                        + np.einsum("cd,ab->cabd", u, I)))
    uuuu = np.einsum("cabd,ce->cabde", uuu, u)
    six = (np.einsum("cab,de->cabde", uu, I) + np.einsum("cad,be->cabde", uu, I)
           + np.einsum("cae,bd->cabde", uu, I) + np.einsum("cbd,ae->cabde", uu, I)
           + np.einsum("cbe,ad->cabde", uu, I) + np.einsum("cde,ab->cabde", uu, I))
    three = (np.einsum("ab,de->abde", I, I) + np.einsum("ad,be->abde", I, I)
             + np.einsum("ae,bd->abde", I, I))
    a4 = rho[:, None, None, None, None] * (
        uuuu + s[:, None, None, None, None] * six
        + (s * s)[:, None, None, None, None] * three[None])
    return [a0, a1, a2, a3, a4]


_FACT = [1.0, 1.0, 2.0, 6.0, 24.0]


def feq(model, rho, u, theta):
    """Discrete equilibrium f_i^eq for each cell.

    rho, theta: [C]; u: [C, D] in unit-variance units (u_xi = sqrt(2) c U_lattice).
    Returns [Q, C].  Works for real or complex inputs (complex-step derivatives).
    """
    xi = model.xi
    H = hermite_tensors(xi)
    a = maxwellian_hermite_coefficients(rho, u, theta)
    Q = xi.shape[0]
    C = rho.shape[0]
    P = np.zeros((C, Q), dtype=np.result_type(rho, u, theta, np.float64))
    for n in range(5):
        An = a[n].reshape(C, -1)
        Hn = H[n].reshape(Q, -1)
        P = P + (An @ Hn.T) / _FACT[n]
    return (P * model.w[None, :]).T


def moments_xi(model, f):
    """rho, u (unit-variance units, [C, D]) and theta of populations f [Q, C] (Formula 1, n <= 2)."""
    xi = model.xi
    D = model.D
    rho = f.sum(axis=0)
    j = xi.T @ f                                   # [D, C]
    E = (xi * xi).sum(axis=1) @ f                  # [C]
    u = (j / rho).T
    theta = (E / rho - (u * u).sum(axis=1)) / D
    return rho, u, theta
