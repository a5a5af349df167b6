"""Exact solution of the one-dimensional Riemann problem for an ideal gas (oracle).

Test infrastructure: imported only by tests; never by the product path.

The paper's only experiment (shock tube, Figure 1) compares the D3Q95 model
with the analytical Riemann solution on the plateaus.  The figure itself is not
available, so the oracle computes that analytical solution: a gas with
p = rho T (lattice units) and gamma = (D + 2)/D, the ratio of a monatomic gas
whose D translational degrees of freedom are the model's D velocity
components.  The solver is the textbook construction: the star pressure p* is
the root of f_L(p) + f_R(p) + (u_R - u_L) = 0 (shock branch from the
Rankine-Hugoniot relations, rarefaction branch from the isentropic relations),
found by Newton's method; the self-similar solution is then sampled at x/t.

Pinned by tests/test_oracle_riemann.py: Rankine-Hugoniot jump conditions
across the computed shock, constancy of the Riemann invariant and entropy across
the rarefaction, the trivial problem with equal states, and mirror symmetry.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class StarState:
    p: float
    u: float
    rho_L: float
    rho_R: float


def _f_branch(p, rho, pk, g):
    """f_K(p) and its derivative for one side K (shock if p > p_K, else rarefaction)."""
    a = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        f = (p - pk) * sq
        df = sq * (1.0 - 0.5 * (p - pk) / (p + B))
    else:
        f = 2.0 * a / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * a) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rho_L, u_L, p_L, rho_R, u_R, p_R, gamma) -> StarState:
    g = gamma
    p = 0.5 * (p_L + p_R)
    for _ in range(200):
        fL, dL = _f_branch(p, rho_L, p_L, g)
        fR, dR = _f_branch(p, rho_R, p_R, g)
        F = fL + fR + (u_R - u_L)
        dp = -F / (dL + dR)
        p_new = max(p + dp, 1e-12 * p)
        if abs(p_new - p) <= 1e-15 * p:
            p = p_new
            break
        p = p_new
    fL, _ = _f_branch(p, rho_L, p_L, g)
    fR, _ = _f_branch(p, rho_R, p_R, g)
    u = 0.5 * (u_L + u_R) + 0.5 * (fR - fL)

    def rho_star(rho, pk):
        if p > pk:
            r = (g - 1.0) / (g + 1.0)
            return rho * (p / pk + r) / (r * p / pk + 1.0)
        return rho * (p / pk) ** (1.0 / g)

    return StarState(p, u, rho_star(rho_L, p_L), rho_star(rho_R, p_R))


def sample(rho_L, u_L, p_L, rho_R, u_R, p_R, gamma, s):
    """(rho, u, p) of the self-similar solution at s = x/t."""
    g = gamma
    st = star_state(rho_L, u_L, p_L, rho_R, u_R, p_R, gamma)
    if s <= st.u:
        rho, u, pk = rho_L, u_L, p_L
        a = math.sqrt(g * pk / rho)
        if st.p > pk:
            S = u - a * math.sqrt((g + 1.0) / (2.0 * g) * st.p / pk + (g - 1.0) / (2.0 * g))
            return (rho, u, pk) if s < S else (st.rho_L, st.u, st.p)
        a_star = a * (st.p / pk) ** ((g - 1.0) / (2.0 * g))
        head, tail = u - a, st.u - a_star
        if s < head:
            return rho, u, pk
        if s > tail:
            return st.rho_L, st.u, st.p
        c = 2.0 / (g + 1.0) * (a + 0.5 * (g - 1.0) * (u - s))
        uu = 2.0 / (g + 1.0) * (a + 0.5 * (g - 1.0) * u + s)
        rr = rho * (c / a) ** (2.0 / (g - 1.0))
        return rr, uu, pk * (c / a) ** (2.0 * g / (g - 1.0))
    rho, u, pk = rho_R, u_R, p_R
    a = math.sqrt(g * pk / rho)
    if st.p > pk:
        S = u + a * math.sqrt((g + 1.0) / (2.0 * g) * st.p / pk + (g - 1.0) / (2.0 * g))
        return (rho, u, pk) if s > S else (st.rho_R, st.u, st.p)
    a_star = a * (st.p / pk) ** ((g - 1.0) / (2.0 * g))
    head, tail = u + a, st.u + a_star
    if s > head:
        return rho, u, pk
    if s < tail:
        return st.rho_R, st.u, st.p
    c = 2.0 / (g + 1.0) * (a - 0.5 * (g - 1.0) * (u - s))
    uu = 2.0 / (g + 1.0) * (-a + 0.5 * (g - 1.0) * u + s)
    rr = rho * (c / a) ** (2.0 / (g - 1.0))
    return rr, uu, pk * (c / a) ** (2.0 * g / (g - 1.0))


def wave_speeds(rho_L, u_L, p_L, rho_R, u_R, p_R, gamma):
    """Leftmost and rightmost signal speeds and the contact speed (for plateau masks)."""
    g = gamma
    st = star_state(rho_L, u_L, p_L, rho_R, u_R, p_R, gamma)
    aL = math.sqrt(g * p_L / rho_L)
    aR = math.sqrt(g * p_R / rho_R)
    if st.p > p_L:
        left = u_L - aL * math.sqrt((g + 1.0) / (2.0 * g) * st.p / p_L + (g - 1.0) / (2.0 * g))
        left_tail = left
    else:
        left = u_L - aL
        left_tail = st.u - aL * (st.p / p_L) ** ((g - 1.0) / (2.0 * g))
    if st.p > p_R:
        right = u_R + aR * math.sqrt((g + 1.0) / (2.0 * g) * st.p / p_R + (g - 1.0) / (2.0 * g))
        right_tail = right
    else:
        right = u_R + aR
        right_tail = st.u + aR * (st.p / p_R) ** ((g - 1.0) / (2.0 * g))
    return {"left": left, "left_tail": left_tail, "contact": st.u,
            "right_tail": right_tail, "right": right}
