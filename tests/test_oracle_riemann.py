"""Pins of oracle/riemann.py: jump conditions and invariants of the exact solution."""
import math

import pytest

from oracle import riemann


@pytest.mark.parametrize("gam", [5.0 / 3.0, 2.0, 1.4])
def test_shock_rankine_hugoniot_and_rarefaction_invariants(gam):
    rL, uL, pL, rR, uR, pR = 4.0, 0.0, 4.0, 1.0, 0.0, 1.0
    st = riemann.star_state(rL, uL, pL, rR, uR, pR, gam)
    ws = riemann.wave_speeds(rL, uL, pL, rR, uR, pR, gam)
    S = ws["right"]
    # right shock: mass, momentum and energy fluxes in the shock frame are continuous
    m1, m2 = rR * (uR - S), st.rho_R * (st.u - S)
    assert math.isclose(m1, m2, rel_tol=1e-12)
    assert math.isclose(m1 * (uR - S) + pR, m2 * (st.u - S) + st.p, rel_tol=1e-12)
    eR = pR / ((gam - 1) * rR) + 0.5 * (uR - S) ** 2 + pR / rR
    eS = st.p / ((gam - 1) * st.rho_R) + 0.5 * (st.u - S) ** 2 + st.p / st.rho_R
    assert math.isclose(eR, eS, rel_tol=1e-12)
    # left rarefaction: isentropic and the Riemann invariant u + 2a/(gamma-1) is constant
    assert math.isclose(pL / rL ** gam, st.p / st.rho_L ** gam, rel_tol=1e-12)
    aL, aS = math.sqrt(gam * pL / rL), math.sqrt(gam * st.p / st.rho_L)
    assert math.isclose(uL + 2 * aL / (gam - 1), st.u + 2 * aS / (gam - 1), rel_tol=1e-12)
    # pressure and velocity are continuous across the contact; ordering of the waves
    assert ws["left"] < ws["left_tail"] < ws["contact"] < ws["right"]
    r, u, p = riemann.sample(rL, uL, pL, rR, uR, pR, gam, 0.5 * (ws["contact"] + ws["right"]))
    assert math.isclose(p, st.p) and math.isclose(r, st.rho_R)
    # inside the fan the Riemann invariant is still constant
    s = 0.5 * (ws["left"] + ws["left_tail"])
    r, u, p = riemann.sample(rL, uL, pL, rR, uR, pR, gam, s)
    a = math.sqrt(gam * p / r)
    assert math.isclose(u + 2 * a / (gam - 1), uL + 2 * aL / (gam - 1), rel_tol=1e-12)
    assert math.isclose(u - a, s, rel_tol=1e-12)


def test_trivial_and_mirror():
    st = riemann.star_state(1.0, 0.0, 1.0, 1.0, 0.0, 1.0, 5.0 / 3.0)
    assert math.isclose(st.p, 1.0) and abs(st.u) < 1e-14
    a = riemann.star_state(4.0, 0.0, 4.0, 1.0, 0.0, 1.0, 5.0 / 3.0)
    b = riemann.star_state(1.0, 0.0, 1.0, 4.0, 0.0, 4.0, 5.0 / 3.0)
    assert math.isclose(a.p, b.p, rel_tol=1e-13) and math.isclose(a.u, -b.u, rel_tol=1e-13)
    assert math.isclose(a.rho_L, b.rho_R, rel_tol=1e-13)
