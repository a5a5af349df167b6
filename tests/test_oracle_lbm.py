"""Pins of oracle/lbm.py: collision invariants, conservation, fixed points, the
streaming permutation, a naive per-cell brute force, and exact Riemann plateaus."""
import math

import numpy as np
import pytest

from oracle import lbm, riemann
from oracle.model import get_model
from paper_1303_4624_gb300 import workloads as W
from test_oracle_equilibrium import feq_by_moment_matching


def random_state(mdl, shape, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp * rng.standard_normal(shape)
    U = 0.05 * rng.standard_normal((mdl.D,) + shape)
    T = mdl.T0 * (1.0 + amp * rng.standard_normal(shape))
    S = lbm.init_populations(mdl, rho, U, T)
    # perturb away from equilibrium so the collision does something
    S = S * (1.0 + 0.02 * rng.standard_normal(S.shape))
    return S


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_collision_invariants_per_cell(name):
    mdl = get_model(name)
    shape = (3, 4, 5) if mdl.D == 3 else (1, 6, 7)
    g = random_state(mdl, shape, 1)
    out = lbm.collide(mdl, g, 1.7)
    xi = mdl.xi
    d = (out - g).reshape(mdl.Q, -1)
    gf = g.reshape(mdl.Q, -1)
    for weight in [np.ones(mdl.Q)] + [xi[:, k] for k in range(mdl.D)] + [(xi * xi).sum(1)]:
        scale = np.abs(weight) @ np.abs(gf)
        assert np.max(np.abs(weight @ d) / scale) < 1e-14


@pytest.mark.parametrize("name,shape", [("D2Q33", (1, 5, 7)), ("D3Q95", (4, 5, 6))])
def test_global_conservation_over_many_steps(name, shape):
    mdl = get_model(name)
    S = random_state(mdl, shape, 2)
    a0 = lbm.audit(mdl, S)
    S = lbm.run(mdl, S, 1.6, 300)
    a1 = lbm.audit(mdl, S)
    # FP64 roundoff accumulates over the 300 steps (about 1e-15 per step)
    assert abs(a1["mass"] - a0["mass"]) / a0["mass"] < 1e-12
    assert abs(a1["energy"] - a0["energy"]) / a0["energy"] < 1e-12
    assert np.max(np.abs(a1["momentum"] - a0["momentum"])) / a0["mass"] < 1e-12


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_rest_and_uniform_flow_are_fixed_points(name):
    mdl = get_model(name)
    shape = (3, 4, 5) if mdl.D == 3 else (1, 4, 6)
    for U0 in (0.0, 0.07):
        rho = np.full(shape, 0.8)
        U = np.zeros((mdl.D,) + shape)
        U[0] = U0
        T = np.full(shape, 1.1 * mdl.T0)
        S = lbm.init_populations(mdl, rho, U, T)
        S2 = lbm.run(mdl, S, 1.5, 200)
        r, u, t = lbm.macroscopic(mdl, S2)
        # roundoff over 200 steps
        assert np.max(np.abs(r - 0.8)) < 1e-12
        assert np.max(np.abs(u[0] - U0)) < 1e-12 and np.max(np.abs(u[1:])) < 1e-12
        assert np.max(np.abs(t / mdl.T0 - 1.1)) < 1e-12
        assert np.max(np.abs(S2 - S)) < 1e-12


@pytest.mark.parametrize("name,shape", [("D2Q33", (1, 3, 7)), ("D3Q95", (2, 3, 4)), ("D3Q95", (7, 1, 11))])
def test_streaming_permutation_integer_labels(name, shape):
    """Pull streaming with omega = 0 moves label(x) to x + n e_i, true modulo, bit for bit.
    The expected labels are computed with explicit index arithmetic, not np.roll."""
    mdl = get_model(name)
    nz, ny, nx = shape
    Q = mdl.Q
    idx = np.arange(nz * ny * nx, dtype=np.float64).reshape(shape)
    S = np.stack([idx + 1000.0 * i + 1.0 for i in range(Q)])
    n = 3
    out = S.copy()
    for _ in range(n):
        out = lbm.step(mdl, out, 0.0)
    for i in range(Q):
        e = mdl.e[i]
        ex, ey = int(e[0]), int(e[1])
        ez = int(e[2]) if mdl.D == 3 else 0
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    sx, sy, sz = (x - n * ex) % nx, (y - n * ey) % ny, (z - n * ez) % nz
                    assert out[i, z, y, x] == (sz * ny + sy) * nx + sx + 1000.0 * i + 1.0


@pytest.mark.parametrize("name,shape", [("D2Q33", (1, 3, 5)), ("D3Q95", (2, 3, 4))])
def test_naive_brute_force_step(name, shape):
    """A naive per-cell loop (modulo indexing, moment sums, linear-solve
    equilibrium, BGK) agrees with the oracle to 1e-13 on grids smaller than the reach."""
    mdl = get_model(name)
    S = random_state(mdl, shape, 3)
    omega = 1.3
    ref = lbm.step(mdl, S, omega)
    nz, ny, nx = shape
    xi = mdl.xi
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                g = np.empty(mdl.Q)
                for i in range(mdl.Q):
                    e = mdl.e[i]
                    ez = int(e[2]) if mdl.D == 3 else 0
                    g[i] = S[i, (z - ez) % nz, (y - int(e[1])) % ny, (x - int(e[0])) % nx]
                rho = g.sum()
                u = (g @ xi) / rho
                theta = ((g @ (xi * xi).sum(1)) / rho - u @ u) / mdl.D
                fe = feq_by_moment_matching(mdl, rho, u, theta)
                new = (1 - omega) * g + omega * fe
                assert np.max(np.abs(new - ref[:, z, y, x])) < 1e-13


@pytest.mark.parametrize("name,nx,steps", [("D3Q95", 1600, 100), ("D2Q33", 1000, 150)])
def test_riemann_plateaus(name, nx, steps):
    """The paper's shock tube states rho = p = 4 | 1, theta = 1, omega = 1.5
    (paragraph before Figure 1) on a quasi-1D periodic tube: density and
    temperature on both plateaus match the exact Riemann solution to 0.5 %."""
    mdl = get_model(name)
    gam = (mdl.D + 2.0) / mdl.D
    f = W.riemann_planar(mdl.D, nx, 1, 1, nx // 2, (4.0, 1.0), (1.0, 1.0), noise=0)
    S = lbm.init_populations(mdl, f.rho, f.U, f.theta * mdl.T0)
    S = lbm.run(mdl, S, 1.5, steps)
    rho, U, T = lbm.macroscopic(mdl, S)
    r, th = rho[0, 0], T[0, 0] / mdl.T0
    T0 = mdl.T0
    st = riemann.star_state(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, gam)
    ws = riemann.wave_speeds(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, gam)
    xc = np.arange(nx) + 0.5 - nx // 2

    def central(a, b):
        L = b - a
        return (xc > a + 0.3 * L) & (xc < b - 0.3 * L)

    mL = central(ws["left_tail"] * steps, ws["contact"] * steps)
    mR = central(ws["contact"] * steps, ws["right"] * steps)
    assert mL.sum() > 20 and mR.sum() > 20
    assert abs(r[mL].mean() / st.rho_L - 1) < 5e-3
    assert abs(r[mR].mean() / st.rho_R - 1) < 5e-3
    assert abs(th[mL].mean() / (st.p / st.rho_L / T0) - 1) < 5e-3
    assert abs(th[mR].mean() / (st.p / st.rho_R / T0) - 1) < 5e-3


def test_paper_shock_tube_with_fixed_ends():
    """The paper's shock tube (paragraph before Figure 1): states rho = p = 4 | 1,
    theta = 1, omega = 1.5, tube along z with the end planes held at C_L and C_R and
    periodic sides (here 1 x 1 cross-section, homogeneous in x and y).  Plateaus
    match the exact Riemann solution to 0.5 %; the end planes stay at f^eq of their
    states exactly."""
    mdl = get_model("D3Q95")
    T0, nz, steps = mdl.T0, 800, 120
    z = np.arange(nz).reshape(nz, 1, 1)
    rho = np.where(z < nz // 2, 4.0, 1.0).astype(float)
    S = lbm.init_populations(mdl, rho, np.zeros((3, nz, 1, 1)), np.full((nz, 1, 1), T0))
    ends = (2, 5, (4.0, np.zeros(3), T0), (1.0, np.zeros(3), T0))
    S = lbm.run(mdl, S, 1.5, steps, ends)
    r, _, T = lbm.macroscopic(mdl, S)
    r, th = r[:, 0, 0], T[:, 0, 0] / T0
    st = riemann.star_state(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, 5.0 / 3.0)
    ws = riemann.wave_speeds(4.0, 0.0, 4.0 * T0, 1.0, 0.0, T0, 5.0 / 3.0)
    zc = np.arange(nz) + 0.5 - nz // 2

    def central(a, b):
        L = b - a
        return (zc > a + 0.3 * L) & (zc < b - 0.3 * L)

    mL = central(ws["left_tail"] * steps, ws["contact"] * steps)
    mR = central(ws["contact"] * steps, ws["right"] * steps)
    assert abs(r[mL].mean() / st.rho_L - 1) < 5e-3 and abs(r[mR].mean() / st.rho_R - 1) < 5e-3
    assert abs(th[mL].mean() / (st.p / st.rho_L / T0) - 1) < 5e-3
    assert abs(th[mR].mean() / (st.p / st.rho_R / T0) - 1) < 5e-3
    fe_lo = lbm.init_populations(mdl, np.full((1, 1, 1), 4.0), np.zeros((3, 1, 1, 1)), np.full((1, 1, 1), T0))
    assert np.array_equal(S[:, :5], np.broadcast_to(fe_lo, (mdl.Q, 5, 1, 1)))


@pytest.mark.parametrize("name,shape", [("D2Q33", (1, 5, 7)), ("D3Q95", (3, 4, 5))])
def test_audit_totals_in_absolute_terms(name, shape):
    """The audit's totals equal the macroscopic definitions (Formula 1 with n <= 2:
    density, momentum and energy moments) of the fields the state was built from,
    in lattice units: mass = sum rho, momentum = sum rho U, energy =
    sum rho (D T + |U|^2) / 2.  The state is the discrete equilibrium of random
    fields, whose moments through order 2 are the Maxwellian's (pinned in
    test_oracle_equilibrium), so the expected totals come from the input fields, not
    from the populations: a missing 1/2, or momentum or energy taken in the
    unit-variance variables xi = sqrt(2) c e instead of e, fails."""
    mdl = get_model(name)
    rng = np.random.default_rng(31)
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, shape)
    U = 0.1 * rng.uniform(-1, 1, (mdl.D,) + shape)
    T = mdl.T0 * (1.0 + 0.2 * rng.uniform(-1, 1, shape))
    a = lbm.audit(mdl, lbm.init_populations(mdl, rho, U, T))
    mass = rho.sum()
    mom = (rho * U).reshape(mdl.D, -1).sum(axis=1)
    energy = (0.5 * rho * (mdl.D * T + (U * U).sum(axis=0))).sum()
    assert abs(a["mass"] - mass) <= 1e-13 * mass
    assert np.max(np.abs(a["momentum"] - mom)) <= 1e-13 * mass
    assert abs(a["energy"] - energy) <= 1e-13 * energy
    assert a["nonfinite"] == 0
    # the rest state f = w at rho = 1: min f / w is exactly 1
    rest = lbm.init_populations(mdl, np.ones(shape), np.zeros((mdl.D,) + shape),
                                np.full(shape, mdl.T0))
    assert abs(lbm.audit(mdl, rest)["min_f_over_w"] - 1.0) < 1e-14


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_audit_minimum_and_nonfinite_count_on_a_hand_built_state(name):
    """f_i = 1.5 w_i everywhere except one population of one cell set to 0.125 w_k
    (k at the end of a symmetry group, so the next direction's weight differs), and
    a NaN and two infinities planted elsewhere: min f / w is exactly 0.125 with the
    weights in direction order, the three non-finite values are counted one by one,
    and NaN never wins the minimum.  A +/- infinity pair would make the minimum
    -inf, so only +inf is planted here beside the NaN."""
    mdl = get_model(name)
    shape = (2, 3, 4) if mdl.D == 3 else (1, 3, 4)
    S = np.broadcast_to((1.5 * mdl.w).reshape(-1, 1, 1, 1), (mdl.Q,) + shape).copy()
    # the last direction of the first non-rest group: its weight differs from the next one's
    k = next(i for i in range(1, mdl.Q - 1) if mdl.w[i] != mdl.w[i + 1])
    S[k, 0, 1, 2] = 0.125 * mdl.w[k]
    S[0, 0, 2, 3] = np.nan
    S[mdl.Q - 1, 0, 0, 0] = np.inf
    S[1, 0, 2, 1] = np.inf
    a = lbm.audit(mdl, S)
    assert a["min_f_over_w"] == 0.125
    assert a["nonfinite"] == 3
    S[1, 0, 2, 1] = -np.inf
    assert lbm.audit(mdl, S)["min_f_over_w"] == -np.inf
