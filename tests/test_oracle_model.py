"""Pins of oracle/model.py against the paper's printed tables and closed forms."""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from conftest import golden_rows
from oracle import model as M


def test_table1_by_enumeration_and_generating_function():
    """Table 1: Omega(m, D) by partition enumeration (Formula 8) and by the
    coefficients of the generating function of Formula 7."""
    rows = golden_rows("table1_omega.txt")
    for r in rows:
        D = int(r[0])
        printed = [int(v) for v in r[1:]]
        enum = [M.omega_count(m, D) for m in range(8)]
        gen = np.cumsum(M.pi_generating(7, D)).tolist()
        assert enum == printed, (D, enum, printed)
        assert gen == printed, (D, gen, printed)


def test_equation_classes_are_doubled_partitions():
    # m = 4: 9 equations in 2D, 11 in 3D (text after Formula 8)
    assert len(M.equation_classes(4, 2)) == 9
    assert len(M.equation_classes(4, 3)) == 11
    assert (8, 0, 0) in M.equation_classes(4, 3) and (4, 2, 2) in M.equation_classes(4, 3)


def test_formula4_double_factorial_identity():
    """Gamma((n+1)/2) = sqrt(pi) (n-1)!! / 2^(n/2) for even n (text after Formula 4)."""
    for n in range(0, 12, 2):
        dfact = 1
        for k in range(n - 1, 0, -2):
            dfact *= k
        assert math.isclose(M.gamma_half(n), math.sqrt(math.pi) * dfact / 2 ** (n / 2), rel_tol=1e-14)
    assert M.gaussian_moment((3, 0)) == 0.0
    assert math.isclose(M.gaussian_moment((0, 0, 0)), math.pi ** 1.5, rel_tol=1e-15)


@pytest.mark.parametrize("name,table,sizes", [
    ("D2Q33", "table2_d2q33.txt", {1: 1, 4: 6, 8: 1}),
    ("D3Q95", "table3_d3q95.txt", {1: 1, 6: 3, 8: 2, 12: 3, 24: 1}),
])
def test_tables_2_3_orbits_counts_and_digits(name, table, sizes):
    """Group sizes G_k, Q (Formula 9), unknowns = equations (Formula 10), and the
    FP64 solution of Formula 5 agreeing with every printed digit."""
    mdl = M.get_model(name)
    rows = golden_rows(table)
    c_printed = float(rows[0][1])
    groups = rows[1:]
    D = mdl.D
    counts = {}
    for r in groups:
        g = int(r[0]) - 1
        size = int(r[1])
        rep = tuple(int(v) for v in r[2:2 + D])
        assert rep == tuple(mdl.reps[g])
        assert len(M.orbit(rep)) == size
        counts[size] = counts.get(size, 0) + 1
    assert counts == sizes
    Q = sum(int(r[1]) for r in groups)
    assert Q == mdl.Q == (33 if D == 2 else 95)
    assert len(groups) + 1 == len(M.equation_classes(4, D))   # Formula 10
    assert mdl.residual < 1e-14
    assert abs(mdl.w.sum() - 1.0) < 1e-14
    assert np.all(mdl.W > 0)

    def half_ulp(s):
        mant = s.lower().split("e")[0]
        exp = int(s.lower().split("e")[1]) if "e" in s.lower() else 0
        dec = len(mant.split(".")[1]) if "." in mant else 0
        return 0.5 * 10.0 ** (exp - dec)

    for r in groups:
        g = int(r[0]) - 1
        assert abs(mdl.W[g] - float(r[-1])) <= half_ulp(r[-1]) * (1 + 1e-9), (g, mdl.W[g], r[-1])
    assert abs(mdl.c - c_printed) <= half_ulp(rows[0][1])


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_quadrature_exact_to_degree_9(name):
    """Formula 3 with m + N = 8 (and odd degrees by symmetry): sum_i w_i p(xi_i)
    equals the standard-normal expectation of every monomial up to degree 9,
    computed independently by a Gauss-Hermite product rule."""
    mdl = M.get_model(name)
    xi = mdl.xi
    D = mdl.D
    z, wz = hermegauss(8)          # exact to degree 15 per axis
    wz = wz / wz.sum()
    grids = np.meshgrid(*([z] * D), indexing="ij")
    wgrid = np.ones_like(grids[0])
    for k in range(D):
        wgrid = wgrid * np.meshgrid(*([wz] * D), indexing="ij")[k]
    import itertools
    worst = 0.0
    for a in itertools.product(range(10), repeat=D):
        if sum(a) > 9:
            continue
        lat = float(np.sum(mdl.w * np.prod(xi ** np.array(a)[None, :], axis=1)))
        ref = float(np.sum(wgrid * np.prod([grids[k] ** a[k] for k in range(D)], axis=0)))
        worst = max(worst, abs(lat - ref) / max(1.0, abs(ref)))
    assert worst < 1e-13
    # degree 10 is not matched for every monomial (the set is exactly 9th-degree)
    a10 = (10,) + (0,) * (D - 1)
    lat = float(np.sum(mdl.w * xi[:, 0] ** 10))
    assert abs(lat - 945.0) > 1e-3


def test_reference_temperature():
    """T0 = 1/(2 c^2) in lattice units (Theta = 2 k_B T0 / m_g with v = c e)."""
    for name in ("D2Q33", "D3Q95"):
        mdl = M.get_model(name)
        xi = mdl.xi
        # second moment of the weights in lattice units equals T0 per component
        e = mdl.e.astype(float)
        assert math.isclose(float(np.sum(mdl.w * e[:, 0] ** 2)), mdl.T0, rel_tol=1e-13)
        assert math.isclose(float(np.sum(mdl.w * xi[:, 0] ** 2)), 1.0, rel_tol=1e-13)


@pytest.mark.parametrize("reps,W,start", [
    (((0, 0), (1, 0), (1, 1)), (4 / 9, 1 / 9, 1 / 36), (0.5, 0.1, 0.03)),
    (((0, 0, 0), (1, 0, 0), (1, 1, 1)), (2 / 9, 1 / 9, 1 / 72), (0.25, 0.1, 0.02)),
    (((0, 0, 0), (1, 0, 0), (1, 1, 0)), (1 / 3, 1 / 18, 1 / 36), (0.3, 0.05, 0.03)),
])
def test_general_solver_reproduces_textbook_second_order_sets(reps, W, start):
    """Formula 10 admits three groups at m = 2 (Omega(2, D) = 4): the Newton solve of
    Formula 5 from a start away from the solution lands on the textbook D2Q9, D3Q15
    and D3Q19 weights with c^2 = 3/2."""
    assert M.omega_count(2, len(reps[0])) == len(reps) + 1
    Ws, c = M.solve_weights(reps, start, 1.1, m=2)
    assert math.isclose(c * c, 1.5, rel_tol=1e-14)
    assert np.allclose(Ws, W, rtol=1e-13, atol=0)
