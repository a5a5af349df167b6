"""The host-side model generator (lbm_equation_count, lbm_generate_model) against
what the paper and the mathematics fix.  Runs on the CPU (no GPU calls).

Pins:
* Table 1: every printed Omega(m, D), D = 1..4, m = 0..7;
* the textbook second-order sets that Formula 10 admits (Omega(2, D) = 4, so three
  groups): D2Q9 (4/9, 1/9, 1/36), D3Q15 (2/9, 1/9, 1/72) and D3Q19 (1/3, 1/18,
  1/36), all with c^2 = 3/2 (unit-variance-1/2 Maxwellian, c_s^2 = 1/3 in e units);
* Tables 2 and 3 (orbit sizes of Formula 9, printed digits of c and every weight)
  and the library's own D2Q33 / D3Q95 tables (a separate Newton solve);
* the defining property itself, checked by brute force over every monomial up to
  degree 2m (odd ones included): sum_i w_i v_i^a equals the Gaussian moment;
* the errors: Formula 10 not met, repeated orbit, no positive solution.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import golden_rows


@pytest.fixture(scope="module")
def gen(built_lib):
    from paper_1303_4624_gb300 import lbm
    return lbm


def gaussian_moment(a):
    """E[prod x_k^a_k] for independent N(0, 1/2) components (Formula 4 over pi^(D/2))."""
    r = 1.0
    for x in a:
        if x % 2:
            return 0.0
        r *= math.prod(range(x - 1, 0, -2)) / 2 ** (x // 2)
    return r


def assert_isotropic_to_order(model, D, m, tol):
    v = model["c"] * model["e"].astype(np.float64)
    for a in itertools.product(range(2 * m + 1), repeat=D):
        if sum(a) > 2 * m:
            continue
        got = float(np.sum(model["w"] * np.prod(v ** np.array(a), axis=1)))
        assert abs(got - gaussian_moment(a)) <= tol, (a, got, gaussian_moment(a))


def test_table1_equation_counts(gen):
    for row in golden_rows("table1_omega.txt"):
        D = int(row[0])
        for m, v in enumerate(row[1:]):
            assert gen.lbm_equation_count(m, D) == int(v), (D, m)


SECOND_ORDER = {
    "D2Q9": (2, [(0, 0), (1, 0), (1, 1)], [4 / 9, 1 / 9, 1 / 36], [1, 4, 4]),
    "D3Q15": (3, [(0, 0, 0), (1, 0, 0), (1, 1, 1)], [2 / 9, 1 / 9, 1 / 72], [1, 6, 8]),
    "D3Q19": (3, [(0, 0, 0), (1, 0, 0), (1, 1, 0)], [1 / 3, 1 / 18, 1 / 36], [1, 6, 12]),
}


@pytest.mark.parametrize("name", sorted(SECOND_ORDER))
def test_second_order_sets_closed_forms(gen, name):
    D, reps, W, sizes = SECOND_ORDER[name]
    r = gen.lbm_generate_model(D, 2, reps)
    assert r["Q"] == sum(sizes) == int(name.split("Q")[1])
    assert r["nsolutions"] == 1
    assert abs(r["c"] - math.sqrt(1.5)) < 1e-15
    k = 0
    for Wg, n in zip(W, sizes):
        assert np.allclose(r["w"][k:k + n], Wg, rtol=1e-14, atol=0)
        k += n
    assert abs(r["w"].sum() - 1.0) < 1e-15
    assert_isotropic_to_order(r, D, 2, 1e-14)


def table(name):
    rows = golden_rows(name)
    c = float(rows[0][1])
    groups = [(int(r[1]), tuple(int(x) for x in r[2:-1]), float(r[-1])) for r in rows[1:]]
    return c, groups


@pytest.mark.parametrize("name,fname,D", [("D2Q33", "table2_d2q33.txt", 2),
                                          ("D3Q95", "table3_d3q95.txt", 3)])
def test_paper_models_regenerated(gen, name, fname, D):
    c_printed, groups = table(fname)
    reps = [g[1] for g in groups]
    r = gen.lbm_generate_model(D, 4, reps)
    assert r["Q"] == sum(g[0] for g in groups) == int(name.split("Q")[1])
    assert r["nsolutions"] == 1
    assert r["residual"] < 1e-13
    # printed digits (six significant figures)
    assert abs(r["c"] / c_printed - 1) < 5e-6
    k = 0
    for size, rep, w_printed in groups:
        assert set(map(tuple, np.abs(r["e"][k:k + size]).tolist())) <= set(
            itertools.permutations(rep)), rep
        assert np.all(r["w"][k:k + size] == r["w"][k]), rep
        assert abs(r["w"][k] / w_printed - 1) < 5e-6, (rep, r["w"][k], w_printed)
        k += size
    # the library's table for the kernels comes from a separate Newton solve
    info = gen.lbm_model_info(name)
    assert abs(r["c"] / info["c"] - 1) < 1e-13
    mine = {tuple(v): wv for v, wv in zip(r["e"].tolist(), r["w"])}
    assert set(mine) == {tuple(v) for v in info["e"].tolist()}
    for v, wv in zip(info["e"].tolist(), info["w"]):
        assert abs(mine[tuple(v)] / wv - 1) < 1e-12
    assert_isotropic_to_order(r, D, 4, 1e-12)


def velocity_count(gen, D, m, reps):
    """*Q from lbm_generate_model with qmax = 0 (set before the solve is attempted)."""
    import ctypes
    reps = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
    Q = ctypes.c_int(0)
    c = ctypes.c_double(0)
    rc = gen._lib.lbm_generate_model(D, m, len(reps), reps.ctypes.data, 0, 0, ctypes.byref(Q),
                                     None, None, ctypes.byref(c), None, None)
    assert rc == gen.LBM_EINVAL
    return Q.value


def test_orbit_sizes_are_the_groups_of_formula_9(gen):
    """n(v) = sum_k k n_k with I_2 = {1, 4, 8} and I_3 = {1, 6, 8, 12, 24, 48}: every
    representative type of the text, as the third group of an m = 2 set."""
    for rep, size in [((0, 0), 1), ((2, 0), 4), ((2, 2), 4), ((2, 1), 8)]:
        reps = [(3, 0), (3, 3), rep]
        assert velocity_count(gen, 2, 2, reps) == 4 + 4 + size, rep
    for rep, size in [((0, 0, 0), 1), ((2, 0, 0), 6), ((2, 2, 2), 8), ((2, 2, 0), 12),
                      ((2, 2, 1), 24), ((2, 1, 0), 24), ((3, 2, 1), 48)]:
        reps = [(3, 0, 0), (3, 3, 3), rep]
        assert velocity_count(gen, 3, 2, reps) == 6 + 8 + size, rep


def test_errors(gen):
    # Formula 10: D3Q27 has four groups but Omega(2, 3) = 4 needs three
    with pytest.raises(gen.LbmError) as ei:
        gen.lbm_generate_model(3, 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)])
    assert ei.value.code == gen.LBM_EINVAL and "Formula 10" in str(ei.value)
    # the same orbit twice
    with pytest.raises(gen.LbmError) as ei:
        gen.lbm_generate_model(2, 2, [(0, 0), (1, 0), (0, -1)])
    assert "same orbit" in str(ei.value)
    # axis-only velocities cannot carry the mixed moment <x^2 y^2> = 1/4
    with pytest.raises(gen.LbmError) as ei:
        gen.lbm_generate_model(2, 2, [(0, 0), (1, 0), (2, 0)])
    assert "no solution" in str(ei.value)
    with pytest.raises(gen.LbmError):
        gen.lbm_equation_count(8, 3)
    with pytest.raises(gen.LbmError):
        gen.lbm_generate_model(2, 2, [(0, 0), (1, 0), (9, 0)])


def test_oracle_general_solver_agrees(gen):
    """The oracle's Newton solve of Formula 5 (started away from the solution) and
    the generator's determinant-root method land on the same D3Q19."""
    from oracle import model as om
    r = gen.lbm_generate_model(3, 2, SECOND_ORDER["D3Q19"][1])
    W, c = om.solve_weights(SECOND_ORDER["D3Q19"][1], [0.3, 0.05, 0.03], 1.2, m=2)
    assert abs(c - r["c"]) < 1e-14
    assert np.allclose(W, [r["w"][0], r["w"][1], r["w"][7]], rtol=1e-13, atol=0)
