"""Velocity sets, weights and equation counts of the on-lattice models (oracle).

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline; never by the product path.

What this module restates from the paper (arXiv:1303.4624):

* Formula 4: the Gaussian moments  int exp(-v^2) v^n dv = prod Gamma((a+1)/2)
  for all-even exponents, zero otherwise.
* Formula 5: the isotropic moment equations  sum_i w_i v_i^n = (Formula 4)
  for even exponent classes up to n_max = 2m, with the right side divided by
  pi^(D/2) so that sum_i w_i = 1 (the printed weights of Tables 2 and 3 sum to
  one, so the tables use this normalisation).
* Formulas 6-8: Omega(m, D) = sum_{q<=m} pi(q, D), the number of equations,
  counted both by enumerating partitions and from the generating function of
  Formula 7.  Pinned by Table 1.
* The symmetry groups G_k (text before Formula 9): every representative
  velocity is expanded by all coordinate permutations and sign changes.
  Formula 9 / 10 give the number of velocities and unknowns.  Pinned by
  Q = 33 / 95 and 9 / 11 unknowns.
* Tables 2 and 3: the representatives, and printed weights / c that start a
  Newton solve of Formula 5 to FP64.  Pinned by the printed digits.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

# Tables 2 and 3: (representative e, printed weight), printed c.
TABLE2_D2Q33 = (
    ((0, 0), 0.161987),
    ((1, 0), 0.143204),
    ((1, 1), 0.0338840),
    ((2, 0), 0.00556112),
    ((2, 2), 8.44799e-5),
    ((3, 0), 0.00113254),
    ((2, 1), 0.0128169),
    ((4, 4), 3.45552e-6),
)
TABLE2_C = 0.819381

TABLE3_D3Q95 = (
    ((0, 0, 0), 0.206847),
    ((2, 0, 0), 0.00442257),
    ((2, 2, 0), 0.0333341),
    ((2, 2, 2), 0.0128902),
    ((3, 0, 0), 0.0287920),
    ((3, 3, 0), 0.00264319),
    ((3, 3, 3), 0.000927908),
    ((2, 2, 5), 0.00106078),
    ((4, 4, 0), 0.000804376),
    ((5, 0, 0), 0.00274697),
)
TABLE3_C = 0.421803

# Order of accuracy of both tabulated models ("fourth-order", text before Table 2).
M_ORDER = 4


def gamma_half(n: int) -> float:
    """Gamma((n+1)/2) for n >= 0 (the factor of Formula 4)."""
    return math.gamma((n + 1) / 2.0)


def gaussian_moment(a: tuple[int, ...]) -> float:
    """Formula 4: int exp(-v^2) v^a dv over R^D (zero unless every a_alpha is even)."""
    if any(x % 2 for x in a):
        return 0.0
    out = 1.0
    for x in a:
        out *= gamma_half(x)
    return out


def normalised_gaussian_moment(a: tuple[int, ...]) -> float:
    """Formula 4 divided by its n = 0 value pi^(D/2): the right side of Formula 5 with sum w = 1."""
    return gaussian_moment(a) / math.pi ** (len(a) / 2.0)


# ---------------------------------------------------------------- partitions (Formulas 6-8)

def partitions(q: int, max_parts: int, largest: int | None = None):
    """All partitions of q into at most ``max_parts`` parts, as non-increasing tuples."""
    if largest is None:
        largest = q
    if q == 0:
        yield ()
        return
    if max_parts == 0:
        return
    for first in range(min(q, largest), 0, -1):
        for rest in partitions(q - first, max_parts - 1, first):
            yield (first,) + rest


def pi_count(q: int, D: int) -> int:
    """pi(q, D): number of partitions of q into at most D parts (pi(0, D) = 1)."""
    return sum(1 for _ in partitions(q, D))


def omega_count(m: int, D: int) -> int:
    """Formula 8: Omega(m, D) = sum_{q=0}^{m} pi(q, D), by enumeration."""
    return sum(pi_count(q, D) for q in range(m + 1))


def pi_generating(qmax: int, D: int) -> list[int]:
    """Coefficients of prod_{k=1}^{D} 1/(1 - x^k) up to x^qmax (Formula 7)."""
    coeff = [1] + [0] * qmax
    for k in range(1, D + 1):
        # multiply by the geometric series 1 + x^k + x^2k + ...
        new = [0] * (qmax + 1)
        for q in range(qmax + 1):
            s = 0
            j = q
            while j >= 0:
                s += coeff[j]
                j -= k
            new[q] = s
        coeff = new
    return coeff


def equation_classes(m: int, D: int) -> list[tuple[int, ...]]:
    """Even exponent classes of Formula 5 up to n_max = 2m.

    Each partition of q <= m into at most D parts, doubled and padded with
    zeros to length D, is one independent equation (the isotropic set makes
    every permutation of the exponents give the same equation).
    """
    out = []
    for q in range(m + 1):
        for p in partitions(q, D):
            a = tuple(2 * x for x in p) + (0,) * (D - len(p))
            out.append(a)
    return out


# ---------------------------------------------------------------- symmetry groups (Formula 9)

def orbit(rep: tuple[int, ...]) -> list[tuple[int, ...]]:
    """All distinct signed permutations of a representative velocity."""
    D = len(rep)
    pts = set()
    for perm in itertools.permutations(range(D)):
        for signs in itertools.product((1, -1), repeat=D):
            pts.add(tuple(signs[k] * rep[perm[k]] for k in range(D)))
    return sorted(pts)


@dataclass
class Model:
    name: str
    D: int
    reps: tuple                  # representative integer velocities, one per group
    W: np.ndarray                # solved weight per group (FP64)
    c: float                     # solved lattice-speed scale c (v_i = c e_i)
    e: np.ndarray                # [Q, D] integer lattice velocities
    group: np.ndarray            # [Q] group index of each velocity
    w: np.ndarray                # [Q] weight per velocity
    residual: float              # max |Formula 5 residual| at the solution

    @property
    def Q(self) -> int:
        return self.e.shape[0]

    @property
    def xi(self) -> np.ndarray:
        """Velocities in unit-variance units xi_i = sqrt(2) v_i = sqrt(2) c e_i."""
        return math.sqrt(2.0) * self.c * self.e.astype(np.float64)

    @property
    def T0(self) -> float:
        """Reference temperature in lattice units (Delta x = Delta t = 1, k_B/m_g = 1).

        The paper's dimensionless velocity is v = Theta^(-1/2) V with
        Theta = 2 k_B T0 / m_g; on the lattice v_i = c e_i with V_i = e_i, so
        Theta = 1/c^2 and T0 = 1/(2 c^2).
        """
        return 1.0 / (2.0 * self.c * self.c)

    @property
    def reach(self) -> int:
        return int(np.abs(self.e).max())


def _group_moments(reps, a):
    """sum over the orbit of each representative of prod e_alpha^a_alpha."""
    out = []
    for r in reps:
        s = 0.0
        for e in orbit(r):
            p = 1.0
            for x, k in zip(e, a):
                p *= float(x) ** k
            s += p
        out.append(s)
    return np.array(out)


def formula5_residual(reps, W, c, m=M_ORDER):
    """Residuals of Formula 5 (normalised) at group weights W and scale c."""
    D = len(reps[0])
    res = []
    for a in equation_classes(m, D):
        n = sum(a)
        lhs = float(np.dot(W, _group_moments(reps, a))) * c ** n
        res.append(lhs - normalised_gaussian_moment(a))
    return np.array(res)


def solve_weights(reps, W_start, c_start, m=M_ORDER, iters=50):
    """Newton's method on Formula 5 for the group weights and c, from a start point.

    Unknowns are (W_1..W_G, c); the system is square when Formula 10 holds.
    """
    D = len(reps[0])
    classes = equation_classes(m, D)
    M = np.array([_group_moments(reps, a) for a in classes])      # [neq, G]
    n = np.array([sum(a) for a in classes], dtype=np.float64)
    rhs = np.array([normalised_gaussian_moment(a) for a in classes])
    if M.shape[0] != M.shape[1] + 1:
        raise ValueError("Formula 10 does not hold: %d equations, %d unknowns"
                         % (M.shape[0], M.shape[1] + 1))
    x = np.concatenate([np.asarray(W_start, dtype=np.float64), [float(c_start)]])
    for _ in range(iters):
        W, c = x[:-1], x[-1]
        cn = c ** n
        F = (M @ W) * cn - rhs
        J = np.empty((len(classes), len(x)))
        J[:, :-1] = M * cn[:, None]
        J[:, -1] = (M @ W) * n * c ** np.maximum(n - 1, 0)
        dx = np.linalg.solve(J, -F)
        x = x + dx
        if np.max(np.abs(dx)) < 1e-17:
            break
    W, c = x[:-1], x[-1]
    return W, c


def build_model(name: str) -> Model:
    """Expand Table 2 or 3 and re-solve Formula 5 in FP64."""
    if name == "D2Q33":
        table, c0 = TABLE2_D2Q33, TABLE2_C
    elif name == "D3Q95":
        table, c0 = TABLE3_D3Q95, TABLE3_C
    else:
        raise ValueError(name)
    reps = tuple(r for r, _ in table)
    W, c = solve_weights(reps, [w for _, w in table], c0)
    e, group = [], []
    for g, r in enumerate(reps):
        for v in orbit(r):
            e.append(v)
            group.append(g)
    e = np.array(e, dtype=np.int64)
    group = np.array(group, dtype=np.int64)
    w = W[group]
    res = float(np.max(np.abs(formula5_residual(reps, W, c))))
    return Model(name, len(reps[0]), reps, W, float(c), e, group, w, res)


_CACHE: dict[str, Model] = {}


def get_model(name: str) -> Model:
    if name not in _CACHE:
        _CACHE[name] = build_model(name)
    return _CACHE[name]
