"""BGK stream-and-collide, macroscopic fields, audit and discrete adjoint (oracle).

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline; never by the product path.

The paper's lattice Boltzmann update (text before the Maxwellian) is

    f_i(x + V_i dt, t + dt) = (1 - omega) f_i(x, t) + omega f_i^eq(x, t).

Conventions of this restatement:

* lattice units, V_i = e_i (integer), Delta x = Delta t = 1;
* pull form with post-collision storage: S_{n+1}(x, i) = C_i(g(x)) with the
  gathered populations g_i(x) = S_n((x - e_i) mod N, i) and
  C_i(g) = (1 - omega) g_i + omega f_i^eq(rho, u, theta of g).
  The paper's push form stores the pre-collision populations; the two differ
  by one collision and have identical rho, U, T because the collision
  conserves them;
* periodic box, true modulo (grids smaller than the stencil reach are legal);
* state arrays are [Q, Nz, Ny, Nx] (x fastest); 2D models use Nz = 1;
* fields in lattice units: U_lat = u_xi / (sqrt(2) c), T_lat = theta * T0 with
  T0 = 1/(2 c^2) (see ``Model.T0``).

Pinned by tests: exact conservation of mass / momentum / energy, rest and
uniform-flow fixed points, an integer-label streaming permutation checked with
explicit index arithmetic, a naive per-cell brute force with a linear-solve
equilibrium on tiny grids, exact Riemann plateaus (physics), and for the
adjoint central finite differences of the whole rollout and a column-by-column
complex-step Jacobian.
"""
from __future__ import annotations

import math

import numpy as np

from .equilibrium import feq


# ------------------------------------------------------------------ unit conversion

def to_xi_units(model, U, T):
    """Lattice-unit U [D, ...] and T [...] -> unit-variance u [C, D] and theta [C]."""
    D = model.D
    s = math.sqrt(2.0) * model.c
    u = (np.asarray(U).reshape(D, -1) * s).T
    theta = np.asarray(T).reshape(-1) / model.T0
    return u, theta


def grid_shape(S):
    return S.shape[1:]


# ------------------------------------------------------------------ forward

def init_populations(model, rho, U, T):
    """S_0 = f^eq(rho, U, T) per cell; rho, T shape [Nz, Ny, Nx], U shape [D, Nz, Ny, Nx]."""
    shape = np.asarray(rho).shape
    u, theta = to_xi_units(model, U, T)
    f = feq(model, np.asarray(rho, dtype=np.float64).reshape(-1), u, theta)
    return f.reshape((model.Q,) + tuple(shape))


def shift3(e, D):
    """(ez, ey, ex) shift of lattice vector e for an array indexed [z, y, x]."""
    if D == 2:
        return (0, int(e[1]), int(e[0]))
    return (int(e[2]), int(e[1]), int(e[0]))


def stream(model, S):
    """Pull streaming: g_i(x) = S_i((x - e_i) mod N)."""
    g = np.empty_like(S)
    for i in range(model.Q):
        g[i] = np.roll(S[i], shift=shift3(model.e[i], model.D), axis=(0, 1, 2))
    return g


def collide(model, g, omega):
    """BGK collision C(g) = (1 - omega) g + omega f^eq(moments of g), per cell."""
    Q = model.Q
    gf = g.reshape(Q, -1)
    rho, u, theta = moments_of(model, gf)
    fe = feq(model, rho, u, theta)
    return ((1.0 - omega) * gf + omega * fe).reshape(g.shape)


def step(model, S, omega):
    return collide(model, stream(model, S), omega)


def run(model, S, omega, nsteps, ends=None):
    """nsteps steps; ``ends`` = (axis, width, (rho, U, T)_lo, (rho, U, T)_hi) holds
    the first and last ``width`` planes along ``axis`` at the discrete equilibrium
    of the two states after every step (see fixed_ends)."""
    for _ in range(nsteps):
        S = step(model, S, omega)
        if ends is not None:
            S = fixed_ends(model, S, *ends)
    return S


def fixed_ends(model, S, axis, width, lo, hi):
    """The shock tube's end conditions (paragraph before Figure 1): the planes
    with coordinate < width along ``axis`` take f^eq of state ``lo``, those with
    coordinate >= N - width take f^eq of ``hi``.  States are (rho, U [D], T) in
    lattice units; axis 0, 1, 2 = x, y, z.  width >= the stencil reach keeps every
    other cell's gathers inside the tube (no wrap through the ends)."""
    S = S.copy()
    arr_axis = 3 - axis                      # S is [Q, z, y, x]
    n = S.shape[arr_axis]
    for state, sl in ((lo, slice(0, width)), (hi, slice(n - width, n))):
        rho, U, T = state
        u, theta = to_xi_units(model, np.asarray(U, dtype=np.float64).reshape(model.D, 1),
                               np.array([T], dtype=np.float64))
        fe = feq(model, np.array([float(rho)]), u, theta)[:, 0]
        idx = [slice(None)] * 4
        idx[arr_axis] = sl
        shape = [model.Q, 1, 1, 1]
        S[tuple(idx)] = fe.reshape(shape)
    return S


# ------------------------------------------------------------------ moments

def raw_moments(model, f):
    """rho = sum f, j = sum f xi, E = sum f |xi|^2 for populations f [Q, C]."""
    xi = model.xi
    rho = f.sum(axis=0)
    j = xi.T @ f
    E = (xi * xi).sum(axis=1) @ f
    return rho, j, E


def fields_from_moments(model, rho, j, E):
    """(rho, u [C, D], theta) from the raw moments; theta = (E/rho - |u|^2)/D."""
    u = (j / rho).T
    theta = (E / rho - (u * u).sum(axis=1)) / model.D
    return rho, u, theta


def moments_of(model, f):
    rho, j, E = raw_moments(model, f)
    return fields_from_moments(model, rho, j, E)


def macroscopic(model, S):
    """rho [grid], U [D, grid] and T [grid] in lattice units."""
    shape = grid_shape(S)
    rho, u, theta = moments_of(model, S.reshape(model.Q, -1))
    U = (u / (math.sqrt(2.0) * model.c)).T.reshape((model.D,) + tuple(shape))
    T = (theta * model.T0).reshape(shape)
    return rho.reshape(shape), U, T


def audit(model, S):
    """Global totals in lattice units: mass, momentum [D], energy (sum f |e|^2 / 2),
    min_i f_i / w_i and the number of non-finite populations.

    The minimum runs over the numbers among the f_i / w_i (infinities included,
    NaN skipped: a NaN is reported by the non-finite count, not as a minimum)."""
    f = S.reshape(model.Q, -1)
    e = model.e.astype(np.float64)
    with np.errstate(invalid="ignore"):
        mass = float(f.sum())
        mom = (e.T @ f).sum(axis=1)
        energy = float(0.5 * ((e * e).sum(axis=1) @ f).sum())
    minratio = float(np.fmin.reduce((f / model.w[:, None]).ravel()))
    nonfinite = int((~np.isfinite(f)).sum())
    return {"mass": mass, "momentum": mom, "energy": energy,
            "min_f_over_w": minratio, "nonfinite": nonfinite}


# ------------------------------------------------------------------ adjoint

_H = 1e-30          # complex-step size (Squire & Trapp 1998): exact to roundoff


def dfeq_dmoments(model, gf):
    """d f_i^eq / d M_m for the raw moments M = (rho, j_1..j_D, E) of g [Q, C].

    Complex-step derivative of f^eq(fields_from_moments(M)); returns [D+2, Q, C].
    """
    rho, j, E = raw_moments(model, gf)
    D = model.D
    out = []
    for m in range(D + 2):
        r = rho.astype(np.complex128)
        jj = j.astype(np.complex128)
        ee = E.astype(np.complex128)
        if m == 0:
            r = r + 1j * _H
        elif m <= D:
            jj[m - 1] = jj[m - 1] + 1j * _H
        else:
            ee = ee + 1j * _H
        fr, fu, ft = fields_from_moments(model, r, jj, ee)
        out.append(feq(model, fr, fu, ft).imag / _H)
    return np.array(out)


def collide_adjoint(model, gf, lam, omega):
    """mu = J^T lam for the collision J = dC/dg at g [Q, C]; lam [Q, C].

    f^eq depends on g only through M, so
    mu_j = (1 - omega) lam_j + omega * sum_m dM_m/dg_j * sum_i lam_i df_i^eq/dM_m,
    with dM/dg_j = (1, xi_j, |xi_j|^2).
    Also returns sum lam_i (f_i^eq - g_i) per cell, the omega-derivative term.
    """
    xi = model.xi
    dF = dfeq_dmoments(model, gf)                       # [D+2, Q, C]
    Lam = np.einsum("mqc,qc->mc", dF, lam)              # [D+2, C]
    dMdg = np.concatenate([np.ones((1, model.Q)), xi.T, (xi * xi).sum(axis=1)[None]], axis=0)
    mu = (1.0 - omega) * lam + omega * (dMdg.T @ Lam)
    rho, u, theta = moments_of(model, gf)
    fe = feq(model, rho, u, theta)
    domega = (lam * (fe - gf)).sum(axis=0)
    return mu, domega


def stream_adjoint(model, mu):
    """Transpose of pull streaming: lam_i(y) = mu_i((y + e_i) mod N)."""
    out = np.empty_like(mu)
    for i in range(model.Q):
        sh = shift3(model.e[i], model.D)
        out[i] = np.roll(mu[i], shift=tuple(-k for k in sh), axis=(0, 1, 2))
    return out


def init_adjoint(model, rho0, U0, T0, lam0):
    """dL/d(rho0, U0, T0) from lam0 = dL/dS_0 through S_0 = f^eq(rho0, U0, T0).

    Each cell's populations depend only on that cell's fields, so one
    complex-step perturbation of a field across all cells gives every cell's
    derivative at once.  U0, T0 in lattice units.
    """
    shape = np.asarray(rho0).shape
    Q, D = model.Q, model.D
    lam = lam0.reshape(Q, -1)
    rho = np.asarray(rho0, dtype=np.float64).reshape(-1)
    u, theta = to_xi_units(model, U0, T0)

    def proj(r, uu, t):
        return (feq(model, r, uu, t).imag / _H * lam).sum(axis=0)

    d_rho = proj(rho + 1j * _H, u.astype(np.complex128), theta.astype(np.complex128))
    d_U = []
    s = math.sqrt(2.0) * model.c
    for a in range(D):
        uu = u.astype(np.complex128)
        uu[:, a] += 1j * _H
        d_U.append(proj(rho.astype(np.complex128), uu, theta.astype(np.complex128)) * s)
    d_T = proj(rho.astype(np.complex128), u.astype(np.complex128), theta + 1j * _H) / model.T0
    return (d_rho.reshape(shape), np.array(d_U).reshape((D,) + tuple(shape)),
            d_T.reshape(shape))


def rollout_gradients(model, rho0, U0, T0, omega, nsteps, dL_drhoN):
    """Forward nsteps from f^eq(rho0, U0, T0), then the exact discrete adjoint.

    The loss is any L(rho_N) whose gradient dL/drho_N [grid] is given; since
    rho_N = sum_i S_N(x, i), lam_N(x, i) = dL/drho_N(x) for every i.
    Returns (rho_N, dL/drho0, dL/dU0, dL/dT0, dL/domega).
    """
    Q = model.Q
    S = init_populations(model, rho0, U0, T0)
    traj = [S]
    for _ in range(nsteps):
        S = step(model, S, omega)
        traj.append(S)
    rhoN = S.sum(axis=0)
    g_rho = dL_drhoN(rhoN) if callable(dL_drhoN) else np.asarray(dL_drhoN)
    lam = np.broadcast_to(g_rho, S.shape).astype(np.float64).copy()
    d_omega = 0.0
    for n in range(nsteps - 1, -1, -1):
        g = stream(model, traj[n]).reshape(Q, -1)
        mu, dom = collide_adjoint(model, g, lam.reshape(Q, -1), omega)
        d_omega += float(dom.sum())
        lam = stream_adjoint(model, mu.reshape(S.shape))
    d_rho, d_U, d_T = init_adjoint(model, rho0, U0, T0, lam)
    return rhoN, d_rho, d_U, d_T, d_omega


def mse_loss(rhoN, target):
    """L = mean over cells of (rho_N - rho*)^2 and its gradient."""
    diff = rhoN - target
    return float((diff * diff).mean()), 2.0 * diff / diff.size
