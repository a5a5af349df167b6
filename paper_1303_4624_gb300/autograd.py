"""torch.autograd.Function over the checkpointed rollout (lbm_record / lbm_backward).

rollout(lattice, rho0, U0, T0, omega, nsteps, ckpt_every) maps the initial
fields (CUDA FP64 tensors: rho0 [Nz, Ny, Nx], U0 [D, Nz, Ny, Nx], T0 [Nz, Ny, Nx],
lattice units) and the relaxation frequency to the density after nsteps.  The
forward records every ckpt_every-th state; the backward runs the hand-written
adjoint kernels through the C ABI.  No arithmetic happens in Python.
"""
from __future__ import annotations

import torch

from . import lbm as _lbm


class LBMRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, U0, T0, omega, lattice, nsteps, ckpt_every):
        for t in (rho0, U0, T0):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("rho0, U0, T0 must be contiguous CUDA float64 tensors")
        h = lattice.ctx
        _lbm.lbm_set_omega(h, float(omega))
        _lbm.lbm_init(h, rho0, U0, T0)
        _lbm.lbm_record(h, nsteps, ckpt_every)
        rhoN = torch.empty_like(rho0)
        _lbm.lbm_moments(h, rhoN, None, None)
        ctx.lattice = lattice
        ctx.omega_like = omega
        return rhoN

    @staticmethod
    def backward(ctx, grad_rhoN):
        lat = ctx.lattice
        g = grad_rhoN.contiguous().to(torch.float64)
        D = lat.info["D"]
        d_rho = torch.empty_like(g)
        d_U = torch.empty((D,) + tuple(g.shape), dtype=torch.float64, device=g.device)
        d_T = torch.empty_like(g)
        d_om = _lbm.lbm_backward(lat.ctx, g, d_rho, d_U, d_T)
        om = ctx.omega_like
        d_omega = torch.tensor(d_om, dtype=om.dtype, device=om.device) if torch.is_tensor(om) else None
        return d_rho, d_U, d_T, d_omega, None, None, None


def rollout(lattice, rho0, U0, T0, omega, nsteps, ckpt_every):
    """Density after nsteps from (rho0, U0, T0) with relaxation omega (differentiable)."""
    return LBMRollout.apply(rho0, U0, T0, omega, lattice, nsteps, ckpt_every)
