"""Differentiable fixed-dt Strang-step sequences (torch.autograd).

The paper has no adjoint; this is the library's differentiation pattern.  The
forward pass runs ``nsteps`` Strang steps S^dt (Algorithm 3) through the C ABI
and keeps a checkpoint of the packed state every ``checkpoint_every`` steps.
The backward pass walks the checkpoints in reverse: for each segment,
``mhd_adjoint_segment`` recomputes the segment once from its checkpoint,
recording every stage state in device memory, and applies the hand-written
step adjoints from the last step of the segment to the first.  All arithmetic
runs in the library's CUDA kernels; torch provides device memory and the
autograd graph.

The derivative is taken at the fixed ``dt``; enabled stabilisation maps are
differentiated with their coefficients frozen at the recomputed forward
values (see ``mhd_adjoint_step``).
"""
from __future__ import annotations

import torch

from .mhd import Solver


class StrangSteps(torch.autograd.Function):
    """x_T = (S^dt)^nsteps (x_0) on the packed state vector of ``solver``."""

    @staticmethod
    def forward(ctx, x0, solver: Solver, dt: float, nsteps: int, checkpoint_every: int):
        if not x0.is_cuda or x0.dtype != torch.float64:
            raise ValueError("x0 must be a CUDA float64 tensor")
        x = x0.detach().contiguous().clone()
        torch.cuda.current_stream().synchronize()  # the library works on its own stream
        ckpts = []
        done = 0
        while done < nsteps:
            m = min(checkpoint_every, nsteps - done)
            ckpts.append(x.clone())
            solver.set_packed(x)
            solver.strang_steps(dt, m)
            solver.get_packed(x)
            done += m
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every = solver, float(dt), int(nsteps), int(checkpoint_every)
        ctx.ckpts = ckpts
        return x

    @staticmethod
    def backward(ctx, lam):
        solver, dt, every = ctx.solver, ctx.dt, ctx.every
        lam = lam.detach().contiguous().clone()
        torch.cuda.current_stream().synchronize()
        for si in reversed(range(len(ctx.ckpts))):
            m = min(every, ctx.nsteps - si * every)
            solver.adjoint_segment(ctx.ckpts[si], m, lam, dt, out=lam)
        ctx.ckpts = None
        return lam, None, None, None, None


def strang_steps(solver: Solver, x0: torch.Tensor, dt: float, nsteps: int, checkpoint_every: int = 20):
    """Differentiable ``nsteps`` Strang steps of size ``dt`` from the packed
    state ``x0`` (CUDA float64 tensor of length ``solver.state_size()``)."""
    return StrangSteps.apply(x0, solver, dt, nsteps, checkpoint_every)


def pack_primitive(rho, u, p, gamma, B):
    """Packed state from nodal primitives (differentiable torch ops): U = (rho,
    rho u, p/(gamma-1) + rho |u|^2/2) followed by the magnetic part ``B``
    (the packed tail [Bx | By | Bz], not differentiated through here)."""
    m = rho * u
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u).sum(dim=0)
    return torch.cat([rho, m[0], m[1], m[2], E, B])
