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


class PackPrimitive(torch.autograd.Function):
    """Packed state [U | B] from nodal primitives (rho, u, p) and the packed
    magnetic tail B; the exchange U(rho, u, p) and its vector-Jacobian product
    run in the library (mhd_primitive_to_conservative and its _vjp)."""

    @staticmethod
    def forward(ctx, rho, u, p, B, solver: Solver):
        for t in (rho, u, p, B):
            if not t.is_cuda or t.dtype != torch.float64:
                raise ValueError("rho, u, p and B must be CUDA float64 tensors")
        rho, u, p = rho.detach().contiguous(), u.detach().contiguous(), p.detach().contiguous()
        N = solver.N
        x = torch.empty(5 * N + B.numel(), dtype=torch.float64, device=rho.device)
        torch.cuda.current_stream().synchronize()  # the library works on its own stream
        solver.primitive_to_conservative(rho, u, p, x[:5 * N])
        x[5 * N:] = B.detach()
        ctx.save_for_backward(rho, u)
        ctx.solver = solver
        return x

    @staticmethod
    def backward(ctx, lam):
        rho, u = ctx.saved_tensors
        solver, N = ctx.solver, ctx.solver.N
        lam = lam.detach().contiguous()
        g_rho, g_u, g_p = torch.empty_like(rho), torch.empty_like(u), torch.empty_like(rho)
        torch.cuda.current_stream().synchronize()
        solver.primitive_to_conservative_vjp(rho, u, lam[:5 * N].contiguous(), g_rho, g_u, g_p)
        return g_rho, g_u, g_p, lam[5 * N:].clone(), None


def pack_primitive(solver: Solver, rho, u, p, B):
    """Differentiable packed state from nodal primitives rho [N], u [3, N],
    p [N] (CUDA float64) and the packed magnetic tail ``B`` = [Bx | By | Bz]:
    U = (rho, rho u, p/(gamma-1) + rho |u|^2/2), computed by the library."""
    return PackPrimitive.apply(rho, u, p, B, solver)
