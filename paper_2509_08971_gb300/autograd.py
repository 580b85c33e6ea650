"""Differentiable rollouts through the CUDA forward and adjoint kernels.

`HydroRollout.apply(U0, gamma, mesh, dts, every)` advances U0 by len(dts)
Heun steps with the given (recorded) time steps and is differentiable with
respect to U0 and gamma.  The dt schedule is a constant of the derivative:
record it once with `schedule` and reuse it, so that finite differences and
the adjoint see the same steps.

Memory: the forward pass keeps a checkpoint every `every` steps.  The
backward pass re-runs each segment from its checkpoint (keeping that
segment's states) and then applies hard_hydro_step_backward step by step in
reverse, accumulating dL/dU and dL/dgamma.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import HardHydro


@dataclass(frozen=True)
class Mesh:
    shape: tuple                    # (nz, ny, nx)
    bc: object = 0                  # one kind or six (x-, x+, y-, y+, z-, z+)
    extent: tuple = (1.0, 1.0, 1.0)


def _handle(mesh: Mesh, gamma: float, dtype):
    return HardHydro(mesh.shape, gamma, mesh.bc, dtype=dtype, extent=mesh.extent)


def schedule(U0, gamma, mesh: Mesh, nsteps: int, cfl: float):
    """The CFL time steps of a forward rollout (host list of floats)."""
    m = _handle(mesh, float(gamma), U0.dtype)
    U = U0.detach().clone()
    dts = []
    for _ in range(nsteps):
        dt = m.cfl_dt(U, cfl)
        dts.append(dt)
        U = m.step(U, dt)
    return dts


class HydroRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, gamma, mesh: Mesh, dts, every: int = 20):
        m = _handle(mesh, float(gamma), U0.dtype)
        U = U0.detach().contiguous().clone()
        ckpts = [U.clone()]
        for i, dt in enumerate(dts):
            U = m.step(U, dt)
            if (i + 1) % every == 0 and i + 1 < len(dts):
                ckpts.append(U.clone())
        ctx.m, ctx.dts, ctx.every, ctx.ckpts = m, list(dts), every, ckpts
        ctx.gamma_dtype = gamma.dtype if torch.is_tensor(gamma) else torch.float64
        return U

    @staticmethod
    def backward(ctx, gU):
        m, dts, every = ctx.m, ctx.dts, ctx.every
        g = gU.contiguous().clone()
        g_gamma = torch.zeros((), dtype=torch.float64, device=gU.device)
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * every
            stop = min(len(dts), start + every)
            states = [ctx.ckpts[seg]]
            for i in range(start, stop - 1):
                states.append(m.step(states[-1], dts[i]))
            for i in reversed(range(start, stop)):
                m.step_backward(states[i - start], g, dts[i], g_gamma, out=g)
        return g, g_gamma.to(ctx.gamma_dtype), None, None, None


def rollout(U0, gamma, mesh: Mesh, dts, every: int = 20):
    if not torch.is_tensor(gamma):
        gamma = torch.tensor(float(gamma), dtype=torch.float64, device=U0.device)
    return HydroRollout.apply(U0, gamma, mesh, dts, every)
