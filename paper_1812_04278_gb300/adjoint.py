"""Gradient of a rollout misfit with respect to the initial density,
velocity and edge vector potential (so that b = curl A + B0 stays
divergence free), computed by libw5ct's adjoint kernels.

`RolloutMisfit` is a torch.autograd.Function: the forward pass builds the
initial state on the device (w5ct_ic_from_potential), advances it nsteps
steps of fixed dt and evaluates L = 1/2 dV |state - target|^2
(w5ct_misfit), keeping the state at the start of every step (per-step
checkpoints).  The backward pass restores each checkpoint in reverse order
and calls w5ct_adjoint_step, which recomputes that step's stages and runs
them backwards, then maps the adjoint of the initial state onto (rho, v, A)
(w5ct_ic_from_potential_adjoint).  Only argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import w5ct as w5


class RolloutMisfit(torch.autograd.Function):
    """L(rho, v, A) for a Solver of one patch; P, B0, the target, dt and
    the step count are fixed.  rho: (nz, ny, nx); v, A: (3, nz, ny, nx);
    float64 CUDA tensors."""

    @staticmethod
    def forward(fctx, rho, v, A, solver, P, B0, target_cons, target_bface, dt, nsteps):
        rho, v, A, P = (t.contiguous() for t in (rho, v, A, P))
        shape = solver.shape
        grid = rho.shape
        cons = torch.empty((5,) + grid, dtype=torch.float64, device=rho.device)
        bface = torch.empty((3,) + grid, dtype=torch.float64, device=rho.device)
        stream = torch.cuda.current_stream().cuda_stream
        w5.w5ct_ic_from_potential(shape, solver.dx, solver.cfg.gamma, B0, rho, v, P, A, cons, bface, stream)
        solver.set_state(cons, bface)
        ckq = torch.empty((nsteps, 5) + grid, dtype=torch.float64, device=rho.device)
        ckb = torch.empty((nsteps, 3) + grid, dtype=torch.float64, device=rho.device)
        for k in range(nsteps):
            w5.w5ct_get_state(solver.ctx, ckq[k], ckb[k], None, 1)
            solver.step(dt)
        lam_q = torch.empty_like(cons)
        lam_b = torch.empty_like(bface)
        L = w5.w5ct_misfit(solver.ctx, target_cons.contiguous(), target_bface.contiguous(), lam_q, lam_b)
        fctx.solver, fctx.dt, fctx.nsteps = solver, float(dt), int(nsteps)
        fctx.save_for_backward(rho, v, bface, ckq, ckb, lam_q, lam_b)
        return torch.tensor(L, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(fctx, gL):
        rho, v, bface, ckq, ckb, lam_q, lam_b = fctx.saved_tensors
        solver = fctx.solver
        g = float(gL)
        lq = lam_q if g == 1.0 else lam_q * g
        lb = lam_b if g == 1.0 else lam_b * g
        oq, ob = torch.empty_like(lq), torch.empty_like(lb)
        for k in reversed(range(fctx.nsteps)):
            solver.set_state(ckq[k], ckb[k])          # recompute from the checkpoint
            w5.w5ct_adjoint_step(solver.ctx, fctx.dt, lq, lb, oq, ob)
            lq, oq = oq, lq
            lb, ob = ob, lb
        lam_rho = torch.empty_like(rho)
        lam_v = torch.empty_like(v)
        lam_A = torch.empty_like(v)
        lam_bt = torch.empty_like(bface)
        w5.w5ct_ic_from_potential_adjoint(solver.shape, solver.dx, rho, v, bface, lq, lb, lam_rho, lam_v, lam_A,
                                          lam_bt, torch.cuda.current_stream().cuda_stream)
        return lam_rho, lam_v, lam_A, None, None, None, None, None, None, None


def rollout_misfit(rho, v, A, solver, P, B0, target_cons, target_bface, dt, nsteps):
    """L(rho, v, A); differentiable in rho, v and A."""
    return RolloutMisfit.apply(rho, v, A, solver, P, B0, target_cons, target_bface, dt, nsteps)


def rollout_value(rho, v, A, solver, P, B0, target_cons, target_bface, dt, nsteps) -> float:
    """L without checkpoints (for finite differences)."""
    grid = rho.shape
    cons = torch.empty((5,) + grid, dtype=torch.float64, device=rho.device)
    bface = torch.empty((3,) + grid, dtype=torch.float64, device=rho.device)
    w5.w5ct_ic_from_potential(solver.shape, solver.dx, solver.cfg.gamma, B0, rho.contiguous(), v.contiguous(),
                              P.contiguous(), A.contiguous(), cons, bface, torch.cuda.current_stream().cuda_stream)
    solver.set_state(cons, bface)
    for _ in range(nsteps):
        solver.step(dt)
    lq, lb = torch.empty_like(cons), torch.empty_like(bface)
    return w5.w5ct_misfit(solver.ctx, target_cons.contiguous(), target_bface.contiguous(), lq, lb)
