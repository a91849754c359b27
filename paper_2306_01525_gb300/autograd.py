"""Differentiable meshless-LBM rollout with sqrt(T) step checkpointing.

``rollout(w, tau, g, rho0, ux0, uy0, nsteps)`` runs ``nsteps`` fused steps from the equilibrium
initial state of the fields (rho0, ux0, uy0) and returns the macroscopic fields of the final
level (rho, ux, uy; FP64, original node order).  Its backward pass gives the gradients with
respect to the relaxation time tau, the body-force magnitude g and the three initial fields,
through the library's adjoint kernels (mlbm_moments_adjoint, mlbm_adjoint_step,
mlbm_init_adjoint).  Only every ``checkpoint``-th state (default ceil(sqrt(nsteps))) is kept
during the forward pass; the backward pass recomputes each segment of states from its
checkpoint and sweeps it in reverse.  One segment (nseg == 1) per weights object, either
stencil rule; each reverse step gets the forward's next state, and under the nearest-node rule
it needs |1 - 1/tau| >= 1/16 (near tau = 1 the interpolated populations cannot be recovered
from that state, and only the own-node rule can recompute them), else the backward pass raises
MLBMError.
"""
from __future__ import annotations

import math

import torch

from . import F32, F64, adjoint_step, init, init_adjoint, moments, moments_adjoint, run, step


def _zeros_state(w, dtype, device):
    return torch.zeros(9 * w.n, dtype=torch.float32 if dtype == F32 else torch.float64,
                       device=device)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, g, rho0, ux0, uy0, w, dtype, nsteps, checkpoint, rho_ref):
        if w.nseg != 1:
            raise ValueError("rollout supports one segment per weights object")
        params = [(float(tau.item()), float(g.item()), float(rho_ref))]
        dev = rho0.device
        s = _zeros_state(w, dtype, dev)
        init(w, params, dtype, rho0.contiguous(), ux0.contiguous(), uy0.contiguous(), s)
        ckpts = []
        nxt = torch.empty_like(s)
        for n0 in range(0, nsteps, checkpoint):
            ckpts.append(s.clone())
            # the segment's steps in one library call (graph-captured step loop)
            if run(w, params, dtype, s, nxt, min(checkpoint, nsteps - n0)) is nxt:
                s, nxt = nxt, s
        rho, ux, uy = moments(w, params, dtype, s)
        ctx.w, ctx.dtype, ctx.nsteps, ctx.checkpoint = w, dtype, nsteps, checkpoint
        ctx.params = params
        ctx.ckpts = ckpts
        ctx.final = s
        ctx.save_for_backward(rho0, ux0, uy0)
        return rho, ux, uy

    @staticmethod
    def backward(ctx, drho, dux, duy):
        w, dtype, T, C, params = ctx.w, ctx.dtype, ctx.nsteps, ctx.checkpoint, ctx.params
        rho0, ux0, uy0 = ctx.saved_tensors
        dev = rho0.device
        z = lambda t: torch.zeros(w.n, dtype=torch.float64, device=dev) if t is None else t.contiguous().to(torch.float64)
        grad = torch.zeros(2, dtype=torch.float64, device=dev)
        lam = _zeros_state(w, dtype, dev)
        moments_adjoint(w, params, dtype, ctx.final, z(drho), z(dux), z(duy), lam, grad)
        lam_prev = torch.empty_like(lam)
        nseg = len(ctx.ckpts)
        after = ctx.final  # the state that follows the segment being swept
        for c in reversed(range(nseg)):
            n0 = c * C
            n1 = min(T, n0 + C)
            states = [ctx.ckpts[c]]
            for n in range(n0, n1 - 1):
                nxt = torch.empty_like(states[-1])
                step(w, params, dtype, states[-1], nxt)
                states.append(nxt)
            states.append(after)
            for n in reversed(range(n0, n1)):
                adjoint_step(w, params, dtype, states[n - n0], lam, lam_prev, grad,
                             s_next=states[n - n0 + 1])
                lam, lam_prev = lam_prev, lam
            after = states[0]
            ctx.ckpts[c] = None
            del states
        ctx.final = None
        d0 = [torch.empty(w.n, dtype=torch.float64, device=dev) for _ in range(3)]
        init_adjoint(w, params, dtype, rho0.contiguous(), ux0.contiguous(), uy0.contiguous(), lam,
                     d0[0], d0[1], d0[2], grad)
        gt = grad[0].to(torch.float64)
        gg = grad[1].to(torch.float64)
        return gt, gg, d0[0], d0[1], d0[2], None, None, None, None, None


def rollout(w, tau, g, rho0, ux0, uy0, nsteps: int, dtype=F64, checkpoint: int | None = None,
            rho_ref: float = 1.0):
    """Final-level (rho, ux, uy) after nsteps steps; differentiable in tau, g and the initial
    fields (tau and g are 0-d float64 tensors on the device)."""
    if checkpoint is None:
        checkpoint = max(1, int(math.ceil(math.sqrt(max(1, nsteps)))))
    return _Rollout.apply(tau, g, rho0, ux0, uy0, w, dtype, int(nsteps), int(checkpoint),
                          float(rho_ref))
