"""torch.autograd wrappers of the FSI cycle and of checkpointed rollouts.

The forward passes call ``fsi_step`` and the backward passes the hand-written adjoint
``fsi_step_vjp`` of the CUDA library; no arithmetic of the method runs here.  Rollouts
keep the state every ``ckpt_every`` steps and recompute each segment during the backward
pass with ``fsi_step_record``, keeping every cycle's input state and intermediates
(a(x0), a(x1), G(x1)) for ``fsi_step_vjp_rec`` (memory O(steps / ckpt_every + ckpt_every)
states).
"""
from __future__ import annotations

import torch

from . import fsi as F


class FSIStep(torch.autograd.Function):
    """(pos, vel) -> state after one FSI cycle of step h; differentiable in pos, vel, mass."""

    @staticmethod
    def forward(ctx, pos, vel, mass, h, fctx):
        p, v = pos.detach().clone(), vel.detach().clone()
        F.fsi_step(fctx, p, v, mass.detach(), h, nsteps=1)
        ctx.save_for_backward(pos.detach(), vel.detach(), mass.detach())
        ctx.h, ctx.fctx = h, fctx
        return p, v

    @staticmethod
    def backward(ctx, gx, gv):
        pos, vel, mass = ctx.saved_tensors
        gx = torch.zeros_like(pos) if gx is None else gx.contiguous()
        gv = torch.zeros_like(vel) if gv is None else gv.contiguous()
        gxi, gvi, gm = F.fsi_step_vjp(ctx.fctx, pos, vel, mass, ctx.h, gx, gv)
        return gxi, gvi, gm, None, None


class FSIRollout(torch.autograd.Function):
    """`steps` FSI cycles with step checkpointing every `ckpt_every` cycles."""

    @staticmethod
    def forward(ctx, pos, vel, mass, h, steps, ckpt_every, fctx):
        p, v = pos.detach().clone(), vel.detach().clone()
        m = mass.detach()
        ckpts = []
        done = 0
        while done < steps:
            ckpts.append((p.clone(), v.clone()))
            k = min(ckpt_every, steps - done)
            for _ in range(k):
                F.fsi_step(fctx, p, v, m, h, nsteps=1)
            done += k
        ctx.ckpts, ctx.m, ctx.h, ctx.steps, ctx.every, ctx.fctx = ckpts, m, h, steps, ckpt_every, fctx
        return p, v

    @staticmethod
    def backward(ctx, gx, gv):
        m, h, fctx = ctx.m, ctx.h, ctx.fctx
        gx = torch.zeros_like(ctx.ckpts[0][0]) if gx is None else gx.contiguous().clone()
        gv = torch.zeros_like(ctx.ckpts[0][1]) if gv is None else gv.contiguous().clone()
        gm = torch.zeros_like(m)
        for s in range(len(ctx.ckpts) - 1, -1, -1):
            p, v = ctx.ckpts[s][0].clone(), ctx.ckpts[s][1].clone()
            k = min(ctx.every, ctx.steps - s * ctx.every)
            states = []
            for _ in range(k):                      # recompute the segment, recording
                p0, v0 = p.clone(), v.clone()
                states.append((p0, v0, F.fsi_step_record(fctx, p, v, m, h)))
            for (p0, v0, rec) in reversed(states):
                gx, gv, gm = F.fsi_step_vjp_rec(fctx, p0, v0, m, h, rec, gx, gv, gm=gm)
        return gx, gv, gm, None, None, None, None


def fsi_rollout(fctx: F.Context, pos, vel, mass, h: float, steps: int, ckpt_every: int = 20):
    """Differentiable rollout of `steps` FSI cycles (returns final pos, vel)."""
    return FSIRollout.apply(pos, vel, mass, h, int(steps), int(ckpt_every), fctx)
