"""Differentiable MPDATA rollouts: gradients of a final-state loss with respect to
the initial field psi0 and the advector components GC.

Forward: n_steps steps through the C ABI (fused kernels where they apply),
keeping psi every `checkpoint_every` steps on the device.  Backward: for each
segment, last first, the states inside the segment are recomputed from its
checkpoint, then the hand-written adjoint kernels (mpdata_adjoint_step) walk
the segment backwards, accumulating dL/dGC over all steps.  Memory is one
field per checkpoint plus one segment of states.
"""
from __future__ import annotations

import torch

from .solver import Mpdata


class MPDATAFunction(torch.autograd.Function):
    """psi_T = MPDATA^n_steps(psi0; GC).  Use as
    ``MPDATAFunction.apply(solver, n_steps, checkpoint_every, psi0, *gc)``."""

    @staticmethod
    def forward(ctx, solver: Mpdata, n_steps: int, checkpoint_every: int, psi0, *gc):
        if n_steps < 1 or checkpoint_every < 1:
            raise ValueError("n_steps and checkpoint_every must be >= 1")
        cur = psi0.detach().contiguous().clone()
        nxt = torch.empty_like(cur)
        gcd = [g.detach().contiguous() for g in gc]
        ckpts = [cur.clone()]
        for s in range(n_steps):
            solver.advance(cur, nxt, gcd)
            cur, nxt = nxt, cur
            if (s + 1) % checkpoint_every == 0 and s + 1 < n_steps:
                ckpts.append(cur.clone())
        ctx.solver = solver
        ctx.n_steps = n_steps
        ctx.every = checkpoint_every
        ctx.n_gc = len(gc)
        ctx.save_for_backward(*ckpts, *gcd)
        return cur

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        n_ck = len(saved) - ctx.n_gc
        ckpts, gc = list(saved[:n_ck]), list(saved[n_ck:])
        solver, n, every = ctx.solver, ctx.n_steps, ctx.every
        pb = grad_out.detach().contiguous().clone()
        gcb = [torch.zeros_like(g) for g in gc]
        for seg in range(n_ck - 1, -1, -1):
            start, end = seg * every, min(seg * every + every, n)
            states = [ckpts[seg]]
            for _ in range(start, end - 1):
                nxt = torch.empty_like(states[-1])
                solver.advance(states[-1], nxt, gc)
                states.append(nxt)
            for s in range(end - 1, start - 1, -1):
                solver.adjoint_step(states[s - start], gc, pb, gc_bar=gcb)
        return (None, None, None, pb, *gcb)


def rollout(solver: Mpdata, psi0, gc, n_steps: int, checkpoint_every: int = 20):
    """Differentiable n-step rollout (see MPDATAFunction)."""
    return MPDATAFunction.apply(solver, n_steps, checkpoint_every, psi0, *gc)
