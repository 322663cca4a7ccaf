"""A whole differentiable rollout as one torch.autograd.Function (Section III: gradients of the
final state with respect to the initial state and to the controller parameters used at every
step).

The forward runs the rollout in libgbmpm, which stores only every k-th state (k from the memory
budget when not given); the backward runs the library's reverse pass, which recomputes each
segment's states from its checkpoint and applies the supplement's adjoint steps.  torch supplies
device memory and the stream; every step of both passes runs in the library's kernels.

    x_T, v_T, C_T, F_T = rollout(scene, n_steps, x0, v0, C0, F0, params)
    loss = x_T[:, 0].mean(); loss.backward()   # fills x0.grad, v0.grad, ..., params.grad
"""
from __future__ import annotations

import torch

from . import mpm


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scene, n_steps, ckpt_interval, mem_budget, x0, v0, C0, F0, params):
        dev = x0.device
        N, d = scene.N, scene.dim
        scene.set_params(params.detach())
        scene.set_state(x0.detach(), v0.detach(), C0.detach(), F0.detach(), step=0)
        scene.rollout(int(n_steps), int(ckpt_interval), int(mem_budget))
        xT = torch.empty((N, d), device=dev)
        vT = torch.empty((N, d), device=dev)
        CT = torch.empty((N, d, d), device=dev)
        FT = torch.empty((N, d, d), device=dev)
        scene.get_state(out=(xT, vT, CT, FT))
        ctx.scene = scene
        ctx.generation = scene.generation
        ctx.n_params = params.numel()
        ctx.dev = dev
        return xT, vT, CT, FT

    @staticmethod
    def backward(ctx, gxT, gvT, gCT, gFT):
        scene = ctx.scene
        if scene.generation != ctx.generation:
            # the library differentiates the scene's latest rollout, not the one this graph recorded
            raise RuntimeError("the scene was rolled out, stepped or changed again after this rollout's forward; "
                               "run backward before reusing the scene, or give each rollout its own scene")
        N, d, dev = scene.N, scene.dim, ctx.dev
        seeds = [None if g is None else g.contiguous().to(dev, torch.float32) for g in (gxT, gvT, gCT, gFT)]
        outs = (torch.empty((N, d), device=dev), torch.empty((N, d), device=dev),
                torch.empty((N, d, d), device=dev), torch.empty((N, d, d), device=dev),
                torch.empty((max(ctx.n_params, 1),), device=dev))
        scene.backward(*seeds, out=outs)
        gx0, gv0, gC0, gF0, gp = outs
        return None, None, None, None, gx0, gv0, gC0, gF0, gp[: ctx.n_params]


def rollout(scene, n_steps, x0, v0, C0, F0, params, ckpt_interval: int = 0, mem_budget: int = 0):
    """Differentiable rollout of ``scene`` (a mpm.Scene on the tensors' device) for n_steps."""
    return Rollout.apply(scene, n_steps, ckpt_interval, mem_budget, x0, v0, C0, F0, params)
