"""torch.autograd wrappers of the projector pair.

``project(vol, plan)`` returns H vol; its backward applies the hand-written adjoint kernel
(H^T grad).  ``backproject(data, plan)`` returns H^T data; its backward applies H.  Because
oat_backproject is the exact transpose of oat_project (same lattice points, same weights,
D^T the exact transpose of D), these are the true gradients of the discrete model
(Sec. II.B, "Adjoints of the system matrices").
"""
from __future__ import annotations

import torch


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol, plan):
        ctx.plan = plan
        return plan.project(vol.contiguous())

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        g = grad.contiguous()
        if g.dtype != plan.torch_data_dtype:
            g = g.to(plan.torch_data_dtype)
        return plan.backproject(g), None


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, data, plan):
        ctx.plan = plan
        d = data.contiguous()
        if d.dtype != plan.torch_data_dtype:
            d = d.to(plan.torch_data_dtype)
        return plan.backproject(d)

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        out = plan.project(grad.contiguous().float())
        return out.to(torch.float32), None


def project(vol: torch.Tensor, plan) -> torch.Tensor:
    """u = H vol (differentiable; d/dvol is the adjoint kernel)."""
    return _Project.apply(vol, plan)


def backproject(data: torch.Tensor, plan) -> torch.Tensor:
    """vol = H^T data (differentiable; d/ddata is the projector)."""
    return _Backproject.apply(data, plan)
