"""torch.autograd bindings of the projector (argument marshalling only).

``project(plan, x)`` computes y = A x with the CUDA forward kernels; its
backward is the CUDA adjoint A^T (Sec. IV-A: the adjoint of the transport is
the transport run the other way), so any objective built from it in torch,
e.g. a data fit plus a TV or learned regulariser, is differentiable end to end.
``backproject(plan, y)`` is the mirror: A^T y with backward A.

Shapes: x is [frames, n_vox] (or [n_vox] when the plan has one frame), y is
[frames, M] (or [M]); both float32 CUDA tensors.
"""
import torch

from . import lt


def _as2d(t, n):
    return t.reshape(-1, n).contiguous()


class Projector(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        ctx.shape = x.shape
        y = plan.forward(_as2d(x.float(), plan.nvox))
        return y.reshape(x.shape[:-1] + (plan.m_total,)) if x.dim() > 1 else y.reshape(-1)

    @staticmethod
    def backward(ctx, gy):
        plan = ctx.plan
        gx = plan.adjoint(_as2d(gy.float(), plan.m_total))
        return gx.reshape(ctx.shape), None


class Backprojector(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, plan):
        ctx.plan = plan
        ctx.shape = y.shape
        x = plan.adjoint(_as2d(y.float(), plan.m_total))
        return x.reshape(y.shape[:-1] + (plan.nvox,)) if y.dim() > 1 else x.reshape(-1)

    @staticmethod
    def backward(ctx, gx):
        plan = ctx.plan
        gy = plan.forward(_as2d(gx.float(), plan.nvox))
        return gy.reshape(ctx.shape), None


def project(plan, x):
    """y = A x, differentiable (backward = A^T)."""
    return Projector.apply(x, plan)


def backproject(plan, y):
    """x = A^T y, differentiable (backward = A)."""
    return Backprojector.apply(y, plan)
