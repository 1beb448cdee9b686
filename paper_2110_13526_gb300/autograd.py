"""Differentiable projector pair: ``ct_project`` and ``ct_backproject`` as
``torch.autograd.Function``s.

The operator is linear, so the vector-Jacobian product of ``y = A x`` is
``A^T g`` and that of ``x = A^T y`` is ``A g``: each Function's backward is
the other hand-written CUDA kernel (exact FP32 transposes of each other, see
``ct_backproject``).  Inputs may carry a leading batch dimension; each item is
projected with the same geometry.

``unrolled_cgls`` composes them into K iterations of Algorithm 1 that autograd
can differentiate with respect to the data ``b`` (and ``x0``).  The operator
calls run in the library's kernels; the few scalar/vector updates between
them are plain tensor arithmetic so that autograd can trace them, and each
iteration is activation-checkpointed.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import Geometry, backproject, project


def _apply(fn, g: Geometry, t: torch.Tensor, in_shape, out_shape) -> torch.Tensor:
    if tuple(t.shape[-3:]) != tuple(in_shape):
        raise ValueError("expected trailing shape %s, got %s" % (tuple(in_shape), tuple(t.shape)))
    lead = t.shape[:-3]
    flat = t.reshape((-1,) + tuple(in_shape)).contiguous()
    out = torch.empty((flat.shape[0],) + tuple(out_shape), dtype=torch.float32, device=t.device)
    for i in range(flat.shape[0]):
        fn(g, flat[i], out=out[i])
    return out.reshape(tuple(lead) + tuple(out_shape))


class ProjectFn(torch.autograd.Function):
    """y = A x (ct_project); backward: grad_x = A^T grad_y (ct_backproject)."""

    @staticmethod
    def forward(ctx, x, g):
        ctx.g = g
        return _apply(project, g, x.detach(), g.vol_shape, g.sino_shape)

    @staticmethod
    def backward(ctx, gy):
        g = ctx.g
        return _apply(backproject, g, gy.contiguous(), g.sino_shape, g.vol_shape), None


class BackprojectFn(torch.autograd.Function):
    """x = A^T y (ct_backproject); backward: grad_y = A grad_x (ct_project)."""

    @staticmethod
    def forward(ctx, y, g):
        ctx.g = g
        return _apply(backproject, g, y.detach(), g.sino_shape, g.vol_shape)

    @staticmethod
    def backward(ctx, gx):
        g = ctx.g
        return _apply(project, g, gx.contiguous(), g.vol_shape, g.sino_shape), None


def A(g: Geometry, x: torch.Tensor) -> torch.Tensor:
    return ProjectFn.apply(x, g)


def AT(g: Geometry, y: torch.Tensor) -> torch.Tensor:
    return BackprojectFn.apply(y, g)


def _dot(a, b):
    return (a.double() * b.double()).flatten(-3).sum(-1)


def _bcast(s, t):
    return s.reshape(s.shape + (1, 1, 1)).to(t.dtype)


def unrolled_cgls(g: Geometry, b: torch.Tensor, K: int = 10, x0=None,
                  use_checkpoint: bool = True) -> torch.Tensor:
    """K updates of Algorithm 1 (direction update d = r + beta d), differentiable.

    b: [..., nviews, nv, nu]; returns x: [..., nz, ny, nx].  Scalars are FP64.
    """
    x = torch.zeros(b.shape[:-3] + g.vol_shape, device=b.device) if x0 is None else x0
    e = b - A(g, x) if x0 is not None else b
    r = AT(g, e)
    d = r
    nr2 = _dot(r, r)
    p = A(g, d)
    alpha = nr2 / _dot(p, p)
    x = x + _bcast(alpha, x) * d
    e = e - _bcast(alpha, e) * p

    def step(x, e, d, nr2):
        r = AT(g, e)
        nr2n = _dot(r, r)
        beta = nr2n / nr2
        d = r + _bcast(beta, r) * d
        p = A(g, d)
        alpha = nr2n / _dot(p, p)
        return x + _bcast(alpha, x) * d, e - _bcast(alpha, e) * p, d, nr2n

    for _ in range(K - 1):
        if use_checkpoint and torch.is_grad_enabled():
            x, e, d, nr2 = checkpoint(step, x, e, d, nr2, use_reentrant=False)
        else:
            x, e, d, nr2 = step(x, e, d, nr2)
    return x
