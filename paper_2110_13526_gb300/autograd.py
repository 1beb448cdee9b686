"""Differentiable projector pair: ``ct_project`` and ``ct_backproject`` as
``torch.autograd.Function``s.

The operator is linear, so the vector-Jacobian product of ``y = A x`` is
``A^T g`` and that of ``x = A^T y`` is ``A g``: each Function's backward is
the other hand-written CUDA kernel (exact FP32 transposes of each other, see
``ct_backproject``).  Inputs may carry leading batch dimensions; all items
share the geometry and go through ``ct_project_batch`` / ``ct_backproject_batch``:
one projector launch for the whole batch (column-major Siddon geometries).

``unrolled_cgls`` composes them into K iterations of Algorithm 1 that autograd
can differentiate with respect to the data ``b`` (and ``x0``).  The operator
calls run in the library's kernels; the few scalar/vector updates between
them are plain tensor arithmetic so that autograd can trace them, and each
iteration is activation-checkpointed.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import Geometry, backproject_batch, project_batch


class ProjectFn(torch.autograd.Function):
    """y = A x (ct_project); backward: grad_x = A^T grad_y (ct_backproject)."""

    @staticmethod
    def forward(ctx, x, g):
        ctx.g = g
        return project_batch(g, x.detach())

    @staticmethod
    def backward(ctx, gy):
        g = ctx.g
        return backproject_batch(g, gy.contiguous()), None


class BackprojectFn(torch.autograd.Function):
    """x = A^T y (ct_backproject); backward: grad_y = A grad_x (ct_project)."""

    @staticmethod
    def forward(ctx, y, g):
        ctx.g = g
        return backproject_batch(g, y.detach())

    @staticmethod
    def backward(ctx, gx):
        g = ctx.g
        return project_batch(g, gx.contiguous()), None


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
