"""x = solve(A, b) as a differentiable torch operation (adjoint method).

Forward: an lAIR hierarchy on A solves A x = b. Backward, given g = dL/dx: the
handle builds (once) a second hierarchy on A^T and solves A^T lambda = g; then
dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored pattern of A (both from
the CUDA library: lair_adjoint and lair_grad_A).
"""
from __future__ import annotations

import torch

from .lair import FGMRES, Hierarchy


class LairSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, row_ptr, col, opts, tol, max_iter):
        h = Hierarchy(row_ptr, col, vals.detach().contiguous(), **opts)
        x = torch.zeros_like(b)
        h.solve(b.detach().contiguous(), x, tol=tol, cycle=FGMRES, max_iter=max_iter, raise_on_nc=True)
        ctx.h = h
        ctx.tol, ctx.max_iter = tol, max_iter
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        lam = torch.zeros_like(g)
        ctx.h.adjoint(g.contiguous(), lam, tol=ctx.tol, cycle=FGMRES, max_iter=ctx.max_iter, raise_on_nc=True)
        grad_vals = ctx.h.grad_A(lam, x)
        return grad_vals, lam, None, None, None, None, None


def solve(row_ptr, col, vals, b, tol=1e-10, max_iter=500, **opts):
    """Differentiable solve of the CSR system (row_ptr, col, vals) x = b on the GPU."""
    return LairSolve.apply(vals, b, row_ptr, col, opts, tol, max_iter)
