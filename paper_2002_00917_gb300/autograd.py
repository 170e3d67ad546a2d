"""Differentiable PSLR-preconditioned solve: u = solve(A(theta), b).

Forward: set up PSLR for A (host set-up, device factors), build the low-rank
term and solve A u = b with FGMRES preconditioned by Algorithm 3.
Backward: the adjoint solve A^T lambda = dL/du with FGMRES preconditioned by
the exact transpose of Algorithm 3 (pslr_apply_T), then dL/db = lambda and
dL/da_ij = -lambda_i u_j on A's sparsity pattern (pslr_grad_values).  Every
solve and the gradient run in the library's kernels; this module only wires
them into torch.autograd.  The chain rule from the values of A to whatever
parameterises them (e.g. a coefficient field kappa) is ordinary torch
autograd through the user's assembly of the values.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pslr


class _CSRPattern:
    def __init__(self, n, rowptr, col, val):
        self.n = n
        self.rowptr = rowptr
        self.col = col
        self.val = val


class PslrSolveFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, rowptr, col, opts):
        n = b.shape[0]
        A = _CSRPattern(n, rowptr, col, vals.detach().double().cpu().numpy())
        p = pslr.Pslr(A, dims=opts["dims"], splits=opts["splits"], factor=opts.get("factor", 0),
                      seed=opts.get("seed", 0))
        p.build_lowrank(opts.get("m", 3), opts.get("rank", 16))
        u = torch.empty_like(b)
        its, rel, st = p.solve(b.contiguous(), u, rtol=opts.get("rtol", 1e-12),
                               restart=opts.get("restart", 60), maxit=opts.get("maxit", 2000))
        if st != pslr.PSLR_OK:
            raise pslr.PslrError(st, f"forward solve did not converge (relres {rel:.2e})")
        ctx.p = p
        ctx.opts = opts
        ctx.nnz = vals.shape[0]
        ctx.save_for_backward(u)
        ctx.info = {"iters": its, "relres": rel}
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        p, opts = ctx.p, ctx.opts
        lam = torch.empty_like(u)
        its, rel, st = p.solve(gu.contiguous().double(), lam, rtol=opts.get("rtol", 1e-12),
                               restart=opts.get("restart", 60), maxit=opts.get("maxit", 2000),
                               transpose=True)
        if st != pslr.PSLR_OK:
            raise pslr.PslrError(st, f"adjoint solve did not converge (relres {rel:.2e})")
        gvals = torch.empty(ctx.nnz, dtype=torch.float64, device=u.device)
        p.grad_values(lam, u, gvals)
        return gvals, lam, None, None, None


def solve(vals, b, rowptr, col, **opts):
    """u = A^{-1} b for the CSR matrix (rowptr, col, vals), differentiable in
    vals and b.  opts: dims, splits (geometric split), factor, m, rank, seed,
    rtol, restart, maxit."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return PslrSolveFunction.apply(vals, b, rowptr, col, opts)
