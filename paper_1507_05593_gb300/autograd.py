"""torch.autograd.Function for x = A^{-1} b with A given by its CSR values.

Forward: new values into the handle from the device (rsc_refactor_values_device, no host
copy), rsc_factor(tol), PCG (rsc_solve_device).  Backward: the adjoint system A lambda = dL/dx is solved by PCG
with the factor kept from the forward pass (no refactorization), then
dL/dA_e = -lambda_i x_j over A's stored pattern (rsc_pattern_outer_device) and
dL/db = lambda.  Chaining dL/dA to parameters theta is torch autograd on the caller's
differentiable value function vals(theta).

Argument marshalling only: the factorization, both solves and the pattern
contraction run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import (Handle, rsc_factor, rsc_pattern_outer_device, rsc_refactor_values, rsc_refactor_values_device,
               rsc_solve_device)


class SparseSPDSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals: torch.Tensor, b: torch.Tensor, handle: Handle, tol: float, rtol: float,
                max_iter: int):
        v = vals.detach().to(torch.float64).contiguous()
        bb = b.detach().to(torch.float64).contiguous()
        x = torch.empty_like(bb)
        if v.is_cuda:   # values read on the caller's stream, no host round trip
            s = torch.cuda.current_stream(v.device)
            rsc_refactor_values_device(handle, v, stream=s)
        else:
            s = torch.cuda.current_stream(bb.device)
            rsc_refactor_values(handle, v.numpy())
        rsc_factor(handle, tol)
        it, rr = rsc_solve_device(handle, bb, x, rtol, max_iter, stream=s)
        ctx.save_for_backward(x)
        ctx.handle, ctx.rtol, ctx.max_iter, ctx.nnz = handle, rtol, max_iter, vals.numel()
        ctx.iters = it
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        g = gx.to(torch.float64).contiguous()
        lam = torch.empty_like(x)
        gvals = torch.empty(ctx.nnz, dtype=torch.float64, device=x.device)
        s = torch.cuda.current_stream(x.device)   # the library's calls run on the caller's stream
        rsc_solve_device(ctx.handle, g, lam, ctx.rtol, ctx.max_iter, stream=s)   # adjoint solve, factor kept
        rsc_pattern_outer_device(ctx.handle, lam, x, -1.0, gvals, stream=s)
        return gvals, lam, None, None, None, None


def sparse_spd_solve(vals, b, handle: Handle, tol: float = 1e-2, rtol: float = 1e-10, max_iter: int = 2000):
    """x = A(vals)^{-1} b, differentiable in vals and b."""
    return SparseSPDSolve.apply(vals, b, handle, tol, rtol, max_iter)
