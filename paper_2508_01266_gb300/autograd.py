"""Differentiable Jacobian product: torch.autograd.Function around lrcc_jacobian_apply.

forward:  y = A x, the derivative of the CCSD residual along x (Eqs. 13-14), batched
          over the leading dimension of x1 [nrhs, Nk, o, v] and x2 [nrhs, Nk, Nk, Nk, o, o, v, v].
backward: the complex vector-Jacobian product of a holomorphic linear map,
          grad_x = A^H g = conj(A^T conj(g)), with A^T the transpose product of the
          Lambda equations (Eqs. 10-11).  The product symmetrises its doubles input
          first (A = A P_sym), so P_sym A^T returned by the library is the full
          transpose and the gradient is exact on arbitrary arrays.
Both directions run in the library's kernels; nothing here computes.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable


class LRCCJacobian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x1, x2, problem, options=None):
        ctx.problem = problem
        ctx.options = options
        return problem.jacobian_apply(x1.detach(), x2.detach(), options=options)

    @staticmethod
    @once_differentiable
    def backward(ctx, g1, g2):
        # conj() is a lazy view in torch: materialise it before the library reads the memory
        b1, b2 = ctx.problem.jacobian_apply(g1.conj().resolve_conj(), g2.conj().resolve_conj(), transpose=True,
                                            options=ctx.options)
        return b1.conj().resolve_conj(), b2.conj().resolve_conj(), None, None


def jacobian(problem, x1: torch.Tensor, x2: torch.Tensor, options=None):
    """y1, y2 = A x with autograd support (see LRCCJacobian)."""
    return LRCCJacobian.apply(x1, x2, problem, options)
