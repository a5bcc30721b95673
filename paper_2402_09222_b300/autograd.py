"""torch.autograd bridge for the macroscopic lookup.

    Sigma = xs_lookup(handle, dens, sigma, E, mat)

is differentiable in the atom densities `dens` [nnz] and the cross-section
table `sigma` [P][n_ch] (both FP64 CUDA tensors).  The forward pass writes
them into the library's tables (rounded to FP32 when the tables are FP32) and
runs the exact lookup kernel; the backward pass is the library's adjoint
kernel (the lookup is linear in both):
    dL/dN_j      = sum_r g_r sigma_{r,j}(E)
    dL/ds_r[k]   += N_j (1 - f) g_r,   dL/ds_r[k+1] += N_j f g_r.
"""
from __future__ import annotations

import torch

from . import mcx


class XsLookup(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dens, sigma, handle, E, mat):
        d, s = dens.detach().clone().contiguous(), sigma.detach().clone().contiguous()
        handle.update_tables_device(dens=d, sigma=s)
        out = handle.xs_lookup(E, mat, flags=mcx.LOOKUP_EXACT)
        ctx.handle = handle
        ctx.save_for_backward(E, mat, d, s)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        E, mat, d, s = ctx.saved_tensors
        # the library's tables may have been overwritten by later forward
        # calls on the same handle: put back the values this forward used
        ctx.handle.update_tables_device(dens=d, sigma=s)
        gd, gs = ctx.handle.xs_lookup_backward(E, mat, grad_out.contiguous().to(torch.float64))
        need_d, need_s = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        return (gd if need_d else None), (gs if need_s else None), None, None, None


def xs_lookup(handle: "mcx.Problem", dens: torch.Tensor, sigma: torch.Tensor, E: torch.Tensor,
              mat: torch.Tensor) -> torch.Tensor:
    """Differentiable macroscopic lookup (exact arithmetic)."""
    return XsLookup.apply(dens, sigma, handle, E, mat)
