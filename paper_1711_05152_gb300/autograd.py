"""Differentiable multiple rank-1 lattice transform.

``reconstruct(y, plan)`` applies Algorithm 2 (the inverse multiple rank-1
lattice FFT, a linear map R from lattice samples to coefficients) on the GPU;
its backward pass applies the conjugate transpose R^H, which is the
hand-written ADJOINT mode of the lattice evaluation:
    (R^H g)_{l,j} = sum_{k in I_l} g_k / (counter_k M_l) exp(2 pi i j k.z_l / M_l).
For a real loss, PyTorch's complex gradient convention (the conjugate
Wirtinger derivative) makes the vector-Jacobian product of the linear map
y -> R y equal to R^H applied to the incoming gradient.
"""

from __future__ import annotations

import torch

from . import MR1L_ADJOINT, Plan


class Mr1lReconstruct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.reconstruct(y.contiguous())

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        g = grad.contiguous()
        return ctx.plan.evaluate(g, MR1L_ADJOINT), None


def reconstruct(y: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable Algorithm 2: y [nrhs, sum_M] (complex128, CUDA) -> [nrhs, nI]."""
    return Mr1lReconstruct.apply(y, plan)
