"""``torch.autograd.Function`` over the library's NLML and its adjoint gradient.

``nlml(log_theta, gp)`` returns the negative log marginal likelihood (the
negative of Eq. 5) at hyperparameters exp(log_theta) = (l, nu, sigma^2) as a
0-d float64 tensor; its backward is the gradient that the fused adjoint kernel
computes, 1/2 tr((K^{-1} - alpha alpha^T) dK/dlog theta), scaled by the
incoming gradient.  Both directions run in the CUDA library; PyTorch only
carries the three scalars.
"""
from __future__ import annotations

import numpy as np
import torch


class GPNLML(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_theta: torch.Tensor, gp) -> torch.Tensor:
        th = log_theta.detach().to("cpu", torch.float64).numpy()
        _, trainable = gp.get_hyper()
        gp.set_hyper(np.exp(th), trainable)
        f, g = gp.nlml_grad()
        ctx.save_for_backward(torch.as_tensor(g, dtype=log_theta.dtype, device=log_theta.device))
        return torch.tensor(f, dtype=log_theta.dtype, device=log_theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def nlml(log_theta: torch.Tensor, gp) -> torch.Tensor:
    """NLML(exp(log_theta)) of the handle ``gp`` (a :class:`gprat.GP`), differentiable in log_theta."""
    return GPNLML.apply(log_theta, gp)
