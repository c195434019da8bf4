"""torch.autograd.Function around the library's forward and adjoint kernels.

`log_target(ctx, theta)` returns log pi_k(theta_j) for particles theta [J, D]
(float32, CUDA, canonical parameter order) under the context's current target
(Sec. 2: the prior plus the c_i-weighted log-likelihood of the annealed subset,
eq. approx-grad).  Both passes run in libsmc: the forward call evaluates the
networks and their adjoint at once (smc_eval_device), and the backward pass
returns grad_output[j] * grad log pi_k(theta_j) from that gradient.  The
context's particles are overwritten with theta, and its stream must be the
caller's current stream (contexts take torch's current stream at creation).
"""
from __future__ import annotations

import torch

from . import smc as S


class LogTarget(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, ctx):
        if theta.dtype != torch.float32 or not theta.is_cuda or theta.dim() != 2:
            raise ValueError("theta must be a float32 CUDA tensor [J, D]")
        theta = theta.detach().contiguous()
        J, D = theta.shape
        S.smc_set_state_device(ctx, theta)
        logpi = torch.empty(J, dtype=torch.float64, device=theta.device)
        grad = torch.empty((J, D), dtype=torch.float32, device=theta.device)
        S.smc_eval_device(ctx, logpi, grad)
        fctx.save_for_backward(grad)
        return logpi

    @staticmethod
    def backward(fctx, grad_out):
        (grad,) = fctx.saved_tensors
        return grad_out.to(grad.dtype).unsqueeze(1) * grad, None


def log_target(ctx, theta):
    """log pi_k(theta) [J] (float64), differentiable in theta."""
    return LogTarget.apply(theta, ctx)
