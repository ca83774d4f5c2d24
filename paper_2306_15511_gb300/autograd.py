"""torch.autograd.Function wrappers around the hand-written adjoint kernels.

- :class:`Alm2Map`: map = Y alm; backward is shtg_alm2map_vjp (the transpose
  kernel with the real-component factor), recomputing lambda_lm on the fly.
- :class:`GaussianLogPosterior`: the a-dependent part of Eq. (joint-posterior)
  for temperature, with gradients w.r.t. alm and the binned log C_l, both
  produced by one shtg_logpost_grad call in the forward pass.
"""
from __future__ import annotations

import torch


class Alm2Map(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, alm, spin=0):
        ctx.plan, ctx.spin = plan, spin
        return plan.alm2map(alm.contiguous(), spin)

    @staticmethod
    def backward(ctx, g):
        return None, ctx.plan.alm2map_vjp(g.contiguous(), ctx.spin), None


def alm2map(plan, alm, spin=0):
    return Alm2Map.apply(plan, alm, spin)


class GaussianLogPosterior(torch.autograd.Function):
    """L(a, theta) with C_l -> C_l exp(theta_k) on bin k; inputs alm
    (complex64, CUDA) and theta (float64, one entry per bin)."""

    @staticmethod
    def forward(ctx, plan, alm, theta, cl, bl, d, ninv, bins):
        # the library applies C_l exp(theta_k) per bin and returns dL/dtheta
        logp, g, gcl = plan.logpost_grad(cl, bl, alm.contiguous(), d, ninv, bins, components=True,
                                         theta=theta.detach().cpu().double().numpy())
        ctx.save_for_backward(g)
        ctx.gcl = torch.as_tensor(gcl, dtype=theta.dtype, device=theta.device)
        return torch.tensor(logp, dtype=torch.float64, device=alm.device)

    @staticmethod
    def backward(ctx, go):
        (g,) = ctx.saved_tensors
        return (None, g * go.to(g.real.dtype), ctx.gcl * go.to(ctx.gcl.dtype),
                None, None, None, None, None)


def log_posterior(plan, alm, theta, cl, bl, d, ninv, bins):
    return GaussianLogPosterior.apply(plan, alm, theta, cl, bl, d, ninv, bins)
