"""The per-site objective g_r^(reg) (Eq. g_regdef2) as a torch.autograd.Function.

forward(h, J) returns f[N] (FP64), one objective per site.  Site r's
objective depends only on its own block (h[r], J[r]), so the adjoint is the
per-site gradient (Eqs. g_gradh2, g_gradJ2) scaled by the incoming
gradient of f[r].  When h or J needs a gradient, f and the gradient come
from one call of the library's evaluation (plm_site_objective_grad: the
one-hot logits contraction, log-softmax, and the transposed one-hot
contraction of w (P - Y) / B_eff plus the l2 term) and backward only
applies the chain-rule scale; otherwise (no_grad, or inputs that do not
require grad) the call computes the objective alone.
"""
from __future__ import annotations

import torch

from . import api

_contexts: dict = {}


def default_context(device: int) -> api.Context:
    if device not in _contexts:
        _contexts[device] = api.Context(device)
    return _contexts[device]


class PlmObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, J, msa, w, beff, lambda_h=0.01, lambda_J=0.01, prec="fp32",
                plm_ctx=None):
        dev = h.device.index if h.device.index is not None else torch.cuda.current_device()
        c = plm_ctx or default_context(dev)
        need = bool(ctx.needs_input_grad[0] or ctx.needs_input_grad[1])
        f, gh, gJ = api.plm_site_objective_grad(
            c, msa, w, float(beff), h.detach().contiguous(), J.detach().contiguous(),
            lambda_h, lambda_J, prec, grad=need)
        if need:
            ctx.save_for_backward(gh, gJ)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        gh, gJ = ctx.saved_tensors
        go = grad_f.to(gh.dtype)
        return (go[:, None] * gh, go[:, None, None, None] * gJ,
                None, None, None, None, None, None, None)


def plm_objective(h, J, msa, w, beff, lambda_h=0.01, lambda_J=0.01, prec="fp32", plm_ctx=None):
    """f[N] = g_r^(reg)(h_r, J_r) for every site, differentiable in h and J."""
    return PlmObjective.apply(h, J, msa, w, beff, lambda_h, lambda_J, prec, plm_ctx)
