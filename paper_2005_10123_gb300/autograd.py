"""torch.autograd.Function over the library's log-likelihood and gradient.

``hawkes_loglik(theta, ctx, set_id)`` returns ell(Theta) of Eq. 1 (Section 2.1) as a 0-d tensor
whose backward pass multiplies the incoming gradient by d ell / d Theta, computed by the
library in the same pass over the pairs (no autograd tape through the O(N^2) sum). ``theta``
is a float64 tensor of shape (6,) or (K, 6) (K <= 64 parameter vectors evaluated in one launch
on the same event set); the result has shape () or (K,).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class HawkesLogLik(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta: torch.Tensor, hctx: "binding.Context", set_id: int, mode: int):
        th = theta.detach().to("cpu", torch.float64).numpy()
        want_grad = theta.requires_grad
        if th.ndim == 1:
            if want_grad:
                ll, g = hctx.hawkes_loglik_grad(set_id, th, mode)
            else:
                ll, g = hctx.hawkes_loglik(set_id, th, mode), np.zeros(6)
            ll = np.asarray(ll)
        else:
            res = hctx.hawkes_loglik_batch(set_id, th, mode, want_grad=want_grad)
            ll, g = res if want_grad else (res, np.zeros_like(th))
        fctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(ll, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(fctx, grad_out: torch.Tensor):
        (g,) = fctx.saved_tensors
        if g.ndim == 1:
            return grad_out * g, None, None, None
        return grad_out.unsqueeze(-1) * g, None, None, None


def hawkes_loglik(theta: torch.Tensor, hctx: "binding.Context", set_id: int,
                  mode: int = binding.HAWKES_MIXED) -> torch.Tensor:
    """ell(Theta) with autograd support (see the module docstring)."""
    return HawkesLogLik.apply(theta, hctx, set_id, mode)
