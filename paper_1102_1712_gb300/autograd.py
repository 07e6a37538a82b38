"""PyTorch autograd wrapper of the differentiable cost (Eq. 2) of the solve.

``pca_cost(w, f0, ...)`` returns J*(w, f0) = min over (a, b) of
||P f(w, f0) - a y - b||^2, with (a, b) from Eq. (A.1), as a 0-d float64
tensor.  Gradients flow to ``w`` (float64, K, on the CPU or a GPU: its
gradient is returned on w's device) and to the reference CT
``f0`` (CUDA float32, N).  Because (a, b) minimise J for fixed (w, f0), the
gradients of J* are the partial derivatives at that (a, b): dJ/dw is the
gradient below Eq. (A.2) and dJ/df0 = W^T (2 P^T r) (warp transpose of the
trilinear interpolation, Eq. A.5).

Forward evaluates J only; backward recomputes the warped volume and the
projection inside the library (nothing of size N is kept between the two
passes) and returns the gradients computed by the CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pcasolve as P


class _Problem:
    """Fixed inputs of one cost: motion model, measured image and geometry.
    Its device workspace serves every cost built on it, one call at a time:
    two costs of one problem evaluated concurrently (other streams or host
    threads) would race on it, so give each concurrent user its own problem."""

    def __init__(self, U, y, vol, cb, step, mean=None):
        self.U, self.y, self.vol, self.cb, self.step, self.mean = U, y, vol, cb, float(step), mean
        self.K = P._K(U, vol)
        self.ws = P.WorkspaceF0(vol, cb, self.K, device=U.device)


class CostFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, f0, prob: _Problem):
        wv = w.detach().cpu().double().numpy()
        J, _, ab, _ = P.cost_grad_f0(f0.detach(), prob.mean, prob.U, wv, prob.y, prob.vol, prob.cb,
                                     prob.step, want_grad=False, want_grad_f0=False, ws=prob.ws)
        ctx.save_for_backward(w, f0)
        ctx.prob = prob
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        w, f0 = ctx.saved_tensors
        prob = ctx.prob
        need_w, need_f0 = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_w or need_f0):
            return None, None, None
        wv = w.detach().cpu().double().numpy()
        _, G, _, dJdf0 = P.cost_grad_f0(f0.detach(), prob.mean, prob.U, wv, prob.y, prob.vol, prob.cb,
                                        prob.step, want_grad=True, want_grad_f0=need_f0, ws=prob.ws)
        gw = ((torch.from_numpy(np.asarray(G)).to(w.dtype) * gJ.detach().to("cpu", w.dtype)).to(w.device)
              if need_w else None)
        gf0 = (dJdf0 * gJ.to(dJdf0.device, torch.float32)).view_as(f0) if need_f0 else None
        return gw, gf0, None


def problem(U, y, vol, cb, step, mean=None) -> _Problem:
    return _Problem(U, y, vol, cb, step, mean)


def pca_cost(w: torch.Tensor, f0: torch.Tensor, prob: _Problem) -> torch.Tensor:
    """J*(w, f0) as a differentiable 0-d float64 tensor (see module docstring)."""
    return CostFunction.apply(w, f0, prob)
