"""0.5 ||A - W H||_F^2 as a torch.autograd.Function over the C ABI.

Forward: aunmf_loss_fwd (products, Gram matrices and FP64 reductions in the
library's kernels); backward: aunmf_loss_bwd, the hand-written kernels for
dW = g (W H H^T - A H^T) and dH = g (W^T W H - W^T A).  No gradient flows to
A.  Argument marshalling only."""
from __future__ import annotations

import torch

from . import aunmf

_handles = {}


def _handle():
    """The library handle of the current device, bound to torch's current
    stream: the inputs were produced there and the outputs are allocated for
    it by torch's caching allocator, so the library's kernels must run on it."""
    dev = torch.cuda.current_device()
    h = _handles.get(dev)
    if h is None:
        h = _handles[dev] = aunmf.Handle()
    h.set_stream(torch.cuda.current_stream())
    return h


class NMFLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, W, H, prec="fp32"):
        h = _handle()
        W = W.contiguous()
        H = H.contiguous()
        loss, wta = h.loss_fwd(A, W, H, prec=prec, save_wta=True)
        ctx.save_for_backward(A, W, H, wta)
        ctx.prec = prec
        return loss

    @staticmethod
    def backward(ctx, grad):
        A, W, H, wta = ctx.saved_tensors
        g = grad.detach().to(torch.float32).reshape(1).contiguous()
        dW, dH = _handle().loss_bwd(A, W, H, grad_out=g, wta=wta, prec=ctx.prec,
                                    need_w=ctx.needs_input_grad[1],
                                    need_h=ctx.needs_input_grad[2])
        return None, dW, dH, None


def nmf_loss(A, W, H, prec="fp32"):
    """0.5 ||A - W H||_F^2 (float64 scalar tensor) with gradients for W and H."""
    return NMFLoss.apply(A, W, H, prec)
