"""Differentiable DISC front: SSD loss and its adjoint as a torch.autograd.Function.

``SSDLoss(ct, cbct, patch)`` fixes the CT (moving image) and the CBCT's patch
normalisation zs = (I_s - E(S)) / STD(S); calling it on a field r
([3][nz][ny][nx], float32, CUDA) returns

    L(r) = sum_x (I_m(x + r(x)) - I'_s(x))^2,   I'_s = zs STD(M) + E(M)

whose backward runs the library's hand-written adjoint kernels
(disc_k_ssd_grad): the patch statistics are recomputed in the backward pass,
not saved.  PyTorch only holds the tensors and the stream.
"""
from __future__ import annotations

import torch

from . import disc


class _SSD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, model):
        loss = torch.zeros(1, dtype=torch.float64, device=r.device)
        disc.k_ssd_loss(model.ct, model.zs, r, loss, model.patch, model.qs, model.var_floor)
        ctx.save_for_backward(r)
        ctx.model = model
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        (r,) = ctx.saved_tensors
        model = ctx.model
        grad = torch.empty_like(r)
        disc.k_ssd_grad(model.ct, model.zs, r, grad, model.patch, model.qs, var_floor=model.var_floor)
        return grad * grad_out.to(grad.dtype), None


class SSDLoss:
    """SSD between the warped CT and the moment-matched CBCT, differentiable in r."""

    def __init__(self, ct, cbct, patch=(3, 3, 3), var_floor=1e-6):
        if not (ct.is_cuda and cbct.is_cuda):
            raise ValueError("ct and cbct must be CUDA tensors")
        self.ct = ct.contiguous().float()
        cb = cbct.contiguous().float()
        self.patch = tuple(int(p) for p in patch)
        self.var_floor = float(var_floor)
        self.qs = disc.qscale(float(self.ct.abs().max()), self.patch)
        qs_s = disc.qscale(float(cb.abs().max()), self.patch)
        self.zs = torch.empty_like(cb)
        disc.k_static_norm(cb, self.zs, self.patch, qs_s, self.var_floor)

    def __call__(self, r):
        return _SSD.apply(r.contiguous(), self)
