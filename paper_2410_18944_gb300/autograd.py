"""The field's training loss as a ``torch.autograd.Function``.

Forward and backward both run in libwost's fused training kernel: the
forward (hash-grid encode, the BF16 MLP on tcgen05 tensor cores, the
normalisation map of Tab. reg_map) is recomputed from the field's training
records, and the hand-written backward takes the one-sample gradients of
Sec. 4.2 Eq. one_sample_kld (the mixture parameters) and Sec. 4.4
Eq. one_sample_sp (the MIS selection logit) back through the MLP on tensor
cores and scatter-adds them into the hash grid.  The loss is the mean over
the records of -(p_t / q) [log p_g + e log(c p_g0 + (1 - c) p_u)] with p_g0
held fixed.  Only argument marshalling happens here.

Usage::

    field.set_records(records)              # 12 floats per record
    loss = field_loss(field, grid, W1, W2, W3, b3)   # CUDA float32 tensors
    loss.backward()                         # grads in the exchange layout

The parameters enter the kernel through the field (its FP32 masters, FP16
grid and BF16 weight copies are refreshed from the tensors on every forward),
so gradients are those of the rounded network, as in online training.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import check


def _fp(t):
    return C.cast(C.c_void_p(t.data_ptr()), L._fp)


class FieldLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field, grid, W1, W2, W3, b3):
        lib = L.load()
        params = []
        for t, (name, shape) in zip((grid, W1, W2, W3, b3), field.shapes().items()):
            if not t.is_cuda or tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name}: expected a CUDA tensor of shape {tuple(shape)}")
            params.append(t.detach().to(torch.float32).contiguous())
        torch.cuda.current_stream().synchronize()
        check(lib.wost_field_set_params(field._h, *[_fp(t) for t in params]))
        grads = [torch.empty_like(t) for t in params]
        e = L.Exec()
        lib.wost_exec_defaults(C.byref(e))
        e.stream = torch.cuda.current_stream().cuda_stream
        loss = C.c_float()
        check(lib.wost_train_grad(field._h, C.byref(e), C.byref(loss), *[_fp(g) for g in grads]))
        ctx.save_for_backward(*grads)
        return torch.tensor(loss.value, dtype=torch.float32, device=grid.device)

    @staticmethod
    def backward(ctx, gout):
        return (None,) + tuple(gout * g for g in ctx.saved_tensors)


def field_loss(field, grid, W1, W2, W3, b3):
    """Mean surrogate training loss of ``field``'s records at the given
    parameters; differentiable with respect to all five tensors."""
    return FieldLoss.apply(field, grid, W1, W2, W3, b3)
