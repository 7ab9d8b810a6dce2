"""The field's training loss as a ``torch.autograd.Function``.

Both passes run in libwost's fused training kernel, which recomputes the
forward (hash-grid encode, the BF16 MLP on tcgen05 tensor cores, the
normalisation map of Tab. reg_map) from the field's training records instead
of storing activations.  ``forward`` runs it in its loss-only mode
(wost_train_loss: no backward pass, the loss written to a device tensor
without a host round trip); ``backward`` runs it with the hand-written
backward (wost_train_grad): the one-sample gradients of Sec. 4.2
Eq. one_sample_kld (the mixture parameters) and Sec. 4.4 Eq. one_sample_sp
(the MIS selection logit) go back through the MLP on tensor cores and are
scatter-added into the hash grid.  The loss is the mean over the records of
-(p_t / q) [log p_g + e log(c p_g0 + (1 - c) p_u)] with p_g0 held fixed.
Only argument marshalling happens here.

Usage::

    field.set_records(records)              # 12 floats per record
    loss = field_loss(field, grid, W1, W2, W3, b3)   # CUDA float32 tensors
    loss.backward()                         # grads in the exchange layout

The parameters enter the kernel through the field (its FP32 masters, FP16
grid and BF16 weight copies are refreshed from the tensors), so gradients
are those of the rounded network, as in online training.  ``backward``
loads the tensors saved by ``forward`` into the field again, so other uses
of the field in between do not change the gradient.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import check


def _fp(t):
    return C.cast(C.c_void_p(t.data_ptr()), L._fp)


def _load_params(lib, field, tensors):
    torch.cuda.current_stream().synchronize()
    check(lib.wost_field_set_params(field._h, *[_fp(t) for t in tensors]))


def _exec(lib, **kw):
    e = L.Exec()
    lib.wost_exec_defaults(C.byref(e))
    e.stream = torch.cuda.current_stream().cuda_stream
    for k, v in kw.items():
        setattr(e, k, v)
    return e


class FieldLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field, grid, W1, W2, W3, b3):
        lib = L.load()
        params = []
        for t, (name, shape) in zip((grid, W1, W2, W3, b3), field.shapes().items()):
            if not t.is_cuda or tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name}: expected a CUDA tensor of shape {tuple(shape)}")
            params.append(t.detach().to(torch.float32).contiguous())
        _load_params(lib, field, params)
        loss = torch.empty((), dtype=torch.float32, device=grid.device)
        e = _exec(lib, out_on_device=1)
        check(lib.wost_train_loss(field._h, C.byref(e), C.c_void_p(loss.data_ptr())))
        ctx.field = field
        ctx.save_for_backward(*params)
        return loss

    @staticmethod
    def backward(ctx, gout):
        lib = L.load()
        params = ctx.saved_tensors
        _load_params(lib, ctx.field, params)
        grads = [torch.empty_like(t) for t in params]
        loss = C.c_float()
        check(lib.wost_train_grad(ctx.field._h, C.byref(_exec(lib)), C.byref(loss), *[_fp(g) for g in grads]))
        return (None,) + tuple(gout * g for g in grads)


def field_loss(field, grid, W1, W2, W3, b3):
    """Mean surrogate training loss of ``field``'s records at the given
    parameters; differentiable with respect to all five tensors."""
    return FieldLoss.apply(field, grid, W1, W2, W3, b3)
