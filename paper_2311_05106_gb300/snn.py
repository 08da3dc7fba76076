"""Differentiable recurrent spiking network over the C ABI (Appendix I).

``bptt_loss(...)`` is a ``torch.autograd.Function``: its forward runs
bp_snn_forward and bp_snn_loss, its backward bp_snn_backward (BPTT with
checkpointed recomputation).  ``SpikingRNN`` holds FP32 master parameters; the
recurrent CSR values are handed to the kernels in BF16 or FP32.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _device_tensor(t, name, dtypes, shape=None):
    """The library reads the parameter pointers as device memory of these
    types and sizes: anything else is rejected here."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if t.dtype not in dtypes:
        raise ValueError("%s has dtype %s, expected one of %s" % (name, t.dtype, dtypes))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


def make_desc(B_, T, n_in, n_rec, n_out, W_in, indptr, indices, w_rec, W_out, b_out, ckpt_every=100, **overrides):
    f32 = (torch.float32,)
    _device_tensor(W_in, "W_in", f32, (n_in, n_rec))
    _device_tensor(indptr, "indptr", (torch.int64,), (n_rec + 1,))
    _device_tensor(indices, "indices", (torch.int32,))
    _device_tensor(w_rec, "w_rec", (torch.float32, torch.bfloat16), (indices.numel(),))
    _device_tensor(W_out, "W_out", f32, (n_rec, n_out))
    _device_tensor(b_out, "b_out", f32, (n_out,))
    d = B.bp_snn_desc_default()
    d.B, d.T, d.n_in, d.n_rec, d.n_out = int(B_), int(T), int(n_in), int(n_rec), int(n_out)
    d.ckpt_every = int(ckpt_every)
    for k, v in overrides.items():
        setattr(d, k, v)
    d.W_in = W_in.data_ptr()
    d.indptr = indptr.data_ptr()
    d.indices = indices.data_ptr()
    d.w_rec = w_rec.data_ptr()
    d.w_rec_kind = B.BP_W_BF16 if w_rec.dtype == torch.bfloat16 else B.BP_W_F32
    d.W_out = W_out.data_ptr()
    d.b_out = b_out.data_ptr()
    d.nnz = int(indices.numel())
    return d


class _BPTT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W_in, w_rec, W_out, b_out, u, labels, indptr, indices, rec_dtype, ckpt_every, overrides):
        Bsz, T, n_in = u.shape
        n_rec, n_out = W_out.shape
        _device_tensor(u, "u", (torch.uint8,))
        _device_tensor(labels, "labels", (torch.int64,), (Bsz,))
        w_k = w_rec.detach().to(rec_dtype).contiguous()
        W_in_c, W_out_c, b_c = W_in.detach().contiguous(), W_out.detach().contiguous(), b_out.detach().contiguous()
        d = make_desc(Bsz, T, n_in, n_rec, n_out, W_in_c, indptr, indices, w_k, W_out_c, b_c, ckpt_every,
                      **overrides)
        ws = torch.empty(B.bp_snn_workspace_bytes(d), dtype=torch.uint8, device=u.device)
        m = torch.empty((Bsz, n_out), dtype=torch.float32, device=u.device)
        loss = torch.empty(1, dtype=torch.float32, device=u.device)
        g_m = torch.empty_like(m)
        B.bp_snn_forward(d, u, m, ws)
        B.bp_snn_loss(m, labels, loss, g_m)
        B.bp_snn_reg_loss(d, ws, loss)
        ctx.keep = (d, ws, u, g_m, w_k, W_in_c, W_out_c, b_c, indptr, indices)
        ctx.shapes = (W_in.shape, w_rec.shape, W_out.shape, b_out.shape)
        ctx.m = m
        return loss[0]

    @staticmethod
    def backward(ctx, gL):
        d, ws, u, g_m, *_ = ctx.keep
        s_in, s_rec, s_out, s_b = ctx.shapes
        dev = u.device
        dW_in = torch.zeros(s_in, dtype=torch.float32, device=dev)
        dw_rec = torch.zeros(s_rec, dtype=torch.float32, device=dev)
        dW_out = torch.zeros(s_out, dtype=torch.float32, device=dev)
        db = torch.zeros(s_b, dtype=torch.float32, device=dev)
        gm = g_m if gL is None else (g_m * gL).contiguous()
        B.bp_snn_backward(d, u, gm, ws, dW_in, dw_rec, dW_out, db)
        return dW_in, dw_rec, dW_out, db, None, None, None, None, None, None, None


def bptt_loss(W_in, w_rec, W_out, b_out, u, labels, indptr, indices, rec_dtype=torch.float32, ckpt_every=100,
              **overrides):
    """Mean cross-entropy loss of the network on inputs u (uint8 [B, T, n_in]),
    plus the voltage regulariser when lambda_v > 0; differentiable with
    respect to W_in, w_rec, W_out and b_out.  Overrides set bp_snn_desc
    fields: e.g. surrogate=BP_SG_RELU, sg_alpha, sg_width, lambda_v, v_hi,
    v_lo, slope."""
    return _BPTT.apply(W_in, w_rec, W_out, b_out, u, labels, indptr, indices, rec_dtype, ckpt_every, overrides)


class SpikingRNN:
    """Recurrent spiking network of Appendix I with FP32 master parameters."""

    def __init__(self, weights: dict, rec_dtype=torch.bfloat16, ckpt_every=100, device="cuda"):
        def t(x):
            return torch.as_tensor(np.ascontiguousarray(x)).to(device)
        self.W_in = t(weights["W_in"]).float().requires_grad_()
        self.w_rec = t(weights["w_rec"]).float().requires_grad_()
        self.W_out = t(weights["W_out"]).float().requires_grad_()
        self.b_out = t(weights["b_out"]).float().requires_grad_()
        self.indptr = t(weights["indptr"]).long()
        self.indices = t(weights["indices"]).int()
        self.rec_dtype = rec_dtype
        self.ckpt_every = ckpt_every

    def parameters(self):
        return [self.W_in, self.w_rec, self.W_out, self.b_out]

    def loss(self, u, labels):
        return bptt_loss(self.W_in, self.w_rec, self.W_out, self.b_out, u, labels, self.indptr, self.indices,
                         self.rec_dtype, self.ckpt_every)
