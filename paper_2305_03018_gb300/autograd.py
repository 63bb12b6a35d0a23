"""PyTorch autograd layer over the library's forward and backward entry points.

A learnable grey-value dilation: activations are quantised to the tonal
range {0..L-1} and the SE offsets to non-negative integers (rounding, with a
straight-through gradient), the forward is the library's exact dilation
(``morph_dilate``, also returning the top counts) and the backward its
tie-split argmax gradient (``morph_dilate_backward``).  Torch provides the
tensors, the stream and the autograd graph; both passes run in the library's
CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import morph as M


class MorphDilateFunction(torch.autograd.Function):
    """y = dilation of round(x) by the SE with offsets round(b) on `mask`.

    x: CUDA float tensor [..., H, W] (leading dims flattened into images);
    b: float tensor [kh, kw] of SE offsets; mask: host array [kh, kw];
    origin: (oy, ox).  Returns a float tensor shaped like x.
    """

    @staticmethod
    def forward(ctx, x, b, L: int, mask, origin):
        shape = x.shape
        H, W = shape[-2], shape[-1]
        q = x.detach().round().clamp_(0, L - 1).to(torch.uint8 if L <= 256 else torch.int32)
        q = q.reshape(-1, H, W).contiguous()
        bq = b.detach().round().clamp_(min=0).to(torch.int32).cpu().numpy()
        se = M.SEView(np.asarray(mask), bq, origin)
        lib = M.get_context(x.device.index or 0)
        D, cD = lib.dilate(q, L, se, count=True)
        ctx.save_for_backward(q, D, cD)
        ctx.se = se
        ctx.L = L
        ctx.shape = shape
        ctx.b_shape = b.shape
        return D.to(x.dtype).reshape(shape)

    @staticmethod
    def backward(ctx, g):
        q, D, cD = ctx.saved_tensors
        se = ctx.se
        lib = M.get_context(q.device.index or 0)
        g32 = g.detach().to(torch.float32).reshape(D.shape).contiguous()
        need_x, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        grad_in = torch.empty(D.shape, dtype=torch.float32, device=q.device) if need_x else None
        grad_se = torch.empty(tuple(ctx.b_shape), dtype=torch.float32, device=q.device) if need_b else None
        img = M.make_image(q, ctx.L)
        M.check(M.morph_dilate_backward(lib.handle, img, se.c, D.data_ptr(), cD.data_ptr(), g32.data_ptr(),
                                        grad_in.data_ptr() if grad_in is not None else None,
                                        grad_se.data_ptr() if grad_se is not None else None,
                                        M.current_stream_handle(q.device)), "morph_dilate_backward")
        gx = grad_in.reshape(ctx.shape).to(g.dtype) if grad_in is not None else None
        return gx, grad_se, None, None, None


def dilate(x, b, L: int, mask=None, origin=None):
    """Differentiable exact dilation (see MorphDilateFunction)."""
    kh, kw = b.shape
    if mask is None:
        mask = np.ones((kh, kw), np.uint8)
    if origin is None:
        origin = (kh // 2, kw // 2)
    return MorphDilateFunction.apply(x, b, int(L), mask, tuple(origin))


class MorphDilate2d(torch.nn.Module):
    """Learnable non-flat dilation layer with a kh x kw SE of offsets >= 0."""

    def __init__(self, L: int, kh: int, kw: int, init=None, mask=None, origin=None):
        super().__init__()
        self.L = int(L)
        w = torch.zeros(kh, kw) if init is None else torch.as_tensor(init, dtype=torch.float32)
        self.offset = torch.nn.Parameter(w.clone())
        self.mask = np.ones((kh, kw), np.uint8) if mask is None else np.asarray(mask, np.uint8)
        self.origin = (kh // 2, kw // 2) if origin is None else tuple(origin)

    def forward(self, x):
        return dilate(x, self.offset, self.L, self.mask, self.origin)
