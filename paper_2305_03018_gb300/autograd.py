"""PyTorch autograd layers over the library's forward and backward entry points.

Learnable grey-value dilation and erosion: activations are quantised to the
tonal range {0..L-1} and the SE offsets to non-negative integers (rounding,
with a straight-through gradient), the forward is the library's exact
operator (``morph_dilate`` / ``morph_erode``, also returning the top counts)
and the backward its tie-split argmax / argmin gradient
(``morph_dilate_backward`` / ``morph_erode_backward``).  Torch provides the
tensors, the stream and the autograd graph; both passes run in the library's
CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import morph as M


class _MorphFunction(torch.autograd.Function):
    """y = op(round(x), SE with offsets round(b) on `mask`); op 0 = dilation,
    1 = erosion.  x: CUDA float tensor [..., H, W] (leading dims flattened
    into images); b: float tensor [kh, kw]; mask: host array [kh, kw];
    origin: (oy, ox).  Returns a float tensor shaped like x."""

    @staticmethod
    def forward(ctx, x, b, L: int, mask, origin, op: int):
        shape = x.shape
        H, W = shape[-2], shape[-1]
        q = x.detach().round().clamp_(0, L - 1).to(torch.uint8 if L <= 256 else torch.int32)
        q = q.reshape(-1, H, W).contiguous()
        bq = b.detach().round().clamp_(min=0).to(torch.int32).cpu().numpy()
        se = M.SEView(np.asarray(mask), bq, origin)
        lib = M.get_context(x.device.index or 0)
        out, cnt = (lib.dilate if op == 0 else lib.erode)(q, L, se, count=True)
        ctx.save_for_backward(q, out, cnt)
        ctx.se, ctx.L, ctx.shape, ctx.b_shape, ctx.op = se, L, shape, b.shape, op
        return out.to(x.dtype).reshape(shape)

    @staticmethod
    def backward(ctx, g):
        q, out, cnt = ctx.saved_tensors
        lib = M.get_context(q.device.index or 0)
        g32 = g.detach().to(torch.float32).reshape(out.shape).contiguous()
        need_x, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        grad_in = torch.empty(out.shape, dtype=torch.float32, device=q.device) if need_x else None
        grad_se = torch.empty(tuple(ctx.b_shape), dtype=torch.float32, device=q.device) if need_b else None
        img = M.make_image(q, ctx.L)
        fn = M.morph_dilate_backward if ctx.op == 0 else M.morph_erode_backward
        M.check(fn(lib.handle, img, ctx.se.c, out.data_ptr(), cnt.data_ptr(), g32.data_ptr(),
                   grad_in.data_ptr() if grad_in is not None else None,
                   grad_se.data_ptr() if grad_se is not None else None,
                   M.current_stream_handle(q.device)),
                "morph_dilate_backward" if ctx.op == 0 else "morph_erode_backward")
        gx = grad_in.reshape(ctx.shape).to(g.dtype) if grad_in is not None else None
        return gx, grad_se, None, None, None, None


class MorphDilateFunction:
    """Differentiable exact dilation: ``MorphDilateFunction.apply(x, b, L, mask, origin)``."""

    @staticmethod
    def apply(x, b, L, mask, origin):
        return _MorphFunction.apply(x, b, L, mask, origin, 0)


class MorphErodeFunction:
    """Differentiable exact erosion: ``MorphErodeFunction.apply(x, b, L, mask, origin)``."""

    @staticmethod
    def apply(x, b, L, mask, origin):
        return _MorphFunction.apply(x, b, L, mask, origin, 1)


def _defaults(b, mask, origin):
    kh, kw = b.shape
    if mask is None:
        mask = np.ones((kh, kw), np.uint8)
    if origin is None:
        origin = (kh // 2, kw // 2)
    return mask, tuple(origin)


def dilate(x, b, L: int, mask=None, origin=None):
    """Differentiable exact dilation."""
    mask, origin = _defaults(b, mask, origin)
    return _MorphFunction.apply(x, b, int(L), mask, origin, 0)


def erode(x, b, L: int, mask=None, origin=None):
    """Differentiable exact erosion."""
    mask, origin = _defaults(b, mask, origin)
    return _MorphFunction.apply(x, b, int(L), mask, origin, 1)


class _MorphLayer(torch.nn.Module):
    def __init__(self, L: int, kh: int, kw: int, init=None, mask=None, origin=None):
        super().__init__()
        self.L = int(L)
        w = torch.zeros(kh, kw) if init is None else torch.as_tensor(init, dtype=torch.float32)
        self.offset = torch.nn.Parameter(w.clone())
        self.mask = np.ones((kh, kw), np.uint8) if mask is None else np.asarray(mask, np.uint8)
        self.origin = (kh // 2, kw // 2) if origin is None else tuple(origin)


class MorphDilate2d(_MorphLayer):
    """Learnable non-flat dilation layer with a kh x kw SE of offsets >= 0."""

    def forward(self, x):
        return dilate(x, self.offset, self.L, self.mask, self.origin)


class MorphErode2d(_MorphLayer):
    """Learnable non-flat erosion layer with a kh x kw SE of offsets >= 0."""

    def forward(self, x):
        return erode(x, self.offset, self.L, self.mask, self.origin)


# ------------------------------------------------------------ composites
# The composite operators (the combinations named in the paper's conclusion)
# as compositions of the exact layers, so their backward composes through
# autograd.  The erosion's output lies in [-max b, L-1]; before a second pass
# it is shifted by max b into the tonal range [0, L + max b) of that pass
# (the shift has gradient 1), which needs L + max b <= 256.

def _tonal_shift(b, L: int):
    mb = int(b.detach().round().clamp(min=0).max().item()) if b.numel() else 0
    if L + mb > 256:
        raise ValueError(f"composite needs L + max b <= 256 (got {L} + {mb})")
    return mb


def opening(x, b, L: int, mask=None, origin=None):
    """Differentiable opening (x erode b) dilate b."""
    mask, origin = _defaults(b, mask, origin)
    mb = _tonal_shift(b, L)
    e = _MorphFunction.apply(x, b, int(L), mask, origin, 1)
    return _MorphFunction.apply(e + mb, b, int(L) + mb, mask, origin, 0) - mb


def closing(x, b, L: int, mask=None, origin=None):
    """Differentiable closing (x dilate b) erode b."""
    mask, origin = _defaults(b, mask, origin)
    mb = _tonal_shift(b, L)
    d = _MorphFunction.apply(x, b, int(L), mask, origin, 0)
    return _MorphFunction.apply(d, b, int(L) + mb, mask, origin, 1)


def gradient(x, b, L: int, mask=None, origin=None):
    """Differentiable Beucher gradient (x dilate b) - (x erode b)."""
    mask, origin = _defaults(b, mask, origin)
    return (_MorphFunction.apply(x, b, int(L), mask, origin, 0) -
            _MorphFunction.apply(x, b, int(L), mask, origin, 1))
