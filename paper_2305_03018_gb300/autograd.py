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
    origin: (oy, ox).  Returns a float tensor shaped like x.

    max_offset None: the rounded offsets are copied to the host (the call
    waits for the device) and every exact route is open to AUTO.  An integer
    bound: the offsets are clamped into [0, max_offset] on the device and the
    FP8 route reads them there (morph_dilate_dev_se), so neither pass waits
    for the device or copies to the host."""

    @staticmethod
    def forward(ctx, x, b, L: int, mask, origin, op: int, max_offset=None):
        shape = x.shape
        H, W = shape[-2], shape[-1]
        q = x.detach().round().clamp_(0, L - 1).to(torch.uint8 if L <= 256 else torch.int32)
        q = q.reshape(-1, H, W).contiguous()
        lib = M.get_context(x.device.index or 0)
        if max_offset is None:
            bq = b.detach().round().clamp_(min=0).to(torch.int32).cpu().numpy()
            se = M.SEView(np.asarray(mask), bq, origin)
            out, cnt = (lib.dilate if op == 0 else lib.erode)(q, L, se, count=True)
        else:
            bq = b.detach().round().clamp_(0, int(max_offset)).to(torch.int32).contiguous()
            se = M.SEDevView(np.asarray(mask), bq, origin, int(max_offset))
            out, cnt = lib.morph_dev_se(op, q, L, se, count=True)
        ctx.save_for_backward(q, out, cnt)
        ctx.se, ctx.L, ctx.shape, ctx.b_shape, ctx.op = se, L, shape, b.shape, op
        ctx.dev = max_offset is not None
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
        if ctx.dev:
            fn = M.morph_dilate_backward_dev_se if ctx.op == 0 else M.morph_erode_backward_dev_se
        else:
            fn = M.morph_dilate_backward if ctx.op == 0 else M.morph_erode_backward
        M.check(fn(lib.handle, img, ctx.se.c, out.data_ptr(), cnt.data_ptr(), g32.data_ptr(),
                   grad_in.data_ptr() if grad_in is not None else None,
                   grad_se.data_ptr() if grad_se is not None else None,
                   M.current_stream_handle(q.device)),
                "morph_dilate_backward" if ctx.op == 0 else "morph_erode_backward")
        gx = grad_in.reshape(ctx.shape).to(g.dtype) if grad_in is not None else None
        return gx, grad_se, None, None, None, None, None


class MorphDilateFunction:
    """Differentiable exact dilation: ``MorphDilateFunction.apply(x, b, L, mask, origin[, max_offset])``."""

    @staticmethod
    def apply(x, b, L, mask, origin, max_offset=None):
        return _MorphFunction.apply(x, b, L, mask, origin, 0, max_offset)


class MorphErodeFunction:
    """Differentiable exact erosion: ``MorphErodeFunction.apply(x, b, L, mask, origin[, max_offset])``."""

    @staticmethod
    def apply(x, b, L, mask, origin, max_offset=None):
        return _MorphFunction.apply(x, b, L, mask, origin, 1, max_offset)


def _defaults(b, mask, origin):
    kh, kw = b.shape
    if mask is None:
        mask = np.ones((kh, kw), np.uint8)
    if origin is None:
        origin = (kh // 2, kw // 2)
    return mask, tuple(origin)


def dilate(x, b, L: int, mask=None, origin=None, max_offset=None):
    """Differentiable exact dilation (max_offset: see _MorphFunction)."""
    mask, origin = _defaults(b, mask, origin)
    return _MorphFunction.apply(x, b, int(L), mask, origin, 0, max_offset)


def erode(x, b, L: int, mask=None, origin=None, max_offset=None):
    """Differentiable exact erosion (max_offset: see _MorphFunction)."""
    mask, origin = _defaults(b, mask, origin)
    return _MorphFunction.apply(x, b, int(L), mask, origin, 1, max_offset)


class _MorphLayer(torch.nn.Module):
    """max_offset: an integer bound keeps the offsets on the device (no host copy or
    wait per step; offsets are clamped into [0, max_offset]); None copies them."""

    def __init__(self, L: int, kh: int, kw: int, init=None, mask=None, origin=None, max_offset=None):
        super().__init__()
        self.L = int(L)
        self.max_offset = max_offset
        w = torch.zeros(kh, kw) if init is None else torch.as_tensor(init, dtype=torch.float32)
        self.offset = torch.nn.Parameter(w.clone())
        self.mask = np.ones((kh, kw), np.uint8) if mask is None else np.asarray(mask, np.uint8)
        self.origin = (kh // 2, kw // 2) if origin is None else tuple(origin)


class MorphDilate2d(_MorphLayer):
    """Learnable non-flat dilation layer with a kh x kw SE of offsets >= 0."""

    def forward(self, x):
        return dilate(x, self.offset, self.L, self.mask, self.origin, self.max_offset)


class MorphErode2d(_MorphLayer):
    """Learnable non-flat erosion layer with a kh x kw SE of offsets >= 0."""

    def forward(self, x):
        return erode(x, self.offset, self.L, self.mask, self.origin, self.max_offset)


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
    e = _MorphFunction.apply(x, b, int(L), mask, origin, 1, None)
    return _MorphFunction.apply(e + mb, b, int(L) + mb, mask, origin, 0, None) - mb


def closing(x, b, L: int, mask=None, origin=None):
    """Differentiable closing (x dilate b) erode b."""
    mask, origin = _defaults(b, mask, origin)
    mb = _tonal_shift(b, L)
    d = _MorphFunction.apply(x, b, int(L), mask, origin, 0, None)
    return _MorphFunction.apply(d, b, int(L) + mb, mask, origin, 1, None)


def gradient(x, b, L: int, mask=None, origin=None):
    """Differentiable Beucher gradient (x dilate b) - (x erode b)."""
    mask, origin = _defaults(b, mask, origin)
    return (_MorphFunction.apply(x, b, int(L), mask, origin, 0, None) -
            _MorphFunction.apply(x, b, int(L), mask, origin, 1, None))
