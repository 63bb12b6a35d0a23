"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: images, structuring elements (SEs) and
upstream gradients.  It holds none of the method's arithmetic, so that both
the CUDA library's tests/benchmarks and the CPU oracle can use it.

The paper's own workloads are ``numpy.random.randint`` images and filters
(Sec. 4.1, first and second experiment; Sec. 4.3 error experiment); its only
natural image is not available, so the smooth-noise image of
:func:`gauss_blurred_u8` stands in for natural 8-bit content.

SE convention: ``mask[r, c] != 0`` means the box entry (r, c) is in B; it is
the SE offset ``y = (r - oy, c - ox)`` with ``origin = (oy, ox)``, and
``offset[r, c]`` is ``b(y) >= 0`` (Sec. 2.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class SE:
    """A non-flat structuring element on a kh x kw box."""
    mask: np.ndarray            # uint8 [kh, kw], nonzero = in B
    offset: np.ndarray          # int32 [kh, kw], b(y) >= 0 (ignored where mask == 0)
    origin: tuple               # (oy, ox): box entry of the spatial origin
    name: str = ""

    @property
    def kh(self) -> int:
        return int(self.mask.shape[0])

    @property
    def kw(self) -> int:
        return int(self.mask.shape[1])

    @property
    def taps(self) -> int:
        return int(np.count_nonzero(self.mask))

    @property
    def max_offset(self) -> int:
        v = self.offset[self.mask != 0]
        return int(v.max()) if v.size else 0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------- SE shapes
def se_flat_square(k: int) -> SE:
    m = np.ones((k, k), np.uint8)
    return SE(m, np.zeros((k, k), np.int32), (k // 2, k // 2), f"flat_square{k}")


def se_flat_disk(radius: int) -> SE:
    k = 2 * radius + 1
    dy, dx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    m = ((dy * dy + dx * dx) <= radius * radius).astype(np.uint8)
    return SE(m, np.zeros((k, k), np.int32), (radius, radius), f"flat_disk_r{radius}")


def se_random(g: np.random.Generator, kh: int, kw: int, p_in: float, max_off: int,
              origin=None, force_origin: bool = True, name: str = "") -> SE:
    """Random support (Bernoulli ``p_in``) with integer offsets uniform in [0, max_off]."""
    oy, ox = origin if origin is not None else (kh // 2, kw // 2)
    m = (g.random((kh, kw)) < p_in).astype(np.uint8)
    if force_origin:
        m[oy, ox] = 1
    off = g.integers(0, max_off + 1, size=(kh, kw)).astype(np.int32)
    off[m == 0] = 0
    return SE(m, off, (oy, ox), name or f"random{kh}x{kw}_p{p_in}_o{max_off}")


def se_full_random(g: np.random.Generator, k: int, max_off: int) -> SE:
    m = np.ones((k, k), np.uint8)
    off = g.integers(0, max_off + 1, size=(k, k)).astype(np.int32)
    return SE(m, off, (k // 2, k // 2), f"full{k}_o{max_off}")


def _convex_hull(pts: np.ndarray) -> np.ndarray:
    """Andrew's monotone chain; returns hull vertices counter-clockwise."""
    p = sorted(set(map(tuple, pts.tolist())))
    if len(p) <= 2:
        return np.array(p, dtype=np.float64)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for q in p:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], q) <= 0:
            lower.pop()
        lower.append(q)
    for q in reversed(p):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], q) <= 0:
            upper.pop()
        upper.append(q)
    return np.array(lower[:-1] + upper[:-1], dtype=np.float64)


def se_random_convex(g: np.random.Generator, k: int, n_points: int, max_off: int) -> SE:
    """Support = lattice points inside the convex hull of ``n_points`` uniform
    points in the k x k box plus the centre; offsets uniform in [0, max_off]."""
    c = k // 2
    pts = g.integers(0, k, size=(n_points, 2))
    pts = np.vstack([pts, [[c, c]]])
    hull = _convex_hull(pts)
    rr, cc = np.mgrid[0:k, 0:k]
    inside = np.ones((k, k), bool)
    nv = len(hull)
    if nv >= 3:
        # hull is counter-clockwise in (row, col): interior points lie left of every edge
        for t in range(nv):
            a, b = hull[t], hull[(t + 1) % nv]
            cr = (b[0] - a[0]) * (cc - a[1]) - (b[1] - a[1]) * (rr - a[0])
            inside &= cr >= -1e-9
    m = inside.astype(np.uint8)
    m[c, c] = 1
    off = g.integers(0, max_off + 1, size=(k, k)).astype(np.int32)
    off[m == 0] = 0
    return SE(m, off, (c, c), f"convex{k}_o{max_off}")


# ------------------------------------------------------------------- images
def uniform_image(g: np.random.Generator, shape, L: int, dtype=np.uint8) -> np.ndarray:
    return g.integers(0, L, size=shape).astype(dtype)


def gauss_blurred_u8(g: np.random.Generator, n: int, sigma: float = 8.0) -> np.ndarray:
    """N(0,1) noise, separable Gaussian blur (radius 3 sigma, reflect boundary),
    min-max rescaled and rounded to [0, 255]."""
    x = g.standard_normal((n, n)).astype(np.float32)
    rad = int(round(3 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k = (k / k.sum()).astype(np.float32)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        xp = np.pad(x, pad, mode="reflect")
        acc = np.zeros_like(x)
        for idx, wgt in enumerate(k):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(idx, idx + x.shape[axis])
            acc += wgt * xp[tuple(sl)]
        x = acc
    lo, hi = float(x.min()), float(x.max())
    q = np.rint(255.0 * (x - lo) / max(hi - lo, 1e-30))
    return np.clip(q, 0, 255).astype(np.uint8)


# ------------------------------------------------------------ the workloads
@dataclass
class Problem:
    """One dilation or erosion problem."""
    f: np.ndarray               # [N, H, W] integer image (uint8 / uint16 / int32)
    L: int                      # tonal range size: values in [0, L-1]
    se: SE
    op: str = "dilate"          # "dilate" | "erode"
    name: str = ""


def c1_small_dilation() -> Problem:
    """256x256, L=16, 7x7 non-flat random 50% support (origin kept), offsets U[0,3]."""
    g = rng(1)
    f = uniform_image(g, (1, 256, 256), 16)
    se = se_random(g, 7, 7, 0.5, 3, origin=(3, 3), name="c1_random7x7_o3")
    return Problem(f, 16, se, "dilate", "c1_256x256_L16_se7x7")


def c2_large_filter() -> List[Problem]:
    """2048x2048, L=64: flat disk r=31 and 63x63 full support offsets U[0,7];
    dilation and erosion for each."""
    g = rng(2)
    f = uniform_image(g, (1, 2048, 2048), 64)
    disk = se_flat_disk(31)
    full = se_full_random(g, 63, 7)
    out = []
    for se in (disk, full):
        for op in ("dilate", "erode"):
            out.append(Problem(f, 64, se, op, f"c2_2048x2048_L64_{se.name}_{op}"))
    return out


def c3_full_tonal() -> Problem:
    """4096x4096 smooth 8-bit image (L=256), 31x31 random convex SE, offsets U[0,15]."""
    g = rng(3)
    f = gauss_blurred_u8(g, 4096, 8.0)[None]
    se = se_random_convex(g, 31, 12, 15)
    return Problem(f, 256, se, "dilate", "c3_4096x4096_L256_convex31")


@dataclass
class LayerCase:
    x: np.ndarray               # fp32 [B, 1, H, W], integer-valued in [0, L-1]
    b: np.ndarray               # fp32 [kh, kw], integer-valued offsets
    g: np.ndarray               # fp32 [B, 1, H, W] upstream gradient
    L: int
    origin: tuple


def c4_layer(batch: int = 64, size: int = 128) -> LayerCase:
    """Differentiable layer: 64x1x128x128 activations on L=32 levels, learnable
    9x9 SE with offsets in [0,7], upstream gradient N(0,1)."""
    g = rng(4)
    x = g.integers(0, 32, size=(batch, 1, size, size)).astype(np.float32)
    b = g.integers(0, 8, size=(9, 9)).astype(np.float32)
    up = g.standard_normal((batch, 1, size, size)).astype(np.float32)
    return LayerCase(x, b, up, 32, (4, 4))


def c5_batch(n: int = 512, seed: int = 5, max_side: int = 1024) -> List[Problem]:
    """Uneven serving-style batch: sides U[64, max_side], L in {16, 64, 256},
    odd SE sizes 3..63, flat (disk or square) or non-flat (full square with
    offsets U[0, L/16]), dilation or erosion, 50/50 each."""
    g = rng(seed)
    out = []
    for t in range(n):
        H = int(g.integers(64, max_side + 1))
        W = int(g.integers(64, max_side + 1))
        L = int(g.choice([16, 64, 256]))
        k = int(g.integers(1, 32)) * 2 + 1          # odd in [3, 63]
        if g.random() < 0.5:
            se = se_flat_disk(k // 2) if g.random() < 0.5 else se_flat_square(k)
        else:
            se = se_full_random(g, k, L // 16)
        op = "dilate" if g.random() < 0.5 else "erode"
        f = uniform_image(g, (1, H, W), L)
        out.append(Problem(f, L, se, op, f"c5_{t}_{H}x{W}_L{L}_{se.name}_{op}"))
    return out
