"""GPU backward (tie-split argmax gradient) against the fp64 CPU oracle.

Tolerance from the arithmetic: the library sums fp32 terms g(x)/cD(x).
grad_in(p) adds at most |B| terms in sequence: |error| <= (|B| + 2) u S(p);
grad_se(y) adds each chunk of pixels with a depth of at most 32 + 5 + 8
additions (a thread's pixels, a warp tree, a CTA's warps; up to 1024 taps the
fused kernel's depth is 8 + 5 + 8), then the chunks in fp64:
|error| <= 48 u S(y) + u |grad_se(y)|,
where u = 2^-24 and S is the same sum taken over |g| (the oracle with |g|).
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _oracle_grads(f, L, mask, off, origin, g):
    D, cD = oracle.dilate(f, L, mask, off, origin)
    gf, gb = oracle.dilate_backward(f, L, mask, off, origin, D, cD, g)
    sf, sb = oracle.dilate_backward(f, L, mask, off, origin, D, cD, np.abs(g))
    return D, cD, gf, gb, sf, sb


def _check(x_np, b_np, mask, origin, L, g_np):
    from paper_2305_03018_gb300.autograd import dilate
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    b = torch.from_numpy(b_np).cuda().requires_grad_(True)
    y = dilate(x, b, L, mask, origin)
    y.backward(torch.from_numpy(g_np).cuda())
    torch.cuda.synchronize()
    H, W = x_np.shape[-2:]
    f = x_np.reshape(-1, H, W).astype(np.int32)
    off = b_np.astype(np.int32)
    D, cD, gf, gb, sf, sb = _oracle_grads(f, L, mask, off, origin, g_np.reshape(-1, H, W).astype(np.float64))
    np.testing.assert_array_equal(y.detach().cpu().numpy().reshape(D.shape).astype(np.int64), D)
    ntaps = int(np.count_nonzero(mask))
    gx = x.grad.cpu().numpy().reshape(gf.shape).astype(np.float64)
    assert (np.abs(gx - gf) <= (ntaps + 2) * U * sf + 1e-30).all(), np.abs(gx - gf).max()
    gbg = b.grad.cpu().numpy().astype(np.float64)
    assert (np.abs(gbg - gb) <= 48 * U * sb + U * np.abs(gb) + 1e-30).all(), np.abs(gbg - gb).max()
    assert (gbg[np.asarray(mask) == 0] == 0).all()
    return x.grad.clone(), b.grad.clone()


def test_c4_layer_forward_backward():
    c = wl.c4_layer()
    mask = np.ones((9, 9), np.uint8)
    gx1, gb1 = _check(c.x, c.b, mask, c.origin, c.L, c.g)
    gx2, gb2 = _check(c.x, c.b, mask, c.origin, c.L, c.g)
    assert torch.equal(gx1, gx2) and torch.equal(gb1, gb2)        # deterministic


def test_irregular_se_with_ties():
    g = wl.rng(31)
    x = g.integers(0, 4, size=(3, 1, 37, 53)).astype(np.float32)       # L = 4: many ties
    se = wl.se_random(g, 7, 5, 0.6, 2, origin=(1, 4))
    up = g.standard_normal(x.shape).astype(np.float32)
    _check(x, se.offset.astype(np.float32), se.mask, se.origin, 4, up)


def test_single_point_se_closed_form():
    g = wl.rng(32)
    x = g.integers(0, 16, size=(2, 1, 20, 24)).astype(np.float32)
    mask = np.zeros((3, 3), np.uint8)
    mask[0, 2] = 1
    off = np.zeros((3, 3), np.float32)
    off[0, 2] = 5
    up = g.standard_normal(x.shape).astype(np.float32)
    gx, gb = _check(x, off, mask, (1, 1), 16, up)
    # y = (-1, 1): p receives g(p + y) where p + y is inside
    exp = np.zeros_like(up)
    exp[:, :, 1:, :-1] = up[:, :, :-1, 1:]
    np.testing.assert_allclose(gx.cpu().numpy(), exp, rtol=0, atol=0)


def _check_erode(x_np, b_np, mask, origin, L, g_np):
    from paper_2305_03018_gb300.autograd import erode
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    b = torch.from_numpy(b_np).cuda().requires_grad_(True)
    y = erode(x, b, L, mask, origin)
    y.backward(torch.from_numpy(g_np).cuda())
    torch.cuda.synchronize()
    H, W = x_np.shape[-2:]
    f = x_np.reshape(-1, H, W).astype(np.int32)
    off = b_np.astype(np.int32)
    gg = g_np.reshape(-1, H, W).astype(np.float64)
    E, cE = oracle.erode(f, L, mask, off, origin)
    gf, gb = oracle.erode_backward(f, L, mask, off, origin, E, cE, gg)
    sf, sb = oracle.erode_backward(f, L, mask, off, origin, E, cE, np.abs(gg))
    np.testing.assert_array_equal(y.detach().cpu().numpy().reshape(E.shape).astype(np.int64), E)
    ntaps = int(np.count_nonzero(mask))
    gx = x.grad.cpu().numpy().reshape(gf.shape).astype(np.float64)
    assert (np.abs(gx - gf) <= (ntaps + 2) * U * sf + 1e-30).all(), np.abs(gx - gf).max()
    gbg = b.grad.cpu().numpy().astype(np.float64)
    assert (np.abs(gbg - gb) <= 48 * U * np.abs(sb) + U * np.abs(gb) + 1e-30).all(), np.abs(gbg - gb).max()
    assert (gbg[np.asarray(mask) == 0] == 0).all()


def test_c4_layer_erosion_backward():
    c = wl.c4_layer()
    _check_erode(c.x, c.b, np.ones((9, 9), np.uint8), c.origin, c.L, c.g)


def test_erosion_backward_irregular_se_with_ties():
    g = wl.rng(33)
    x = g.integers(0, 4, size=(2, 1, 29, 41)).astype(np.float32)
    se = wl.se_random(g, 5, 7, 0.6, 2, origin=(3, 1))
    up = g.standard_normal(x.shape).astype(np.float32)
    _check_erode(x, se.offset.astype(np.float32), se.mask, se.origin, 4, up)


@pytest.mark.parametrize("shape", [(2, 1, 5, 9000), (1, 1, 300, 1), (3, 1, 70, 33), (1, 1, 1, 40)])
def test_chunking_edge_shapes(shape):
    # SE-gradient chunks (runs of consecutive pixels, or rows x columns blocks above 1024
    # taps): rows wider than a chunk, one-column images, ragged chunk tails
    g = wl.rng(sum(shape))
    x = g.integers(0, 8, size=shape).astype(np.float32)
    se = wl.se_random(g, 3, 5, 0.7, 3, origin=(1, 2))
    up = g.standard_normal(shape).astype(np.float32)
    _check(x, se.offset.astype(np.float32), se.mask, se.origin, 8, up)
    _check_erode(x, se.offset.astype(np.float32), se.mask, se.origin, 8, up)


def test_more_than_1024_taps():
    # above 1024 taps the two gradients come from the two gathers instead of the fused pass
    g = wl.rng(35)
    x = g.integers(0, 6, size=(2, 1, 48, 61)).astype(np.float32)
    se = wl.se_full_random(g, 33, 3)
    up = g.standard_normal(x.shape).astype(np.float32)
    _check(x, se.offset.astype(np.float32), se.mask, se.origin, 6, up)
    _check_erode(x, se.offset.astype(np.float32), se.mask, se.origin, 6, up)
