"""Backward of the composite operators through autograd against the fp64
oracle's chain rule (erosion / dilation backward composed by hand), with the
tolerance of the single-operator backward summed over the two passes."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _oracle_chain(which, f, L, se, g):
    """(y, grad_x, grad_b, scale_x, scale_b): the chain rule in fp64, and the
    same chain with |g| and each pass's contribution taken in absolute value
    (the scale of the fp32 rounding, free of cancellation between passes)."""
    m, o, org = se.mask, se.offset, se.origin
    mb = int(o[m != 0].max()) if m.any() else 0
    a = np.abs(g)
    if which == "open":
        E, cE = oracle.erode(f, L, m, o, org)
        Es = E + mb
        D, cD = oracle.dilate(Es, L + mb, m, o, org)
        g1, gb2 = oracle.dilate_backward(Es, L + mb, m, o, org, D, cD, g)
        gx, gb1 = oracle.erode_backward(f, L, m, o, org, E, cE, g1)
        a1, ab2 = oracle.dilate_backward(Es, L + mb, m, o, org, D, cD, a)
        ax, ab1 = oracle.erode_backward(f, L, m, o, org, E, cE, a1)
        return D - mb, gx, gb1 + gb2, np.abs(ax), np.abs(ab1) + np.abs(ab2)
    if which == "close":
        D, cD = oracle.dilate(f, L, m, o, org)
        E, cE = oracle.erode(D, L + mb, m, o, org)
        g1, gb2 = oracle.erode_backward(D, L + mb, m, o, org, E, cE, g)
        gx, gb1 = oracle.dilate_backward(f, L, m, o, org, D, cD, g1)
        a1, ab2 = oracle.erode_backward(D, L + mb, m, o, org, E, cE, a)
        ax, ab1 = oracle.dilate_backward(f, L, m, o, org, D, cD, a1)
        return E, gx, gb1 + gb2, np.abs(ax), np.abs(ab1) + np.abs(ab2)
    D, cD = oracle.dilate(f, L, m, o, org)
    E, cE = oracle.erode(f, L, m, o, org)
    gx1, gb1 = oracle.dilate_backward(f, L, m, o, org, D, cD, g)
    gx2, gb2 = oracle.erode_backward(f, L, m, o, org, E, cE, -g)
    ax1, ab1 = oracle.dilate_backward(f, L, m, o, org, D, cD, a)
    ax2, ab2 = oracle.erode_backward(f, L, m, o, org, E, cE, a)
    return D - E, gx1 + gx2, gb1 + gb2, np.abs(ax1) + np.abs(ax2), np.abs(ab1) + np.abs(ab2)


@pytest.mark.parametrize("which", ["open", "close", "gradient"])
@pytest.mark.parametrize("case", [(2, 33, 41, 16, 5, 5, 0.6, 3, None), (1, 50, 47, 64, 7, 3, 0.8, 9, (2, 0)),
                                  (3, 20, 20, 4, 3, 3, 1.0, 1, None)])
def test_composite_backward_matches_oracle_chain(which, case):
    from paper_2305_03018_gb300 import autograd as ag
    N, H, W, L, kh, kw, p_in, mo, origin = case
    g = wl.rng(hash((which, H, W)) & 0xFFFF)
    f = g.integers(0, L, size=(N, H, W)).astype(np.int32)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin)
    up = g.standard_normal((N, H, W))
    x = torch.from_numpy(f.astype(np.float32)).cuda().requires_grad_(True)
    b = torch.from_numpy(se.offset.astype(np.float32)).cuda().requires_grad_(True)
    y = {"open": ag.opening, "close": ag.closing, "gradient": ag.gradient}[which](x, b, L, se.mask, se.origin)
    y.backward(torch.from_numpy(up.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    ref_y, ref_gx, ref_gb, abs_gx, abs_gb = _oracle_chain(which, f, L, se, up)
    np.testing.assert_array_equal(y.detach().cpu().numpy().astype(np.int64), ref_y)
    taps = int(np.count_nonzero(se.mask))
    gx = x.grad.cpu().numpy().astype(np.float64)
    # two passes: the first pass's fp32 rounding is propagated by the second (gain <= 1 per tap)
    assert (np.abs(gx - ref_gx) <= 2 * (taps + 2) * U * abs_gx * (taps + 1) + 1e-30).all(), np.abs(gx - ref_gx).max()
    gb = b.grad.cpu().numpy().astype(np.float64)
    assert (np.abs(gb - ref_gb) <= 2 * (48 + taps + 2) * U * abs_gb + U * np.abs(ref_gb) + 1e-30).all(), \
        np.abs(gb - ref_gb).max()
