"""SEs whose offsets live in device memory (learnable layers) against the oracle.

morph_dilate_dev_se / morph_erode_dev_se plan from the host mask and a bound
on the offsets and read the offsets on the device, so a layer's step neither
copies them to the host nor waits for the device.  Results must equal the
oracle's (values and top counts), the backward must equal the host-SE
backward bit for bit (same kernels, same tap order), and an offset outside
the declared bound must be reported as a data error.
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2305_03018_gb300.morph import get_context
    return get_context(0)


CASES = [
    # (n, h, w, L, kh, kw, p_in, max_off, bound, origin)
    (2, 70, 130, 32, 9, 9, 1.0, 7, 7, (4, 4)),
    (1, 150, 90, 64, 7, 11, 0.6, 5, 9, (1, 8)),
    (1, 96, 200, 256, 15, 15, 0.5, 15, 15, None),
    (3, 40, 41, 16, 5, 3, 0.8, 3, 3, (-2, 1)),
]


@pytest.mark.parametrize("case", CASES)
def test_device_offsets_match_the_oracle(ctx, case):
    from paper_2305_03018_gb300 import morph as M
    n, h, w, L, kh, kw, p_in, mo, bound, origin = case
    g = wl.rng(900 + kh * kw + L)
    f = g.integers(0, L, size=(n, h, w)).astype(np.uint8)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin, force_origin=origin is None)
    ft = torch.from_numpy(f).cuda()
    off = torch.from_numpy(se.offset.astype(np.int32)).cuda()
    sev = M.SEDevView(se.mask, off, se.origin, bound)
    for op in (0, 1):
        D, cD = ctx.morph_dev_se(op, ft, L, sev, count=True)
        ctx.check()
        fn = oracle.dilate if op == 0 else oracle.erode
        rD, rC = fn(f, L, se.mask, se.offset, se.origin, nthreads=0)
        assert np.array_equal(D.cpu().numpy(), rD), op
        assert np.array_equal(cD.cpu().numpy(), rC), op
    # new offsets in the same device tensor: the next call reads them (no stale plan)
    new = g.integers(0, bound + 1, size=(kh, kw)).astype(np.int32) * (se.mask != 0)
    off.copy_(torch.from_numpy(new))
    D = ctx.morph_dev_se(0, ft, L, sev)
    ctx.check()
    rD, _ = oracle.dilate(f, L, se.mask, new, se.origin, nthreads=0)
    assert np.array_equal(D.cpu().numpy(), rD)


def test_offset_outside_the_bound_is_a_data_error(ctx):
    from paper_2305_03018_gb300 import morph as M
    g = wl.rng(911)
    f = torch.from_numpy(g.integers(0, 64, size=(1, 50, 60)).astype(np.uint8)).cuda()
    mask = np.ones((5, 5), np.uint8)
    off = torch.full((5, 5), 3, dtype=torch.int32, device="cuda")
    off[2, 3] = 9                                   # bound 7
    sev = M.SEDevView(mask, off, (2, 2), 7)
    ctx.morph_dev_se(0, f, 64, sev)
    with pytest.raises(M.MorphError) as ei:
        ctx.check()
    assert ei.value.status == M.MORPH_E_RANGE


@pytest.mark.parametrize("op", [0, 1])
def test_backward_equals_the_host_se_backward(ctx, op):
    from paper_2305_03018_gb300 import morph as M
    g = wl.rng(920 + op)
    L = 32
    f = g.integers(0, L, size=(4, 60, 70)).astype(np.uint8)
    se = wl.se_full_random(g, 9, 7)
    ft = torch.from_numpy(f).cuda()
    off = torch.from_numpy(se.offset.astype(np.int32)).cuda()
    sev = M.SEDevView(se.mask, off, se.origin, 7)
    D, cD = ctx.morph_dev_se(op, ft, L, sev, count=True)
    up = torch.from_numpy(g.standard_normal(f.shape).astype(np.float32)).cuda()
    img = M.make_image(ft, L)
    res = []
    for dev in (True, False):
        gin = torch.empty(f.shape, dtype=torch.float32, device="cuda")
        gse = torch.empty((9, 9), dtype=torch.float32, device="cuda")
        st = M.current_stream_handle(ft.device)
        if dev:
            fn = M.morph_dilate_backward_dev_se if op == 0 else M.morph_erode_backward_dev_se
            M.check(fn(ctx.handle, img, sev.c, D.data_ptr(), cD.data_ptr(), up.data_ptr(), gin.data_ptr(),
                       gse.data_ptr(), st), "backward_dev_se")
        else:
            sv = M.se_view(se)
            fn = M.morph_dilate_backward if op == 0 else M.morph_erode_backward
            M.check(fn(ctx.handle, img, sv.c, D.data_ptr(), cD.data_ptr(), up.data_ptr(), gin.data_ptr(),
                       gse.data_ptr(), st), "backward")
        ctx.check()
        res.append((gin.cpu().numpy(), gse.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_layer_with_a_bound_equals_the_host_copy_path(ctx):
    from paper_2305_03018_gb300.autograd import dilate, erode
    c = wl.c4_layer(batch=4, size=64)
    grads = []
    for bound in (7, None):
        x = torch.from_numpy(c.x).cuda().requires_grad_(True)
        b = torch.from_numpy(c.b).cuda().requires_grad_(True)
        up = torch.from_numpy(c.g).cuda()
        y = dilate(x, b, c.L, None, c.origin, max_offset=bound) + erode(x, b, c.L, None, c.origin, max_offset=bound)
        y.backward(up)
        torch.cuda.synchronize()
        grads.append((y.detach().cpu().numpy(), x.grad.cpu().numpy(), b.grad.cpu().numpy()))
    for a, b2 in zip(grads[0], grads[1]):
        assert np.array_equal(a, b2)
    rD, _ = oracle.dilate(c.x.reshape(-1, 64, 64).astype(np.int32), c.L, np.ones((9, 9)), c.b.astype(np.int32),
                          c.origin, nthreads=0)
    rE, _ = oracle.erode(c.x.reshape(-1, 64, 64).astype(np.int32), c.L, np.ones((9, 9)), c.b.astype(np.int32),
                         c.origin, nthreads=0)
    assert np.array_equal(grads[0][0].reshape(-1, 64, 64), (rD + rE).astype(np.float32))
