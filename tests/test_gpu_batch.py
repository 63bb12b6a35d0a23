"""GPU batches (one persistent launch for the FP8 route, graph capture)
against the oracle."""
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


def _items(probs):
    items, outs = [], []
    for p in probs:
        ft = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
        o = torch.full(ft.shape, -99, dtype=torch.int32, device="cuda")
        c = torch.full(ft.shape, -99, dtype=torch.int32, device="cuda")
        items.append((ft, p.L, p.se, p.op, o, c))
        outs.append((o, c))
    return items, outs


def _check(p, o, c, rows=None):
    fn = oracle.dilate if p.op == "dilate" else oracle.erode
    H = p.f.shape[1]
    r = rows if rows is not None else (0, H)
    D, cD = fn(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, rows=r, nthreads=0)
    got_d = o.cpu().numpy()[:, r[0]:r[1]]
    got_c = c.cpu().numpy()[:, r[0]:r[1]]
    assert np.array_equal(got_d, D[:, r[0]:r[1]]), p.name
    assert np.array_equal(got_c, cD[:, r[0]:r[1]]), p.name


def test_small_heterogeneous_batch(ctx):
    probs = wl.c5_batch(n=24, seed=55, max_side=160)
    items, outs = _items(probs)
    ctx.run_batch(items, method="direct_fp8")
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)


def test_auto_batch_mixes_routes(ctx):
    probs = wl.c5_batch(n=16, seed=56, max_side=120)
    probs.append(wl.Problem(wl.uniform_image(wl.rng(1), (1, 90, 70), 16), 16, wl.se_flat_square(3), "erode", "tiny"))
    items, outs = _items(probs)
    ctx.run_batch(items, method="auto")
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)


def test_captured_graph_replays_current_inputs(ctx):
    probs = wl.c5_batch(n=12, seed=57, max_side=140)
    items, outs = _items(probs)
    b = ctx.capture_batch(items, method="direct_fp8")
    b.launch()
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)
    # new pixel values in the same buffers: the replay must see them
    g = wl.rng(58)
    for p, it in zip(probs, items):
        p.f = g.integers(0, p.L, size=p.f.shape).astype(p.f.dtype)
        it[0].copy_(torch.from_numpy(p.f))
    b.launch()
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)
    b.close()


@pytest.fixture(scope="module")
def c5():
    probs = wl.c5_batch()                       # 512 problems, sides up to 1024
    refs = []
    for p in probs:
        fn = oracle.dilate if p.op == "dilate" else oracle.erode
        refs.append(fn(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, nthreads=0))
    return probs, refs


@pytest.mark.parametrize("method", ["auto", "direct_fp8"])
def test_c5_full_batch_every_pixel(ctx, c5, method):
    # all 512 problems in one captured graph; every pixel's value and top count of
    # every problem against the oracle
    probs, refs = c5
    items, outs = _items(probs)
    b = ctx.capture_batch(items, method=method)
    b.launch()
    ctx.check()
    for p, (o, c), (rD, rC) in zip(probs, outs, refs):
        assert np.array_equal(o.cpu().numpy(), rD), p.name
        assert np.array_equal(c.cpu().numpy(), rC), p.name
    b.close()


@pytest.mark.parametrize("method", ["ntt", "fft_f64"])
def test_transform_batch_on_branch_streams(ctx, method):
    # many transform-route problems: they are spread over branch streams that fork
    # from and join into the caller's stream (run) or become parallel graph branches
    # (capture); each branch has its own workspace slice
    g = wl.rng(59 if method == "ntt" else 60)
    probs = []
    for k in range(9):
        h, w = int(g.integers(20, 140)), int(g.integers(20, 160))
        L = [16, 64, 256][k % 3]
        f = g.integers(0, L, size=(1, h, w)).astype(np.uint8)
        se = wl.se_random(g, int(g.integers(1, 12)), int(g.integers(1, 12)), 0.7, int(g.integers(0, 9)))
        probs.append(wl.Problem(f, L, se, "dilate" if k % 2 else "erode", f"b{k}"))
    items, outs = _items(probs)
    ctx.run_batch(items, method=method)
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)
    for o, c in outs:
        o.fill_(-99)
        c.fill_(-99)
    b = ctx.capture_batch(items, method=method)
    b.launch()
    b.launch()
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)
    b.close()


def test_autotuned_routes_are_exact_and_cached(ctx):
    # measured route choice: every timed candidate writes the same exact result,
    # and the choice is cached for later AUTO calls with or without the flag
    g = wl.rng(61)
    cases = [(1, 200, 180, 256, 15, 200), (1, 300, 256, 16, 9, 3), (2, 90, 70, 64, 31, 7)]
    for (n, h, w, L, k, mo) in cases:
        f = g.integers(0, L, size=(n, h, w)).astype(np.uint8)
        se = wl.se_full_random(g, k, mo)
        ft = torch.from_numpy(f).cuda()
        out, cnt = ctx.dilate(ft, L, se, method="auto", count=True, autotune=True)
        ctx.check()
        D, cD = oracle.dilate(f, L, se.mask, se.offset, se.origin, nthreads=0)
        assert np.array_equal(out.cpu().numpy(), D) and np.array_equal(cnt.cpu().numpy(), cD)
        tuned = ctx.plan(ft, L, se, method="auto").method
        assert tuned in (1, 2, 3, 4)
        out2 = ctx.dilate(ft, L, se, method="auto")
        ctx.check()
        assert np.array_equal(out2.cpu().numpy(), D)


def test_autotuned_capture_is_exact(ctx):
    probs = wl.c5_batch(n=16, seed=62, max_side=200)
    items, outs = _items(probs)
    b = ctx.capture_batch(items, method="auto", autotune=True)
    b.launch()
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check(p, o, c)
    b.close()
