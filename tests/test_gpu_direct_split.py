"""GPU parity of the FP8 direct route's split two-tile units against the oracle.

A split unit holds two horizontally adjacent tiles of J output columns whose
K windows (J + kw - 1 image columns each) do not fit one 128-byte block
together: tile 1 reads the same staged B blocks as tile 0 shifted by J bytes.
The cases cover J = 64 and 32 (two and four offset groups), ragged right edges
where tile 1 of the last unit lies partly or wholly outside the image,
erosion, and a batch that mixes unit kinds in one launch.  With J = 128 (one
group) and L > 16 the two tiles' running results of 32 or 64 image rows would
overflow the kernel's per-unit buffer, so those windows run as single-tile
units, also checked here.
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


def _run(ctx, f, L, se, op):
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    fn = ctx.dilate if op == "dilate" else ctx.erode
    out, cnt = fn(ft, L, se, method="direct_fp8", count=True)
    ctx.check()
    return out.cpu().numpy(), cnt.cpu().numpy()


def _check(got, f, L, se, op, rows=None):
    fn = oracle.dilate if op == "dilate" else oracle.erode
    H = f.shape[1]
    r = rows if rows is not None else (0, H)
    D, cD = fn(f, L, se.mask, se.offset, se.origin, rows=r, nthreads=0)
    for a, b in zip(got, (D, cD)):
        a, b = a[:, r[0]:r[1]], b[:, r[0]:r[1]]
        bad = np.argwhere(a != b)
        assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:3].tolist()}"


def _unit(ctx, f, L, se, op=0):
    info = ctx.plan(torch.from_numpy(np.ascontiguousarray(f)).cuda(), L, se, op=op, method="direct_fp8")
    return info.groups, info.tile_w, info.unit_tiles, info.unit_blocks


# (name, shape, L, SE factory, expected (groups, J, unit tiles, staged blocks per SE row))
CASES = [
    ("J128 flat 9x9, single tiles", (2, 600, 700), 64, lambda g: wl.se_flat_square(9), (1, 128, 1, 2)),
    ("J128 flat 9x9, ragged", (4, 300, 600), 64, lambda g: wl.se_flat_square(9), (1, 128, 1, 2)),
    ("J64 two levels, kw 95", (2, 1600, 1000), 32, lambda g: wl.se_random(g, 3, 95, 0.7, 1, origin=(1, 40)),
     (2, 64, 2, 2)),
    ("J32 four levels, kw 99", (1, 160, 2000), 16, lambda g: wl.se_random(g, 3, 99, 0.7, 3, origin=(2, 70)),
     (4, 32, 2, 2)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_split_units_bit_exact(ctx, case):
    name, shape, L, mk, expect = case
    g = wl.rng(510 + [c[0] for c in CASES].index(name))
    f = g.integers(0, L, size=shape).astype(np.uint8)
    se = mk(g)
    assert _unit(ctx, f, L, se) == expect
    for op in ("dilate", "erode"):
        _check(_run(ctx, f, L, se, op), f, L, se, op)


def test_disk_radius_31_single_tiles(ctx):
    # the flat disk of the 2048 x 2048 workload on a smaller image: one 128-column tile per
    # unit, two 128-byte blocks per SE row
    g = wl.rng(501)
    f = g.integers(0, 64, size=(2, 160, 1000)).astype(np.uint8)
    se = wl.se_flat_disk(31)
    assert _unit(ctx, f, 64, se) == (1, 128, 1, 2)
    for op in ("dilate", "erode"):
        got = _run(ctx, f, 64, se, op)
        for rows in ((0, 40), (120, 160)):
            _check(got, f, 64, se, op, rows=rows)


def test_no_split_where_it_would_not_pay_or_fit(ctx):
    g = wl.rng(502)
    se = wl.se_flat_square(9)
    # L = 16, 600 x 700: fewer than two waves of two-tile units on 152 SMs
    f16 = g.integers(0, 16, size=(2, 600, 700)).astype(np.uint8)
    assert _unit(ctx, f16, 16, se)[2:] == (1, 2)
    # fewer than two waves of units on 152 SMs
    fs = g.integers(0, 64, size=(1, 64, 300)).astype(np.uint8)
    assert _unit(ctx, fs, 64, se)[2:] == (1, 2)
    for f, L in ((f16, 16), (fs, 64)):
        for op in ("dilate", "erode"):
            _check(_run(ctx, f, L, se, op), f, L, se, op, rows=(0, 64))


def test_batch_mixes_unit_kinds(ctx):
    # one persistent launch whose problems use split, packed and single-tile units
    g = wl.rng(503)
    probs = [
        wl.Problem(g.integers(0, 64, size=(2, 600, 700)).astype(np.uint8), 64, wl.se_flat_square(9), "dilate",
                   "single J128"),
        wl.Problem(g.integers(0, 64, size=(1, 200, 300)).astype(np.uint8), 64, wl.se_full_random(g, 15, 7),
                   "erode", "packed"),
        wl.Problem(g.integers(0, 16, size=(1, 100, 500)).astype(np.uint8), 16, wl.se_flat_square(9), "dilate",
                   "single"),
        wl.Problem(g.integers(0, 32, size=(2, 1600, 1000)).astype(np.uint8), 32,
                   wl.se_random(g, 3, 95, 0.7, 1, origin=(1, 40)), "erode", "split J64"),
    ]
    kinds = [_unit(ctx, p.f, p.L, p.se, 0 if p.op == "dilate" else 1)[2:] for p in probs]
    assert kinds == [(1, 2), (2, 1), (1, 2), (2, 2)]
    items, outs = [], []
    for p in probs:
        ft = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
        o = torch.full(ft.shape, -99, dtype=torch.int32, device="cuda")
        c = torch.full(ft.shape, -99, dtype=torch.int32, device="cuda")
        items.append((ft, p.L, p.se, p.op, o, c))
        outs.append((o, c))
    ctx.run_batch(items, method="direct_fp8")
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        _check((o.cpu().numpy(), c.cpu().numpy()), p.f, p.L, p.se, p.op, rows=(0, 100))
