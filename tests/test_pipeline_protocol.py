"""CPU checks of the FP8 direct kernel's index math and stage protocol.

These restate, on the host, the schedule `k_direct_fp8` follows, and check
its invariants for every window width the planner can produce:

* split two-tile units: K step ks of tile tt (shift tt J bytes) reads B block
  (32 ks + tt J) / 128 inside one 128-byte row, and its A block ks / 4 is the
  block staged with that B block or the one before; every (tile, K step) pair
  is issued exactly once, and the row stages ceil((J + 32 ksteps) / 128)
  blocks;
* the stage ring (STAGES slots, the library's own ring depth, one "landed" and
  one "consumed" barrier each), and the unit queue through which the producer
  hands each unit to the MMA issuer and the epilogue:
  with split units a stage is released after the next stage's MMAs.  A
  random-interleaving model of the producer, the MMA issuer and the
  asynchronous releases never deadlocks and never lets the producer refill
  a slot whose data an issued MMA still reads, for any mix of unit kinds in
  one persistent launch.
"""
import random

import pytest

def _ring_stages(kw=3, L=16, side=64, levels=1):
    """The direct kernel's ring depth as the library reports it (host-only plan query) for a
    kw x kw SE with `levels` offset levels: two-tile units for a small SE with several levels,
    one-tile units for a wide flat one."""
    import ctypes

    import numpy as np

    from paper_2305_03018_gb300 import morph as M
    from paper_2305_03018_gb300 import workloads as wl
    buf = ctypes.create_string_buffer(16)
    im = M.morph_image()
    im.data = ctypes.addressof(buf)
    im.dtype = M.MORPH_U8
    im.n, im.h, im.w, im.row_stride, im.batch_stride, im.L = 1, side, side, side, side * side, L
    se = wl.se_flat_square(kw) if levels == 1 else wl.se_full_random(wl.rng(1), kw, levels - 1)
    sv = M.se_view(se)
    info = M.morph_plan_query(None, im, sv.c, 0, M.make_opts("direct_fp8"))
    return info.ring_stages, info.unit_tiles


_STAGES = []


def _stage_depths():
    """The ring depths of the kernel's unit kinds (two-tile and one-tile units)."""
    if not _STAGES:
        d2, t2 = _ring_stages(9, 64, 256, levels=8)
        d1, t1 = _ring_stages(63, 64, 2048)
        assert (t2, t1) == (2, 1)
        _STAGES.extend(sorted({d1, d2}))
    return list(_STAGES)


def _stages():
    return min(_stage_depths())


def _unit_queue():
    """The direct kernel's unit-queue depth as the library reports it."""
    import ctypes

    from paper_2305_03018_gb300 import morph as M
    from paper_2305_03018_gb300 import workloads as wl
    buf = ctypes.create_string_buffer(16)
    im = M.morph_image()
    im.data = ctypes.addressof(buf)
    im.dtype = M.MORPH_U8
    im.n, im.h, im.w, im.row_stride, im.batch_stride, im.L = 1, 64, 64, 64, 64 * 64, 16
    sv = M.se_view(wl.se_flat_square(3))
    return M.morph_plan_query(None, im, sv.c, 0, M.make_opts("direct_fp8")).unit_queue


def split_schedule(J, ksteps):
    """(stage kc, tile tt, K step ks, A block, B byte offset) in issue order."""
    nb = (J + 32 * ksteps + 127) // 128
    sh1 = J // 32
    out = []
    for kc in range(nb):
        for tt in range(2):
            sh = tt * sh1
            for ks in range(max(0, 4 * kc - sh), min(ksteps, 4 * kc + 4 - sh)):
                out.append((kc, tt, ks, ks // 4, 32 * ((ks + sh) % 4)))
    return nb, out


@pytest.mark.parametrize("J", [32, 64, 128])
def test_split_schedule_covers_each_k_step_once(J):
    for kw in range(1, 513):
        ksteps = (J + kw - 1 + 31) // 32
        nk = (J + kw - 1 + 127) // 128
        nb, sched = split_schedule(J, ksteps)
        assert nk <= nb <= nk + 1
        seen = set()
        for kc, tt, ks, ka, boff in sched:
            assert (tt, ks) not in seen
            seen.add((tt, ks))
            assert ka in (kc, kc - 1) and ka < nk          # staged now or one stage earlier
            pos = 32 * ks + tt * J                          # byte of the unit's K window
            assert pos // 128 == kc and pos % 128 == boff and boff + 32 <= 128
        assert seen == {(tt, ks) for tt in range(2) for ks in range(ksteps)}
        assert 32 * ksteps >= J + kw - 1                    # the window covers every tap column


def _ring_model(units, seed, STAGES=None):
    """units: (blocks per SE row, split) per row, in launch order."""
    STAGES = STAGES or _stages()
    rnd = random.Random(seed)
    program = [(r, kc) for r, (nb, _) in enumerate(units) for kc in range(nb)]
    slot = [None] * STAGES
    released = [0] * STAGES
    landed = [0]
    pending = []

    def issuer():
        it = 0
        for r, (nb, split) in enumerate(units):
            prev = None
            for kc in range(nb):
                s = it % STAGES
                while landed[0] <= it:
                    yield False
                assert slot[s] == (r, kc), "issuer read a refilled slot"
                if split and kc > 0:
                    assert slot[prev] == (r, kc - 1), "previous A block overwritten"
                if split:
                    if kc > 0:
                        pending.append(prev)
                    if kc == nb - 1:
                        pending.append(s)
                else:
                    pending.append(s)
                prev = s
                it += 1
                yield True

    gen, done, p, idle = issuer(), False, 0, 0
    while not (done and p == len(program) and not pending):
        moved = False
        c = rnd.random()
        if c < 0.4 and p < len(program):
            s = landed[0] % STAGES
            if released[s] >= landed[0] // STAGES:          # the slot's previous use was consumed
                slot[s] = program[p]
                landed[0] += 1
                p += 1
                moved = True
        elif c < 0.7 and pending:
            released[pending.pop(0)] += 1                   # an MMA batch completes
            moved = True
        elif not done:
            try:
                moved = next(gen)
            except StopIteration:
                done, moved = True, True
        idle = 0 if moved else idle + 1
        assert idle < 20000, "deadlock"
    assert sum(released) == landed[0]


def test_stage_ring_never_deadlocks_or_overwrites():
    rnd = random.Random(11)
    kinds = [(3, True), (2, True), (5, True), (1, False), (2, False), (3, False)]
    for trial in range(150):
        units = [rnd.choice(kinds) for _ in range(rnd.randint(1, 10))]
        for seed in range(4):
            for depth in _stage_depths():
                _ring_model(units, 97 * trial + seed, depth)


def _plan(kw, nlev, h=2048, w=2048):
    """The library's own host-side plan (no GPU) of a one-row SE of width kw
    with nlev offset levels, on an h x w image with L = 64."""
    import ctypes

    import numpy as np

    from paper_2305_03018_gb300 import morph as M
    from paper_2305_03018_gb300 import workloads as wl
    buf = ctypes.create_string_buffer(16)
    im = M.morph_image()
    im.data = ctypes.addressof(buf)
    im.dtype = M.MORPH_U8
    im.n, im.h, im.w = 1, h, w
    im.row_stride, im.batch_stride, im.L = w, h * w, 64
    m = np.ones((1, kw), np.uint8)
    off = (np.arange(kw) % nlev).astype(np.int32)[None]
    sv = M.se_view(wl.SE(m, off, (0, kw // 2)))
    return M.morph_plan_query(None, im, sv.c, 0, M.make_opts("direct_fp8"))


@pytest.mark.parametrize("nlev", [1, 2, 3, 5, 8])
def test_model_matches_the_library_plan(nlev):
    # the schedule above is checked against the (J, K steps, staged blocks, unit kind) that the
    # library itself plans, so the model cannot drift from the kernel's planner unnoticed
    kinds = []
    for kw in list(range(1, 70, 3)) + [100, 130, 200, 257, 400, 512]:
        info = _plan(kw, nlev)
        J, ks, nb, T = info.tile_w, info.k_steps, info.unit_blocks, info.unit_tiles
        # L = 64: units of 32 image rows x 8-level chunks (64 x 4 where an accumulation has enough
        # MMAs, which a one-row SE never has), 8 of them when a band holds every level
        assert info.groups * J == 128 and info.tile_h == 32 and info.level_chunks == 8
        assert ks == (J + kw - 1 + 31) // 32
        nk = (J + kw - 1 + 127) // 128
        split = T == 2 and J + kw - 1 > 128
        if split:
            got_nb, sched = split_schedule(J, ks)
            assert got_nb == nb < 2 * nk and J >= 32
            assert {(tt, k) for _, tt, k, _, _ in sched} == {(tt, k) for tt in range(2) for k in range(ks)}
        elif T == 2:
            assert 2 * J + kw - 1 <= 128 and J + 32 * ks <= 128 and nb == nk == 1
        else:
            assert nb == nk
        kinds.append((nb, split))
    for seed in range(6):
        _ring_model(kinds, seed)


# ------------------------------------------------------------------ abort path
def _abort_model(n_units, blocks_per_unit, seed, inject_p, always_drain=True, STAGES=None):
    """The three roles of k_direct_fp8 (one tile per unit, accumulator slots used
    alternately) with one injected wait timeout at a random blocked wait.  The
    producer publishes each unit (then -1) through the unit queue, whose slot is
    free again once the MMA issuer and the epilogue have both read it.  Waits
    fail once the CTA's abort flag is up.  Copies land in any order; MMA batches
    complete in issue order, each then arriving on its barrier.  Returns the
    copies and MMA batches still in flight when all roles reach the final barrier
    (after which TMEM is freed and the CTA exits), or raises on a deadlock."""
    STAGES, Q = STAGES or _stages(), _unit_queue()
    rnd = random.Random(seed)
    st = {"abort": False, "injected": False}
    landed = set()            # copy ids that have landed
    inflight_copies = set()
    mma_q = []                # in-flight MMA batches: ("empty", slot) / ("tfull", slot) / ("drain",)
    released = [0] * STAGES   # empty-barrier phases completed per stage slot
    tfull = [0, 0]            # accumulator-full arrivals per TMEM slot
    tempty = [0, 0]           # accumulator-free arrivals per TMEM slot (epilogue)
    drained = [False]
    ufull = [0] * Q           # units published per queue slot
    uread = [0] * Q           # reader arrivals per queue slot (two per publication)
    uval = [None] * Q

    def wait(cond):
        while not cond():
            if st["abort"]:
                return False
            if not st["injected"] and rnd.random() < inject_p:
                st["injected"] = st["abort"] = True      # this wait reached its limit
                return False
            yield None
        return True

    def read_unit(uq):
        q = uq % Q
        ok = yield from wait(lambda: ufull[q] > uq // Q)
        if not ok:
            return False, None
        t = uval[q]
        assert t == (uq if uq < n_units else -1), "a reader saw another publication of the slot"
        uread[q] += 1
        return True, t

    def producer():
        it, ok = 0, True
        for u in range(n_units + 1):
            q = u % Q
            ok = yield from wait(lambda: uread[q] >= 2 * (u // Q))
            if not ok:
                break
            uval[q] = u if u < n_units else -1
            ufull[q] += 1
            if u == n_units:
                break
            for kc in range(blocks_per_unit):
                s = it % STAGES
                ok = yield from wait(lambda: released[s] >= it // STAGES)
                if not ok:
                    break
                inflight_copies.add(it)
                it += 1
            if not ok:
                break
        if always_drain or not ok:
            for k in range(max(0, it - STAGES), it):
                while k in inflight_copies:
                    yield None

    def mma():
        it, use, nxt, ok, uq = 0, [0, 0], 0, True, 0
        while True:
            ok, t = yield from read_unit(uq)
            uq += 1
            if not ok or t < 0:
                break
            s0, nxt = nxt, nxt ^ 1
            ok = yield from wait(lambda: tempty[s0] >= use[s0])
            if not ok:
                break
            for kc in range(blocks_per_unit):
                k = it
                ok = yield from wait(lambda: k in landed)
                if not ok:
                    break
                mma_q.append(("empty", k % STAGES))
                it += 1
            if not ok:
                break
            mma_q.append(("tfull", s0))
            use[s0] += 1
        if always_drain or not ok:
            mma_q.append(("drain",))
            while not drained[0]:
                yield None

    def epilogue():
        use, nxt, uq = [0, 0], 0, 0
        while True:
            ok, t = yield from read_unit(uq)
            uq += 1
            if not ok or t < 0:
                break
            s0, nxt = nxt, nxt ^ 1
            ok = yield from wait(lambda: tfull[s0] > use[s0])
            if not ok:
                break
            tempty[s0] += 1
            use[s0] += 1

    roles = [producer(), mma(), epilogue()]
    done = [False] * 3
    steps = 0
    while not all(done):
        steps += 1
        assert steps < 200000, "deadlock"
        c = rnd.random()
        if c < 0.25 and inflight_copies:
            k = rnd.choice(sorted(inflight_copies))       # a copy lands
            inflight_copies.discard(k)
            landed.add(k)
        elif c < 0.45 and mma_q:
            ev = mma_q.pop(0)                             # the oldest MMA batch completes
            if ev[0] == "empty":
                released[ev[1]] += 1
            elif ev[0] == "tfull":
                tfull[ev[1]] += 1
            else:
                drained[0] = True
        else:
            r = rnd.randrange(3)
            if not done[r]:
                try:
                    next(roles[r])
                except StopIteration:
                    done[r] = True
    if not st["abort"]:
        assert tempty == tfull and sum(tfull) == n_units, "a unit was not completed"
    return len(inflight_copies), len(mma_q)


def test_abort_drains_every_copy_and_mma_before_exit():
    # a timeout at any wait of any role: when all roles meet at the final barrier, no TMA copy
    # can still land in shared memory and no MMA can still write TMEM
    hits = 0
    for trial in range(600):
        n_units = 1 + trial % 9                 # up to twice the unit queue
        blocks = 1 + (trial // 9) % 4
        for depth in _stage_depths():
            copies, mmas = _abort_model(n_units, blocks, trial, inject_p=0.02, STAGES=depth)
            assert copies == 0 and mmas == 0, (trial, depth, copies, mmas)
        assert copies == 0 and mmas == 0, (trial, copies, mmas)
        hits += 1
    assert hits == 600


def test_unit_queue_completes_every_unit_without_a_timeout():
    # no injected timeout: every unit passes through the queue and the accumulators, in any
    # interleaving, and nothing is in flight at the end
    for trial in range(300):
        copies, mmas = _abort_model(1 + trial % 12, 1 + trial % 3, 7000 + trial, inject_p=0.0)
        assert copies == 0 and mmas == 0


def test_abort_model_catches_a_drain_taken_only_by_the_role_that_failed():
    # planted mistake, on the CPU: drain only when this role's own wait failed.  When the
    # epilogue gives up after the MMA issuer has run to its end, MMAs are still in flight at
    # the final barrier, which the model must see
    found = False
    for trial in range(3000):
        copies, mmas = _abort_model(2 + trial % 3, 1 + trial % 2, trial, inject_p=0.05, always_drain=False)
        if copies or mmas:
            found = True
            break
    assert found
