"""CPU checks of the FP8 direct kernel's index math and stage protocol.

These restate, on the host, the schedule `k_direct_fp8` follows, and check
its invariants for every window width the planner can produce:

* split two-tile units: K step ks of tile tt (shift tt J bytes) reads B block
  (32 ks + tt J) / 128 inside one 128-byte row, and its A block ks / 4 is the
  block staged with that B block or the one before; every (tile, K step) pair
  is issued exactly once, and the row stages ceil((J + 32 ksteps) / 128)
  blocks;
* the stage ring (4 slots, one "landed" and one "consumed" barrier each):
  with split units a stage is released after the next stage's MMAs.  A
  random-interleaving model of the producer, the MMA issuer and the
  asynchronous releases never deadlocks and never lets the producer refill
  a slot whose data an issued MMA still reads, for any mix of unit kinds in
  one persistent launch.
"""
import random

import pytest

STAGES = 4


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


def _ring_model(units, seed):
    """units: (blocks per SE row, split) per row, in launch order."""
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
            _ring_model(units, 97 * trial + seed)
