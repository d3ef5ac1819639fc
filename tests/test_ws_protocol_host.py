"""A model of the hand-off protocol of the n = 4 tensor-core walk
(k_walks_mma4), checked under random interleavings of its warps on the CPU.

The model mirrors the kernel's control flow:
- 12 stage warps and 8 MMA warps;
- the walk sets (the kernel runs two; three are checked too), whose "rows ready" and "sums ready" mbarriers complete a
  phase when every expected warp has arrived, and whose waiters wait on a
  phase parity;
- the stage warps' single-producer rings of distinguished points, drained by
  their owning MMA warps (ring r by MMA warp r % 8) while those wait for rows
  and after their last product, until every producer is done; a full ring
  makes the producer store the point itself.

Properties checked for many random schedules and sizes:
- every warp finishes: no deadlock;
- no barrier ever runs two phases ahead of a waiter, so a parity wait cannot
  alias;
- every distinguished point a stage warp finds is stored exactly once.
"""
import random

import pytest

STAGE, MMA = 12, 8


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0  # phase: completed phases

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):
        # the phase of this parity has completed (the next one has begun)
        return self.phase % 2 != parity


class Ring:
    def __init__(self, cap):
        self.cap, self.items, self.head, self.tail, self.done = cap, [], 0, 0, False


def stage_warp(wi, st, groups, steps, dp_prob, rng):
    """Generator of one stage warp: yields ("wait", predicate) to block."""
    SETS = st["sets"]
    ph = [0] * SETS
    ring = st["rings"][wi]
    for _ in range(groups):
        def phase_a(x):
            st["rows"][x].arrive()
        def phase_c(x):
            for _ in range(2):  # two walks of each set
                if rng.random() < dp_prob:
                    st["found"] += 1
                    pid = st["found"]
                    if ring.tail - ring.head < ring.cap:
                        ring.items.append(pid)
                        ring.tail += 1
                    else:
                        st["stored"].append(pid)  # the ring is full: store it here
        if steps > 0:
            for x in range(SETS):
                phase_a(x)
                yield ("run", None)
        for step in range(steps):
            for x in range(SETS):
                b = st["sums"][x]
                p = ph[x]
                st["ahead"] = max(st["ahead"], b.phase - st["sums_seen"][wi][x])
                yield ("wait", lambda b=b, p=p: b.done(p))
                st["sums_seen"][wi][x] += 1
                ph[x] ^= 1
                phase_c(x)
                yield ("run", None)
                if step + 1 < steps:
                    phase_a(x)
                    yield ("run", None)
    ring.done = True


def mma_warp(m, st, groups, steps):
    SETS = st["sets"]
    ph = [0] * SETS
    owned = [st["rings"][r] for r in (m, m + MMA) if r < STAGE]

    def drain(most):
        moved = False
        for ring in owned:
            k = 0
            while ring.head != ring.tail and k < most:
                st["stored"].append(ring.items[ring.head])
                ring.head += 1
                k += 1
                moved = True
        return moved

    for _ in range(groups):
        for _ in range(steps):
            for x in range(SETS):
                b = st["rows"][x]
                p = ph[x]
                st["ahead"] = max(st["ahead"], b.phase - st["rows_seen"][m][x])
                while not b.done(p):
                    drain(1)  # store points while waiting for the set's rows
                    yield ("wait_or_drain", lambda b=b, p=p: b.done(p) or any(r.head != r.tail for r in owned))
                st["rows_seen"][m][x] += 1
                ph[x] ^= 1
                yield ("run", None)  # the set's products
                st["sums"][x].arrive()
    # after the last product: drain until every owned producer is done and empty
    while not all(r.done and r.head == r.tail for r in owned):
        if not drain(64):
            yield ("wait_or_drain", lambda: all(r.done and r.head == r.tail for r in owned)
                   or any(r.head != r.tail for r in owned))


def model_state(sets, ring_cap, rows_count=STAGE):
    return {"sets": sets, "rows": [Barrier(rows_count) for _ in range(sets)],
            "sums": [Barrier(MMA) for _ in range(sets)], "rings": [Ring(ring_cap) for _ in range(STAGE)],
            "found": 0, "stored": [], "ahead": 0, "sums_seen": [[0] * sets for _ in range(STAGE)],
            "rows_seen": [[0] * sets for _ in range(MMA)]}


def run_model(seed, sets, groups, steps, dp_prob, ring_cap, max_events=2_000_000):
    rng = random.Random(seed)
    st = model_state(sets, ring_cap)
    warps = [stage_warp(i, st, groups, steps, dp_prob, random.Random(rng.random())) for i in range(STAGE)]
    warps += [mma_warp(m, st, groups, steps) for m in range(MMA)]
    blocked = {}  # warp index -> predicate
    live = set(range(len(warps)))
    events = 0
    while live:
        runnable = [i for i in live if i not in blocked or blocked[i]()]
        assert runnable, "deadlock: every live warp waits"
        i = rng.choice(runnable)
        blocked.pop(i, None)
        try:
            kind, pred = next(warps[i])
        except StopIteration:
            live.discard(i)
            continue
        if kind != "run":
            blocked[i] = pred
        events += 1
        assert events < max_events, "no progress"
    return st


@pytest.mark.parametrize("sets", [2, 3])
@pytest.mark.parametrize("seed", range(12))
def test_protocol_finishes_and_stores_every_point_once(seed, sets):
    rng = random.Random(1000 + seed)
    groups = rng.choice([0, 1, 2, 3])
    steps = rng.choice([0, 1, 2, 5, 9])
    dp_prob = rng.choice([0.0, 0.05, 0.25, 0.5, 1.0])
    ring_cap = rng.choice([1, 2, 64])
    st = run_model(seed, sets, groups, steps, dp_prob, ring_cap)
    # every phase every waiter waited for completed exactly once per step and set
    for b in st["rows"] + st["sums"]:
        assert b.phase == groups * steps
    assert st["ahead"] <= 1  # a barrier never ran two phases ahead of a waiter
    assert sorted(st["stored"]) == list(range(1, st["found"] + 1))


def test_a_missing_arrival_is_a_deadlock_the_model_sees():
    """The checker itself: with one stage warp's arrival count too high, the
    rows barrier never completes and the model reports the deadlock (on the
    GPU, the bounded waits would give up and the launch report a stall)."""
    rng = random.Random(5)
    st = model_state(3, 64, rows_count=STAGE + 1)
    warps = [stage_warp(i, st, 1, 2, 0.1, random.Random(i)) for i in range(STAGE)]
    warps += [mma_warp(m, st, 1, 2) for m in range(MMA)]
    blocked, live = {}, set(range(len(warps)))
    with pytest.raises(AssertionError, match="deadlock"):
        while live:
            runnable = [i for i in live if i not in blocked or blocked[i]()]
            assert runnable, "deadlock: every live warp waits"
            i = rng.choice(runnable)
            blocked.pop(i, None)
            try:
                kind, pred = next(warps[i])
            except StopIteration:
                live.discard(i)
                continue
            if kind != "run":
                blocked[i] = pred
