"""Host logic of DP-owner sharding (paper_1606_07413_gb300.shard; Sec. 4.2
collectors) on CPU: two gloo ranks run the real exchange and stop rule over a
CPU stand-in for the device steps (a seeded random walk on 4096 states with
its own distinguished points, trails and table).  The sharded level must
queue exactly the merges one table over all walks queues: for every
distinguished point, the same set of trails reached it."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

DOMAIN, DP_MOD, MAX_LEN = 4096, 16, 200


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class ToyEngine:
    """A seeded random function on DOMAIN states stands in for f; a point is
    distinguished when it is 0 mod DP_MOD; a trail of (walk, seq) starts at a
    seeded state; the table keeps the newest trail per point (no capacity
    limit) and queues a merge when a point arrives from another trail."""

    def __init__(self, n_owners):
        rng = np.random.default_rng(5)
        self.f = rng.integers(0, DOMAIN, DOMAIN)
        self.n_owners = n_owners
        self.table, self.merges = {}, []

    def start(self, walk, seq):
        return int(np.random.default_rng(1000003 * walk + seq).integers(0, DOMAIN))

    def begin(self, k, version, dp_bits, walk_base, total_walks):
        self.walks = {}
        for w in range(walk_base, walk_base + (total_walks // self.n_owners if self.n_owners else total_walks)):
            self.walks[w] = [self.start(w, 1), 1, 0]  # cur, seq, len
        self.table, self.merges = {}, []

    def owner(self, dp):
        return (dp * 2654435761 >> 7) % self.n_owners

    def walk_and_bin(self, steps):
        out = []
        for w, st in self.walks.items():
            for _ in range(steps):
                y = int(self.f[st[0]])
                st[2] += 1
                if y % DP_MOD == 0:
                    out.append((y, (w << 40) | (st[1] << 20) | st[2]))
                    st[1] += 1
                    st[0], st[2] = self.start(w, st[1]), 0
                elif st[2] >= MAX_LEN:
                    st[1] += 1
                    st[0], st[2] = self.start(w, st[1]), 0
                else:
                    st[0] = y
        out.sort(key=lambda p: self.owner(p[0]))
        counts = [sum(1 for p in out if self.owner(p[0]) == r) for r in range(self.n_owners)]
        pts = torch.tensor(out, dtype=torch.int64).reshape(-1, 2)
        return pts, counts, 0

    def insert(self, points):
        for dp, ref in points.tolist():
            old = self.table.get(dp)
            self.table[dp] = ref
            if old is not None and old != ref:
                self.merges.append((old, ref, dp))

    def rewalk_collect(self):
        return {"status_name": "searching", "merges": len(self.merges)}


def merge_groups(merges):
    groups = {}
    for a, b, dp in merges:
        groups.setdefault(dp, set()).update((a, b))
    return {dp: frozenset(s) for dp, s in groups.items()}


def _rank_main(rank, world, port, walks, rounds, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1606_07413_gb300 import shard

    eng = ToyEngine(world)
    lvl = shard.ShardedLevel(eng, walks)
    lvl.begin(3)
    received = 0
    for _ in range(rounds):
        r = lvl.round(steps)
        received += r["received"]
    mine = merge_groups(eng.merges)
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, received, sorted(eng.table)))
    out.put((rank, gathered))
    dist.destroy_process_group()


def test_two_ranks_queue_the_merges_of_one_table():
    world, walks, rounds, steps = 2, 48, 6, 25
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, walks, rounds, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = results[0]
    # one table over all walks, same trails, every round's points in one insert
    ref = ToyEngine(1)
    ref.begin(3, 0, 0, 0, world * walks)
    emitted = 0
    for _ in range(rounds):
        pts, _, _ = ref.walk_and_bin(steps)
        emitted += pts.shape[0]
        ref.insert(pts)
    want = merge_groups(ref.merges)
    got = {}
    for groups, _, _ in gathered:
        assert not set(got) & set(groups)  # each point is owned by one rank
        got.update(groups)
    assert got == want and len(want) > 10
    # every distinguished point was stored by exactly its owner
    tables = [set(t) for _, _, t in gathered]
    assert not tables[0] & tables[1] and tables[0] | tables[1] == set(ref.table)
    # the all-to-all delivered every point reached, once
    assert sum(r for _, r, _ in gathered) == emitted


def test_exchange_sends_each_group_to_its_rank():
    """exchange() alone with one rank: the points come back unchanged."""
    from paper_1606_07413_gb300 import shard

    port = _free_port()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        pts = torch.arange(10, dtype=torch.int64).reshape(5, 2)
        got = shard.exchange(pts, [5])
        assert torch.equal(got, pts)
    finally:
        dist.destroy_process_group()
