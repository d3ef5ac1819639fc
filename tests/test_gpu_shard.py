"""DP-owner sharding on the device (Sec. 4.2 collectors), with two ranks
emulated in one process on one GPU: each "rank" is a problem walking its
half of the global walks with its distinguished points sent to an outbox,
the outboxes are grouped by owner (qcs_shard_bin), each group goes to its
owner's table (qcs_level_insert).  No kernel waits on another, so the ranks
run one after the other.  The merges the two tables queue must be those one
table over all walks queues: for every distinguished point, the same set of
trails (the ranks walk the very trails of the single table, since trails are
named by their global walk index).  Also the whole ShardedLevel round on one
NCCL rank."""
import os
import socket

import numpy as np
import pytest

import paper_1606_07413_gb300 as Q
from paper_1606_07413_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, VERSION, DPB, STEPS, WALKS = 4, 3, 4, 32, 2048


def groups_of(merges):
    g = {}
    for a, b, dp in merges.tolist():
        g.setdefault(dp, set()).update((a, b))
    return g


def make(walks):
    gates, _ = W.config_target(2)
    return Q.Problem.from_circuit(3, gates, 5, Q.default_params(3, walks=walks, table_log2=22))


def test_two_owner_tables_queue_the_merges_of_one_table():
    from paper_1606_07413_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    with make(2 * WALKS) as one:
        one.level_begin_shard(K, VERSION, DPB, 0, 2 * WALKS)
        one.level_walk(STEPS)
        want = groups_of(one.level_merges())
        one.level_rewalk()
        r_one = one.level_collect()
    assert r_one["dropped"] == 0 and len(want) > 20  # no point overwritten: the merge sets are complete

    ranks = [make(WALKS), make(WALKS)]
    try:
        binned, counts, reached = [], [], 0
        for r, prob in enumerate(ranks):
            prob.level_begin_shard(K, VERSION, DPB, r * WALKS, 2 * WALKS)
            outbox = torch.zeros(2 * 65536, dtype=torch.int64, device=dev)
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            prob.level_walk_out(STEPS, outbox, cnt)
            n = int(cnt.item())
            reached += n
            out = torch.zeros_like(outbox)
            oc = torch.zeros(4, dtype=torch.int32, device=dev)
            Q.shard_bin(outbox, n, 2, out, oc)
            c = oc[:2].tolist()
            assert sum(c) == n
            # binning permutes the points
            assert sorted(map(tuple, out[: 2 * n].view(-1, 2).tolist())) == \
                sorted(map(tuple, outbox[: 2 * n].view(-1, 2).tolist()))
            binned.append(out[: 2 * n].view(-1, 2))
            counts.append(c)
        assert reached == r_one["dps"]
        got, owner_of = {}, {}
        for owner, prob in enumerate(ranks):
            parts = []
            for src in range(2):
                lo = sum(counts[src][:owner])
                part = binned[src][lo: lo + counts[src][owner]]
                for dp in part[:, 0].tolist():
                    assert owner_of.setdefault(dp, owner) == owner  # one owner per point, on every rank
                parts.append(part)
            prob.level_insert(torch.cat(parts).contiguous())
            g = groups_of(prob.level_merges())
            assert not set(g) & set(got)
            got.update(g)
            prob.level_rewalk()
            r = prob.level_collect()
            assert r["dropped"] == 0
        assert got == want
    finally:
        for p in ranks:
            p.close()


def test_sharded_level_round_on_one_nccl_rank():
    import torch.distributed as dist

    from paper_1606_07413_gb300 import build, shard

    build.build()
    dev = torch.device("cuda:0")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=dev)
    try:
        with make(WALKS) as prob:
            eng = shard.DeviceEngine(prob, dev, 1 << 16, 1)
            lvl = shard.ShardedLevel(eng, WALKS)
            lvl.begin(K, VERSION, DPB)
            total = 0
            for _ in range(3):
                r = lvl.round(STEPS)
                total += r["received"]
            assert lvl.lost == 0 and total == r["dps"] and r["steps"] == 3 * WALKS * STEPS
    finally:
        dist.destroy_process_group()
