"""One level of the collision search sharded across ranks by distinguished-
point owner (Sec. 4.2, Fig. 4: workers send every distinguished point to the
collector that owns it; the collector stores it and hands merged trails to a
verifier).

Every rank is worker, collector and verifier at once.  Rank r walks the
global walks r W .. (r + 1) W - 1 (the same walk seed on every rank, so trail
references name walks by their global index and any rank can recompute a
trail's start), and owns the distinguished points whose owner hash is r.  A
round is:

1. walk: every walk advances; the distinguished points it reaches go to an
   outbox on the device (qcs_level_walk_out);
2. bin: the outbox is grouped by owner rank on the device (qcs_shard_bin);
3. exchange: the group sizes, then the groups, in one all-to-all each
   (torch.distributed: NCCL between GPUs, gloo in the CPU tests);
4. insert: each rank stores the points it received in its own table, which
   queues merges exactly as a single table would (qcs_level_insert);
5. re-walk and collect: each rank re-walks its merges and checks claw
   candidates exactly (qcs_level_rewalk, qcs_level_collect); a claw found
   anywhere ends the level on every rank (one all-reduce of a flag).

The device work of steps 1, 2, 4 and 5 is behind an engine object so that the
host logic -- the exchange and the stop rule -- runs unchanged against a CPU
stand-in in the tests.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class DeviceEngine:
    """The device steps of one rank on a GPU, through libqcs."""

    def __init__(self, prob, device, outbox_cap: int, n_owners: int, stream=None):
        import paper_1606_07413_gb300 as Q

        self.Q, self.prob, self.device, self.stream = Q, prob, device, stream
        self.outbox = torch.zeros(2 * outbox_cap, dtype=torch.int64, device=device)
        self.binned = torch.zeros_like(self.outbox)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.owner_counts = torch.zeros(2 * n_owners, dtype=torch.int32, device=device)
        self.n_owners = n_owners

    def begin(self, k, version, dp_bits, walk_base, total_walks):
        self.prob.level_begin_shard(k, version, dp_bits, walk_base, total_walks, self.stream)

    def walk_and_bin(self, steps):
        """Walk, then group the outbox by owner: (binned points as an (m, 2)
        int64 tensor on the device, group sizes as a list, points lost to a
        full outbox)."""
        self.prob.level_walk_out(steps, self.outbox, self.count, self.stream)
        n_total = int(self.count.item())  # synchronizes the walk
        n = min(n_total, self.outbox.numel() // 2)
        self.Q.shard_bin(self.outbox, n, self.n_owners, self.binned, self.owner_counts, self.stream)
        counts = self.owner_counts[: self.n_owners].tolist()
        return self.binned[: 2 * n].view(-1, 2), counts, n_total - n

    def insert(self, points):
        self.prob.level_insert(points.reshape(-1), points.shape[0], self.stream)

    def rewalk_collect(self) -> dict:
        self.prob.level_rewalk(self.stream)
        return self.prob.level_collect(self.stream)


def exchange(points, counts, group=None):
    """All-to-all of distinguished points grouped by owner: points is an
    (m, 2) int64 tensor whose first counts[0] rows go to rank 0, the next
    counts[1] to rank 1, and so on; returns the (m', 2) rows every rank sent
    to this one, in rank order."""
    world = dist.get_world_size(group)
    dev = points.device
    send_counts = torch.tensor(counts, dtype=torch.int64, device=dev)
    assert send_counts.numel() == world and int(send_counts.sum()) == points.shape[0]
    recv_counts = torch.empty_like(send_counts)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    rc = recv_counts.tolist()
    recv = torch.empty((sum(rc), 2), dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv, points.contiguous(), output_split_sizes=rc, input_split_sizes=list(counts),
                           group=group)
    return recv


class ShardedLevel:
    """Level k of one target walked by every rank of `group`, each rank with
    the same number of walks (engine.begin gets this rank's global walk
    range)."""

    def __init__(self, engine, walks_per_rank: int, group=None):
        self.engine, self.group = engine, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.walks = walks_per_rank
        self.lost = 0

    def begin(self, k, version=0, dp_bits=0):
        self.engine.begin(k, version, dp_bits, self.rank * self.walks, self.world * self.walks)

    def round(self, steps) -> dict:
        """One round; returns this rank's collect result plus "found_any": a
        verified claw on any rank."""
        points, counts, lost = self.engine.walk_and_bin(steps)
        self.lost += lost
        recv = exchange(points, counts, self.group)
        self.engine.insert(recv)
        res = self.engine.rewalk_collect()
        flag = torch.tensor([1 if res.get("status_name") == "found" else 0], dtype=torch.int64,
                            device=points.device)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=self.group)
        res["found_any"] = bool(flag.item())
        res["received"] = int(recv.shape[0])
        return res
