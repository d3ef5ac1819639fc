"""The multi-GPU form of the bench on CPU: two gloo ranks combine their
timings (max time over ranks, sum of walk steps) and walk with distinct
seeds; no GPU is involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, u = bench.combine_ranks(1.5 + rank, 100.0 * (rank + 1), world, dist)
    mine = bench.rank_seed(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    dist.barrier()
    out.put((rank, t, u, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_timings():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, gathered in results:
        assert t == 2.5 and u == 300.0  # slowest rank, all ranks' units
        assert len(set(gathered)) == world  # each replica its own walk family


def test_single_rank_is_identity():
    import bench

    assert bench.combine_ranks(2.0, 7.0, 1) == (2.0, 7.0)
    assert bench.rank_seed(0) != bench.rank_seed(1)
