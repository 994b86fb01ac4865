"""Host logic of the N-GPU bench path on CPU ranks (gloo, world size 2):
scans are sharded with no overlap and the timing is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, batch, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first = bench.shard_first_scan(rank, batch)
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    q.put((rank, list(range(first, first + batch)), slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_scans_and_take_the_slowest_time():
    world, batch = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, batch, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scans = sorted(s for _, shard, _ in out for s in shard)
    assert scans == list(range(world * batch))           # disjoint, complete
    assert all(slowest == 11.0 for _, _, slowest in out)


def test_single_process_timing_is_unchanged():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
