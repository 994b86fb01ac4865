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


def test_gpus_flag_launches_one_rank_per_gpu_and_rank_zero_prints():
    """`bench.py --gpus 2` without a launcher relaunches itself as two ranks of
    torch.distributed.run; the reference arm runs on rank 0 only, which prints
    the one JSON line with the world size as n_gpus."""
    import json
    import subprocess
    import sys

    from conftest import ROOT
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--config", "das2d_64", "--steps", "1", "--warmup", "3",
                        "--cpu-pool", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT, env={k: v for k, v in os.environ.items()
                                      if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["cores"] >= 1
