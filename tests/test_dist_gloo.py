"""Multi-process host logic of the replica path (bench.py --gpus N under torchrun: one
independent replica per GPU, no data-path collective): max-over-ranks timing, the
whole-job rate and the partition of serving requests, with world_size 2 on the gloo
backend (CPU)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_2404_02521_gb300 import serving
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_rank = 100.0 + 50.0 * rank            # this rank's timed region, ms
    t_max = bench.barrier_max(t_rank, world)
    bench.barrier(world)
    mine = serving.shard(10, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out[rank] = (t_max, bench.whole_job_rate(1000.0, 3, world, t_max), gathered)
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t_max, rate, gathered = res[rank]
        assert t_max == 150.0                              # the slowest rank's time
        assert rate == pytest.approx(2 * 3 * 1000.0 / 0.150)
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(10))                     # every request exactly once
        assert not set(gathered[0]) & set(gathered[1])
