"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0909_0001_gb300 import multirank


def test_shard_channels_covers_all_once():
    for total in (1, 7, 64, 100):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s, c = multirank.shard_channels(total, world, r)
                seen += list(range(s, s + c))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        multirank.shard_channels(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, count = multirank.shard_channels(64, world, rank)
    seconds = 0.5 + rank          # rank 1 is the slow one
    rate, slowest = multirank.job_rate(count * 1000.0, seconds)
    dist.barrier()
    out[rank] = (start, count, rate, slowest)
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert out[0][:2] == (0, 32) and out[1][:2] == (32, 32)
    for r in range(world):
        assert out[r][3] == pytest.approx(1.5)              # the slowest rank's time
        assert out[r][2] == pytest.approx(64000.0 / 1.5)     # all units over that time
