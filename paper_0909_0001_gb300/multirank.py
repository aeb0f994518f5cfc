"""Host logic for running the correlator on several GPUs of one node.

Frequency channels are independent problems (Appendix A repeats the per-sample
work for every frequency bin), so ranks split the channels and never exchange
data on the correlation path.  The only collectives are for timing: a barrier
around the timed region and the maximum of the per-rank times.
"""
from __future__ import annotations

import os
from typing import Tuple

import torch
import torch.distributed as dist


def rank_env() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def shard_channels(total: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous channel range [start, start + count) of a rank; sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def _reduce(value: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    return _reduce(value, dist.ReduceOp.SUM, device)


def job_rate(units_local: float, seconds_local: float, device="cpu") -> Tuple[float, float]:
    """Whole-job throughput: all ranks' units over the slowest rank's time.

    Returns (units per second, slowest time in seconds)."""
    slowest = max_over_ranks(seconds_local, device)
    total = sum_over_ranks(units_local, device)
    return total / slowest, slowest
