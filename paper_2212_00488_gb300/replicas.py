"""Replica bookkeeping for runs on several GPUs of one node.

Frames are independent, so N GPUs run N replicas, each on its own frames; no
data crosses between them. The only cross-rank steps are timing plumbing: a
barrier before and after the timed region and the maximum of the per-rank
elapsed times, from which the whole-job throughput is computed.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class ReplicaTiming:
    world: int
    units_total: float      # units (frames) processed by all ranks
    seconds_max: float      # slowest rank's elapsed time
    throughput: float       # units_total / seconds_max


def frames_for_rank(n_frames: int, rank: int, world: int) -> range:
    """Frames [0, n_frames) dealt round-robin: rank r takes r, r + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank or world size")
    return range(rank, n_frames, world)


def aggregate(units_local: float, seconds_local: float, group=None) -> ReplicaTiming:
    """Whole-job throughput from per-rank counts and times.

    With torch.distributed initialised, sums the units and takes the maximum
    time over the ranks of `group` (any backend: nccl on GPUs, gloo on CPUs);
    without it, a single replica.
    """
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return ReplicaTiming(1, units_local, seconds_local, units_local / seconds_local)
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([seconds_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    world = dist.get_world_size(group)
    return ReplicaTiming(world, float(u.item()), float(t.item()), float(u.item()) / float(t.item()))
