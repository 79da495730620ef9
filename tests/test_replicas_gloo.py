"""Multi-GPU host logic on CPU: two gloo ranks aggregate replica timings.

The method shards by frame (independent pairs), so N GPUs run N replicas with
no data-path collective; the cross-rank step is the timing reduction that
bench.py performs (sum of frames, max of times). Each rank also reports the
frames the split gives it, and the test checks that every frame is covered
exactly once.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2212_00488_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = list(replicas.frames_for_rank(5, rank, world))
        # rank r pretends to take (r + 1) seconds for its frames
        t = replicas.aggregate(float(len(frames)), float(rank + 1))
        q.put((rank, frames, t.world, t.units_total, t.seconds_max, t.throughput))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_is_sum_over_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    frames = sorted(f for o in out for f in o[1])
    assert frames == [0, 1, 2, 3, 4]                     # every frame exactly once
    for _, _, world, units, secs, thr in out:
        assert world == 2 and units == 5.0 and secs == 2.0 and thr == pytest.approx(2.5)


def test_single_replica_without_process_group():
    from paper_2212_00488_gb300 import replicas
    t = replicas.aggregate(10.0, 4.0)
    assert (t.world, t.throughput) == (1, 2.5)
    with pytest.raises(ValueError):
        replicas.frames_for_rank(3, 2, 2)
