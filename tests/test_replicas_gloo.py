"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) combine
into the whole-job figures -- the slowest rank's time and the sum of events."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    assert bench.dist_env() == (rank, rank, world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, ev = bench.combine_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, "cpu")
    out.put((rank, ms, ev))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_rank_passes_through():
    import bench
    assert bench.combine_ranks(7.5, 42, None) == (7.5, 42)
