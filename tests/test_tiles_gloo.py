"""Host side of the column-tile exchange (paper Sec. 2 "Delivery of spiking
messages": counts, then payload, every step), without a GPU.

- The columns each column's synapses reach are taken from the projection;
  they are checked against every synapse the oracle generates on small tori
  (including sides 2 and 3, where ring members coincide).
- Packing sends a spike to exactly the tiles its synapses reach.
- Two gloo ranks exchange counts then payloads with torch.distributed
  all-to-all calls and receive exactly the spikes addressed to them; the
  in-process exchange gives the same lists.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads
from paper_1310_8478_gb300 import tiles


@pytest.mark.parametrize("gx,gy,mix", [(4, 2, (40, 30, 20, 10)), (3, 3, (40, 30, 20, 10)), (5, 4, (76, 12, 8, 4)),
                                       (2, 2, (40, 30, 20, 10)), (6, 1, (50, 50, 0, 0))])
def test_reached_columns_cover_every_generated_synapse(orc, gx, gy, mix):
    cfg = workloads.custom(grid_x=gx, grid_y=gy, fanout=60, pct_ring=mix, seed=31)
    npc = cfg["neurons_per_col"]
    for col in range(gx * gy):
        reach = tiles.reached_columns(cfg, col)
        got = set()
        for local in (0, 1, 999, 1000, 1249):          # excitatory and inhibitory sources
            tg, _ = orc.generate_row(cfg, col * npc + local)
            got |= set((tg // npc).tolist())
        assert got <= reach, (col, got - reach)
        # every reachable column is used by some excitatory source of the column
        exc = set()
        for local in range(0, 1000, 37):
            tg, _ = orc.generate_row(cfg, col * npc + local)
            exc |= set((tg // npc).tolist())
        assert exc == reach, (col, reach - exc)


def test_column_ranges_and_destinations():
    r = tiles.column_ranges(8, 3)
    assert r == [(0, 3), (3, 3), (6, 2)]
    assert list(tiles.tile_of_column(r)) == [0, 0, 0, 1, 1, 1, 2, 2]
    cfg = workloads.custom(grid_x=4, grid_y=2, fanout=60, pct_ring=(40, 30, 20, 10), seed=1)
    dest = tiles.destinations(cfg, tiles.column_ranges(8, 2))
    # on a 4x2 torus split into the rows y = 0 and y = 1, every column
    # reaches the other row (ring 1 at (0, +-1))
    assert all(d == [1] for d in dest[:4]) and all(d == [0] for d in dest[4:])
    cfg1 = workloads.custom(grid_x=8, grid_y=1, fanout=60, pct_ring=(100, 0, 0, 0), seed=1)
    assert all(d == [] for d in tiles.destinations(cfg1, tiles.column_ranges(8, 2)))


def _expected(gids_by_rank, npc, dest, me):
    return sorted(g for src, gids in enumerate(gids_by_rank) if src != me
                  for g in gids if me in dest[g // npc])


def _spikes(rank, ranges, npc, seed):
    rng = np.random.default_rng(seed + rank)
    first, count = ranges[rank]
    return np.sort(rng.choice(np.arange(first * npc, (first + count) * npc), size=300, replace=False)).astype(np.int32)


def test_pack_counts_match_payload():
    cfg = workloads.custom(grid_x=5, grid_y=3, fanout=60, pct_ring=(40, 30, 20, 10), seed=1)
    ranges = tiles.column_ranges(15, 3)
    dest = tiles.destinations(cfg, ranges)
    g = _spikes(1, ranges, 1250, 9)
    counts, payload = tiles.pack(g, 1250, dest, 3)
    assert counts[1] == 0 and counts.sum() == len(payload)
    off = np.concatenate([[0], np.cumsum(counts)])
    for k in range(3):
        part = payload[off[k]:off[k + 1]]
        assert sorted(part.tolist()) == sorted(x for x in g.tolist() if k in dest[x // 1250])


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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import workloads as wl
    from paper_1310_8478_gb300 import tiles as tl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = wl.custom(grid_x=4, grid_y=3, fanout=60, pct_ring=(40, 30, 20, 10), seed=1)
    ranges = tl.column_ranges(12, world)
    dest = tl.destinations(cfg, ranges)
    ex = tl.DistExchange(dist)
    got = []
    for step in range(3):                      # three steps of counts, then payload
        g = _spikes(rank, ranges, 1250, 100 * step)
        counts, payload = tl.pack(g, 1250, dest, world)
        got.append(sorted(ex.exchange_one(counts, payload).tolist()))
    out.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_counts_then_payload():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = workloads.custom(grid_x=4, grid_y=3, fanout=60, pct_ring=(40, 30, 20, 10), seed=1)
    ranges = tiles.column_ranges(12, world)
    dest = tiles.destinations(cfg, ranges)
    for step in range(3):
        gids = [_spikes(r, ranges, 1250, 100 * step) for r in range(world)]
        local = tiles.LocalExchange().exchange([tiles.pack(g, 1250, dest, world) for g in gids])
        for r in range(world):
            exp = _expected(gids, 1250, dest, r)
            assert res[r][step] == exp
            assert sorted(local[r].tolist()) == exp
