"""Column tiles of a torus and the per-step exchange of spike lists between
them (the paper's Sec. 2 "Delivery of spiking messages": every process owns
a set of columns; after each step it sends, to every process that hosts
synapses of its neurons, first how many spikes it has for it, then the spike
ids themselves -- two all-to-all messages per step).

A tile is a net (snn_set_tile) that owns a contiguous range of columns: it
integrates their neurons and delivers to them.  After every step each tile
reads its own spikes of that step, sends to every other tile the spikes of
its neurons whose synapses reach that tile's columns, and injects what it
receives (snn_inject_spikes) before the next step.  Which source columns
reach which columns follows from the projection: an inhibitory neuron reaches
its own column, an excitatory one its own column and the four member columns
of every ring with a non-zero share (ring 1 at (+-1, 0), (0, +-1); ring 2 at
(+-1, +-1); ring 3 at (+-2, 0), (0, +-2); on the torus).  Sending a spike to a
tile it does not reach would be harmless (that tile delivers only to its own
columns); not sending one it does reach would change the results.

Everything on the device is the engine's (include/snn.h); this module packs,
exchanges and unpacks host arrays.  The exchange is an object with one
method, all_to_all(counts, payload): LocalExchange moves lists between tiles
living in one process; DistExchange does the two all-to-all calls over
torch.distributed (one tile per rank).
"""
from __future__ import annotations

import numpy as np

RING_OFFSETS = {
    1: [(1, 0), (-1, 0), (0, 1), (0, -1)],
    2: [(1, 1), (-1, 1), (1, -1), (-1, -1)],
    3: [(2, 0), (-2, 0), (0, 2), (0, -2)],
}


def column_ranges(n_columns: int, n_tiles: int) -> list[tuple[int, int]]:
    """Contiguous (first column, count) of every tile, sizes differing by one at most."""
    if not 1 <= n_tiles <= n_columns:
        raise ValueError("need 1 <= tiles <= columns")
    base, extra = divmod(n_columns, n_tiles)
    out, c = [], 0
    for k in range(n_tiles):
        n = base + (1 if k < extra else 0)
        out.append((c, n))
        c += n
    return out


def tile_of_column(ranges) -> np.ndarray:
    n = sum(c for _, c in ranges)
    owner = np.empty(n, np.int32)
    for k, (first, count) in enumerate(ranges):
        owner[first:first + count] = k
    return owner


def reached_columns(cfg: dict, col: int) -> set[int]:
    """Columns that the synapses of column `col`'s neurons can reach."""
    gx, gy = cfg["grid_x"], cfg["grid_y"]
    x, y = col % gx, col // gx
    out = {col}
    for ring in (1, 2, 3):
        if cfg["pct_ring"][ring] > 0:
            for dx, dy in RING_OFFSETS[ring]:
                out.add(((y + dy) % gy) * gx + (x + dx) % gx)
    return out


def destinations(cfg: dict, ranges) -> list[list[int]]:
    """For every column, the tiles other than its owner that its spikes must reach."""
    owner = tile_of_column(ranges)
    out = []
    for col in range(len(owner)):
        tiles = sorted({int(owner[c]) for c in reached_columns(cfg, col)} - {int(owner[col])})
        out.append(tiles)
    return out


def pack(gids: np.ndarray, npc: int, dest, n_tiles: int):
    """Counts (one per destination tile) and the payload ordered by destination."""
    gids = np.asarray(gids, np.int32)
    per = [[] for _ in range(n_tiles)]
    cols = gids // npc
    for g, c in zip(gids.tolist(), cols.tolist()):
        for k in dest[c]:
            per[k].append(g)
    counts = np.array([len(p) for p in per], np.int64)
    payload = np.array([g for p in per for g in p], np.int32)
    return counts, payload


class LocalExchange:
    """All-to-all among tiles held by one process: exchange(sends) takes, per
    tile, its (counts, payload) and returns, per tile, the ids it receives."""

    def exchange(self, sends):
        n = len(sends)
        received = [[] for _ in range(n)]
        for src, (counts, payload) in enumerate(sends):
            off = np.concatenate([[0], np.cumsum(counts)])
            for dst in range(n):
                if dst != src and counts[dst]:
                    received[dst].append(payload[off[dst]:off[dst + 1]])
        return [np.concatenate(r) if r else np.zeros(0, np.int32) for r in received]


class DistExchange:
    """One tile per rank over torch.distributed: the counts first (one
    integer per pair of ranks), then the payload split by those counts."""

    def __init__(self, dist, device="cpu"):
        self.dist = dist
        self.device = device

    def exchange_one(self, counts, payload):
        import torch
        c = torch.as_tensor(np.asarray(counts, np.int64), device=self.device)
        rc = torch.empty_like(c)
        self.dist.all_to_all_single(rc, c)
        send = torch.as_tensor(np.asarray(payload, np.int32), device=self.device)
        recv = torch.empty(int(rc.sum().item()), dtype=torch.int32, device=self.device)
        self.dist.all_to_all_single(recv, send, output_split_sizes=rc.tolist(), input_split_sizes=c.tolist())
        return recv.cpu().numpy()


def step_local(nets, cfg: dict, ranges, dest, exchange: LocalExchange | None = None, n_ms: int = 1):
    """Advance tiles held by one process n_ms steps, exchanging the spikes of
    every step before the next (nets[k] owns ranges[k])."""
    exchange = exchange or LocalExchange()
    npc = cfg["neurons_per_col"]
    for _ in range(n_ms):
        t = nets[0].t
        for n in nets:
            n.run(1)
        sends = []
        for n in nets:
            _, g = n.raster(t, t + 1)
            sends.append(pack(g, npc, dest, len(nets)))
        for n, got in zip(nets, exchange.exchange(sends)):
            n.inject_spikes(np.sort(got))
