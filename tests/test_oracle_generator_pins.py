"""Pins of the oracle's draws against an independent restatement.

The network generator and the thalamic drive are readings (the paper gives
fractions and a "simple statistical model", not a generator): each draw is
Philox4x32-10 (Salmon et al., SC'11), keyed by the seed, at a counter that
names what is drawn.  Here Philox4x32-10 is written again in plain Python
from its published definition -- checked on the same known-answer vectors
as the oracle's -- and the readings are restated draw by draw, so that a
wrong word, counter, ring order, range map or self-exclusion in the oracle
fails these tests.

Readings restated (Sec. 2 "Projection of synapses with individual delay" and
"Bidimensional arrays of neural columns"; Sec. 3 per-neighbour percentages):
  synapse j of source p: words r = Philox((p, j, 0, 0), seed); range map
  floor(r * n / 2^32);
  inhibitory source: target = an excitatory neuron of its own column,
  floor(r0 * ne / 2^32); delay 1;
  excitatory source: delay 1 + floor(r1 * D / 2^32); ring = first k with
  j < floor(M * (p0 + .. + pk) / 100); inside ring k >= 1, member
  (j - start_k) mod 4 of the offsets
      ring 1: (+1, 0) (-1, 0) (0, +1) (0, -1)
      ring 2: (+1, +1) (-1, +1) (+1, -1) (-1, -1)
      ring 3: (+2, 0) (-2, 0) (0, +2) (0, -2)
  on the torus; in the own column any neuron but the source
  (floor(r0 * (npc - 1) / 2^32), shifted past the source), elsewhere
  floor(r0 * npc / 2^32);
  thalamic event k of column c at step t: neuron floor(r0 * npc / 2^32) of
  the column, r = Philox((t, c, 1, k), seed).
"""
import os

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32-10 from its definition: 10 rounds of two 32x32->64-bit
    multiplications with the published multipliers, the key bumped by the
    published Weyl constants between rounds."""
    m0, m1 = 0xD2511F53, 0xCD9E8D57
    w0, w1 = 0x9E3779B9, 0xBB67AE85
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for rnd in range(10):
        p0, p1 = m0 * c0, m1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0, k1 = (k0 + w0) & MASK, (k1 + w1) & MASK
    return [c0, c1, c2, c3]


def test_python_philox_reproduces_the_known_answer_vectors():
    n = 0
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                assert philox4x32_10(w[0:4], w[4:6]) == w[6:10]
                n += 1
    assert n >= 3


RINGS = {1: [(1, 0), (-1, 0), (0, 1), (0, -1)],
         2: [(1, 1), (-1, 1), (1, -1), (-1, -1)],
         3: [(2, 0), (-2, 0), (0, 2), (0, -2)]}


def scale(r, n):
    return (r * n) >> 32


def restated_synapse(cfg, p, j):
    npc, ne, m, d_max = cfg["neurons_per_col"], cfg["exc_per_col"], cfg["fanout"], cfg["max_delay_ms"]
    key = (cfg["seed"] & MASK, cfg["seed"] >> 32)
    r = philox4x32_10((p, j, 0, 0), key)
    col, local = divmod(p, npc)
    if local >= ne:
        return col * npc + scale(r[0], ne), 1
    delay = 1 + scale(r[1], d_max)
    acc, ring, start, prev_end = 0, 3, 0, 0
    for k in range(4):
        acc += cfg["pct_ring"][k]
        end = (m * acc) // 100
        if j < end:
            ring, start = k, prev_end
            break
        prev_end = end
    gx, gy = cfg["grid_x"], cfg["grid_y"]
    cx, cy = col % gx, col // gx
    tx, ty = cx, cy
    if ring > 0:
        dx, dy = RINGS[ring][(j - start) % 4]
        tx, ty = (cx + dx) % gx, (cy + dy) % gy
    tcol = ty * gx + tx
    if tcol == col:
        tl = scale(r[0], npc - 1)
        if tl >= local:
            tl += 1
    else:
        tl = scale(r[0], npc)
    return tcol * npc + tl, delay


@pytest.mark.parametrize("cfg", [
    workloads.custom(grid_x=5, grid_y=4, neurons_per_col=40, exc_per_col=32, fanout=101,
                     pct_ring=(40, 30, 20, 10), seed=0x123456789),
    workloads.custom(grid_x=7, grid_y=3, neurons_per_col=25, exc_per_col=20, fanout=77,
                     pct_ring=(76, 12, 8, 4), seed=7, max_delay_ms=13),
])
def test_generated_rows_equal_the_restated_reading(orc, cfg):
    n = workloads.n_neurons(cfg)
    rng = np.random.default_rng(11)
    sources = sorted(set(int(x) for x in rng.integers(0, n, 40)) | {0, n - 1, cfg["exc_per_col"] - 1,
                                                                        cfg["exc_per_col"]})
    for p in sources:
        tg, dl = orc.generate_row(cfg, p)
        for j in range(cfg["fanout"]):
            assert (int(tg[j]), int(dl[j])) == restated_synapse(cfg, p, j), (p, j)


def test_thalamic_targets_equal_the_restated_reading(orc):
    cfg = workloads.custom(grid_x=6, grid_y=5, neurons_per_col=123, exc_per_col=98, seed=0xDEADBEEF12)
    key = (cfg["seed"] & MASK, cfg["seed"] >> 32)
    for t in (0, 1, 17, 999, 123456):
        for col in (0, 7, 29):
            for k in (0, 1, 3):
                r = philox4x32_10((t, col, 1, k), key)
                assert orc.thalamic_target(cfg, t, col, k) == col * 123 + scale(r[0], 123), (t, col, k)
