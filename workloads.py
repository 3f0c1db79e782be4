"""Named workloads of the DPSNN-STDP step: plain parameter dictionaries.

This module holds only sizes, seeds and model constants; it contains none of
the method's arithmetic.  Both the CUDA path's binding and the CPU oracle take
these dictionaries, so it is the one module the two sides share.

Model constants follow the paper (Sec. 2 "Spiking neuron model": 80 % RS / 20 %
FS Izhikevich neurons; "Projection of synapses with individual delay": delays
1..20 ms, inhibitory synapses at the minimum delay and local to excitatory
targets; "Synaptic update": the STDP pair rule), with the column size, fan-out,
projection mix, initial/maximum weights, STDP amplitudes, long-term plasticity
constants and thalamic drive of the benchmark workloads below.  Q16 means
value * 65536 (1 mV = 65536).
"""
from __future__ import annotations

import copy

Q16 = 65536

# Parameters shared by every workload (per-column model).
BASE = dict(
    neurons_per_col=1250,        # 1000 RS excitatory + 250 FS inhibitory
    exc_per_col=1000,
    max_delay_ms=20,
    w_exc0_q16=6 * Q16,          # +6 mV
    w_inh0_q16=-5 * Q16,         # -5 mV
    wmax_q16=10 * Q16,           # 10 mV
    a_plus_mv=0.1,
    a_minus_mv=0.12,
    tau_plus_ms=20.0,
    tau_minus_ms=20.0,
    deriv_period_ms=1000,
    deriv_bias_q16=655,          # 0.01 mV
    deriv_decay_q16=58982,       # 0.9
    thal_per_col_per_ms=1,
    thal_amp_q16=20 * Q16,       # 20 mV
    flags=0,
)

WORKLOADS = {
    # one column, 100 synapses per neuron to random targets of the column
    "col1_m100": dict(grid_x=1, grid_y=1, fanout=100, pct_ring=(100, 0, 0, 0),
                      seed=1, sim_ms=1000),
    # 8x8 torus, 1125 synapses per neuron, 40/30/20/10 projection mix
    "grid8_m1125": dict(grid_x=8, grid_y=8, fanout=1125, pct_ring=(40, 30, 20, 10),
                        seed=2, sim_ms=5000),
    # 16x16 torus (320 k neurons, 360 M synapses), same mix: a smaller case of
    # the same kernels for profiling (a few GB on the device)
    "grid16_m1125": dict(grid_x=16, grid_y=16, fanout=1125, pct_ring=(40, 30, 20, 10),
                         seed=4, sim_ms=1000),
    # 64x64 torus (5.12 M neurons, 5.76 G synapses), same mix
    "grid64_m1125": dict(grid_x=64, grid_y=64, fanout=1125, pct_ring=(40, 30, 20, 10),
                         seed=3, sim_ms=2000),
    # the same 5.12 M neurons with 16 synapses each (82 M synapses, ~1.5 GB
    # on the device): the neuron update at full width, for profiling
    "grid64_m16": dict(grid_x=64, grid_y=64, fanout=16, pct_ring=(40, 30, 20, 10),
                       seed=3, sim_ms=100),
}

# The paper's own geometry (Sec. 2 and Table 1): columns of 1000 neurons (800
# RS, 200 FS), M = 200 synapses per neuron, 76/12/8/4 projection mix; grid
# sizes of Table 1 (200 K ... 6.6 G synapses).  Neuron, STDP and plasticity
# constants as above (the paper does not print its weights).
PAPER_GRIDS = {"1x1": (1, 1), "2x2": (2, 2), "4x4": (4, 4), "8x8": (8, 8), "16x16": (16, 16),
               "32x32": (32, 32), "64x64": (64, 64), "128x128": (128, 128), "256x128": (256, 128)}
for _name, (_gx, _gy) in PAPER_GRIDS.items():
    WORKLOADS["paper_" + _name] = dict(grid_x=_gx, grid_y=_gy, neurons_per_col=1000, exc_per_col=800,
                                       fanout=200, pct_ring=(76, 12, 8, 4), seed=7, sim_ms=2000)


def workload(name: str, **overrides) -> dict:
    """Full parameter dictionary of a named workload (a fresh copy)."""
    cfg = copy.deepcopy(BASE)
    cfg.update(copy.deepcopy(WORKLOADS[name]))
    cfg.update(overrides)
    cfg["name"] = name
    return cfg


def custom(**fields) -> dict:
    """A parameter dictionary from BASE plus explicit fields (tests, sweeps)."""
    cfg = copy.deepcopy(BASE)
    cfg.update(dict(grid_x=1, grid_y=1, fanout=100, pct_ring=(100, 0, 0, 0), seed=1, sim_ms=100))
    cfg.update(fields)
    cfg.setdefault("name", "custom")
    return cfg


def n_neurons(cfg: dict) -> int:
    return cfg["grid_x"] * cfg["grid_y"] * cfg["neurons_per_col"]


def n_synapses(cfg: dict) -> int:
    return n_neurons(cfg) * cfg["fanout"]


def batch_workloads(n: int = 256, first_seed: int = 1000, side=(1, 16), fanouts=(100, 400, 1125),
                    draw_seed: int = 2024, sim_ms: int = 1000) -> list:
    """Independent uneven networks: grid side uniform in [side], fan-out uniform
    over `fanouts`, network seeds first_seed, first_seed + 1, ...; the sizes
    are drawn from a fixed numpy generator (draw_seed) so the list is the same
    every time."""
    import numpy as np
    rng = np.random.default_rng(draw_seed)
    out = []
    for i in range(n):
        sd = int(rng.integers(side[0], side[1] + 1))
        m = int(fanouts[int(rng.integers(0, len(fanouts)))])
        mix = (40, 30, 20, 10) if sd > 1 else (100, 0, 0, 0)
        out.append(custom(grid_x=sd, grid_y=sd, fanout=m, pct_ring=mix, seed=first_seed + i, sim_ms=sim_ms,
                          name="batch%03d_%dx%d_m%d" % (i, sd, sd, m)))
    return out


def serve_request_params(i: int, rng, side=(1, 32), fanouts=(100, 400, 1125), duration=(100, 5000),
                         first_seed: int = 5000):
    """One simulation request of the serving workload: grid side log-uniform
    in [side], fan-out uniform over `fanouts`, duration uniform in [duration]
    ms; `rng` is a numpy Generator owned by the caller."""
    import math
    sd = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1])))))
    sd = max(side[0], min(side[1], sd))
    m = int(fanouts[int(rng.integers(0, len(fanouts)))])
    mix = (40, 30, 20, 10) if sd > 1 else (100, 0, 0, 0)
    cfg = custom(grid_x=sd, grid_y=sd, fanout=m, pct_ring=mix, seed=first_seed + i,
                 name="req%04d_%dx%d_m%d" % (i, sd, sd, m))
    dur = int(rng.integers(duration[0], duration[1] + 1))
    return cfg, dur
