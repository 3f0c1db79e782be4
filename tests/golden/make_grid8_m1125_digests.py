"""Write grid8_m1125_digests.json: checkpoints of the 8x8 torus workload
(80 000 neurons, M = 1125, 40/30/20/10 projection mix, seed 2) simulated by
the CPU oracle across its first long-term plasticity update.

The run covers steps 0 .. 1009, so it crosses the update that closes step 999
(the paper's "long term synaptic plasticity" block of Table 2, one period of
1000 ms) on a torus whose ring members are all distinct columns, at the
fan-out of the benchmark.  At every checkpoint t (the net has simulated steps
0 .. t-1) the file records
  - the event counters (spikes, synaptic events, excitatory events,
    potentiation visits) since step 0;
  - the sha256 of the raster of steps [previous checkpoint, t) as little-endian
    int32 (t, gid) pairs sorted by (t, gid);
  - at the weight checkpoints, the sha256 of w and of sd, little-endian int32
    in canonical (source, ordinal) order.

Only the oracle is called.  The run takes several hours of one CPU core (the
net fires at several hundred Hz for most of the first second); the file is
rewritten after every checkpoint, with "complete": false until the last one.
Run:  python tests/golden/make_grid8_m1125_digests.py
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

WORKLOAD = "grid8_m1125"
RASTER_POINTS = [10, 20, 30, 50, 100, 200, 300, 400, 500, 600, 700, 800, 900, 999, 1000, 1010]
WEIGHT_POINTS = [30, 100, 500, 999, 1000, 1010]
OUT = os.path.join(HERE, "grid8_m1125_digests.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a.astype("<i4")).tobytes()).hexdigest()


def raster_digest(t: np.ndarray, g: np.ndarray, t0: int, t1: int) -> tuple[str, int]:
    sel = (t >= t0) & (t < t1)
    pairs = np.stack([t[sel], g[sel]], axis=1)
    return sha(pairs), int(sel.sum())


def main():
    cfg = workloads.workload(WORKLOAD)
    sim = oracle.Oracle(cfg)
    doc = {"workload": WORKLOAD, "seed": cfg["seed"], "grid": [cfg["grid_x"], cfg["grid_y"]],
           "fanout": cfg["fanout"], "written_by": "tests/golden/make_grid8_m1125_digests.py (oracle only)",
           "complete": False, "checkpoints": []}
    prev = 0
    t_start = time.time()
    for point in RASTER_POINTS:
        sim.run(point - sim.t)
        t, g = sim.raster()
        rd, n = raster_digest(t, g, prev, point)
        entry = {"t": point, "counters": sim.counters(), "raster_from": prev, "raster_sha256": rd,
                 "raster_spikes": n}
        if point in WEIGHT_POINTS:
            syn = sim.synapses()
            entry["w_sha256"] = sha(syn["w"])
            entry["sd_sha256"] = sha(syn["sd"])
            entry["sd_nonzero"] = int(np.count_nonzero(syn["sd"]))
        doc["checkpoints"].append(entry)
        prev = point
        doc["complete"] = point == RASTER_POINTS[-1]
        doc["oracle_cpu_s"] = round(time.time() - t_start, 1)
        with open(OUT + ".tmp", "w") as f:
            json.dump(doc, f, indent=1)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)
        print("t=%d %.0f s %s" % (point, time.time() - t_start, entry["counters"]), flush=True)


if __name__ == "__main__":
    main()
