"""The 8x8 torus workload (80 000 neurons, M = 1125, 40/30/20/10, seed 2)
against the oracle across its first long-term plasticity update.

The oracle run takes hours of one CPU core, so its checkpoints were written
once by tests/golden/make_grid8_m1125_digests.py (oracle only) into
grid8_m1125_digests.json: at every checkpoint the event counters, the sha256
of the raster since the previous checkpoint and, at some, the sha256 of w
and sd in canonical order.  The CUDA path must reproduce every one of them,
bit for bit, in each way of taking the steps: the device's own choice, the
event-driven deliveries only, the column walk only, the ring-list delivery
only, the 13-column staged delivery, and the dense pass whenever anything
fired.  The run crosses the update that closes step
999 (paper Table 2, "long term synaptic plasticity") while nearly every
neuron fires every step, so the dense pass's long-term-update branch and the
fold of the event-driven potentiation run on full 1128-slot rows of a torus
whose ring members are all distinct columns.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads
from conftest import golden_path

pytestmark = pytest.mark.gpu

MODES = {"auto": None,
         "sparse": dict(dense_permille=1001, staged_permille=0xffffffff),
         "staged": dict(dense_permille=1001, staged_permille=1),
         "dense": dict(dense_permille=1),
         "ordered": dict(dense_permille=1001, staged_permille=0xffffffff, ring_permille=1),
         "ring": dict(dense_permille=1001, staged_permille=0xffffffff, ring_permille=0xffffffff)}


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(np.asarray(a).astype("<i4")).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def golden():
    p = golden_path("grid8_m1125_digests.json")
    if not os.path.exists(p):
        pytest.skip("no oracle checkpoints recorded")
    doc = json.load(open(p))
    if not doc["checkpoints"]:
        pytest.skip("no oracle checkpoints recorded")
    return doc


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


@pytest.mark.parametrize("mode", sorted(MODES))
def test_grid8_m1125_matches_oracle_checkpoints(eng, golden, mode):
    cfg = workloads.workload("grid8_m1125")
    assert golden["seed"] == cfg["seed"] and golden["fanout"] == cfg["fanout"]
    last = golden["checkpoints"][-1]["t"]
    cap = 80_000 * (last + 2)
    with eng.Network(cfg, raster_capacity=cap) as n:
        if MODES[mode] is not None:
            n.set_launch(**MODES[mode])
        for cp in golden["checkpoints"]:
            n.run(cp["t"] - n.t)
            c = n.counters()
            assert c["error"] == 0 and c["raster_dropped"] == 0
            for k in ("spikes", "e_all", "e_exc", "l_exc"):
                assert c[k] == cp["counters"][k], (mode, cp["t"], k, c[k], cp["counters"][k])
            t, g = n.raster(cp["raster_from"], cp["t"])
            assert len(t) == cp["raster_spikes"], (mode, cp["t"])
            assert _sha(np.stack([t, g], axis=1)) == cp["raster_sha256"], (mode, cp["t"])
            if "w_sha256" in cp:
                w, sd = n.weights()
                assert _sha(w) == cp["w_sha256"], (mode, cp["t"], "w")
                assert _sha(sd) == cp["sd_sha256"], (mode, cp["t"], "sd")
                assert int(np.count_nonzero(sd)) == cp["sd_nonzero"]
