"""Full-size checks: the 64x64 benchmark torus (5.12 M neurons, 5.76 G
synapses) and the largest paper geometry (256x128, 6.6 G synapses), built in
the launch configuration bench.py times.

The oracle cannot simulate these sizes, so the checks are (a) outputs the
oracle computes one by one -- sampled rows of the generated network and
sampled thalamic draws -- and (b) properties that hold at any size: the same
run through the dense/automatic path and through each event-driven delivery
only (global reductions; column by column through shared memory) gives
bit-identical rasters, weights and counters,
the raster is sorted, unique and in range, and the counters agree with it.
"""
import hashlib

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

STEPS = 40      # spans the onset of the 64x64 run: event-driven steps, then dense ones


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


def _sample_sources(cfg, k, seed):
    rng = np.random.default_rng(seed)
    n = workloads.n_neurons(cfg)
    npc, ne = cfg["neurons_per_col"], cfg["exc_per_col"]
    picks = set(int(x) for x in rng.integers(0, n, k))
    picks |= {0, n - 1, ne - 1, ne, npc - 1, npc}          # column and kind boundaries
    return sorted(picks)


def _run(eng, cfg, shape, sources):
    n_neurons = workloads.n_neurons(cfg)
    with eng.Network(cfg, raster_capacity=n_neurons * (STEPS + 1)) as n:
        if shape:
            n.set_launch(**shape)
        rows = {p: n.synapses(p, 1) for p in sources}       # structure at t = 0
        n.run(STEPS)
        t, g = n.raster()
        after = {p: n.synapses(p, 1, fields=("w", "sd")) for p in sources}
        c = n.counters()
        h = hashlib.sha256()
        h.update(t.tobytes())
        h.update(g.tobytes())
        for p in sources:
            h.update(after[p]["w"].tobytes())
            h.update(after[p]["sd"].tobytes())
        return rows, (t, g), h.hexdigest(), c


@pytest.mark.parametrize("name", ["grid64_m1125", "paper_256x128"])
def test_full_size_structure_paths_and_invariants(eng, orc, name):
    cfg = workloads.workload(name)
    sources = _sample_sources(cfg, 24, seed=len(name))
    rows, (t, g), digest_auto, c_auto = _run(eng, cfg, None, sources)

    # (a) sampled rows equal the oracle's generator, ordinal by ordinal
    for p in sources:
        tg, dl = orc.generate_row(cfg, p)
        assert np.array_equal(rows[p]["tgt"], tg), p
        assert np.array_equal(rows[p]["delay"], dl), p
        w0 = cfg["w_exc0_q16"] if p % cfg["neurons_per_col"] < cfg["exc_per_col"] else cfg["w_inh0_q16"]
        assert np.all(rows[p]["w"] == w0) and np.all(rows[p]["sd"] == 0)

    # (a) sampled thalamic draws of the host generator equal the oracle's
    from paper_1310_8478_gb300 import snn
    ev = snn.snn_thalamic_events(cfg, 0, 3)
    C = cfg["grid_x"] * cfg["grid_y"]
    for i in np.random.default_rng(3).integers(0, len(ev), 64):
        e = ev[int(i)]
        assert orc.thalamic_target(cfg, int(e["t"]), int(i) % C) == int(e["gid"])

    # (b) raster invariants and counters
    n = workloads.n_neurons(cfg)
    assert len(t) == c_auto["spikes"] > 0 and c_auto["raster_dropped"] == 0
    key = t.astype(np.int64) * n + g
    assert np.all(np.diff(key) > 0) and g.min() >= 0 and g.max() < n and t.max() < STEPS
    assert 0 < c_auto["e_exc"] <= c_auto["e_all"] and c_auto["error"] == 0

    # (b) the event-driven path alone, with global reductions or column by
    # column through shared memory, gives the identical run
    for shape in (dict(dense_permille=1001, staged_permille=0xffffffff, graph_steps=1),
                  dict(dense_permille=1001, staged_permille=1)):
        _, _, digest_sparse, c_sparse = _run(eng, cfg, shape, sources)
        assert digest_sparse == digest_auto, shape
        for k in ("spikes", "e_all", "e_exc", "l_exc"):
            assert c_sparse[k] == c_auto[k], (shape, k)
