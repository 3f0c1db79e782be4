"""Batches of independent uneven networks and the launch-shape autotuner:
every net of a batch must evolve exactly as it does alone (and as the
oracle), whatever the graph chunking, tails and launch shapes."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import paper_1310_8478_gb300 as e
    e.build_engine()
    return e


def _small_mix():
    cfgs = workloads.batch_workloads(n=6, side=(1, 3), fanouts=(60, 100, 400), draw_seed=7)
    assert len({(c["grid_x"], c["fanout"]) for c in cfgs}) > 2     # really uneven
    return cfgs


def _net(eng, c, T):
    return eng.Network(c, raster_capacity=workloads.n_neurons(c) * T + 1024)


def _state(net):
    t, g = net.raster()
    w, sd = net.weights()
    return t, g, w, sd, net.counters()["e_all"]


def _same(a, b):
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert a[4] == b[4]


@pytest.mark.parametrize("graph_steps,T", [(10, 1100), (4, 1003), (50, 1050)])
def test_batch_equals_nets_run_alone(eng, graph_steps, T):
    cfgs = _small_mix()
    alone = []
    for c in cfgs:
        with _net(eng, c, T) as n:
            n.run(T)
            alone.append(_state(n))
    nets = [_net(eng, c, T) for c in cfgs]
    try:
        with eng.Batch(nets, graph_steps=graph_steps) as b:
            b.run(7)                 # a tail before the first aligned chunk
            b.run(T - 7)
        for n, ref in zip(nets, alone):
            assert n.counters()["t"] == T
            _same(_state(n), ref)
    finally:
        for n in nets:
            n.close()


def test_batch_equals_oracle(eng, orc):
    # low fan-outs keep the oracle fast; the uneven batch above covers M = 400
    cfgs = [workloads.custom(grid_x=1, grid_y=1, fanout=100, seed=1101),
            workloads.custom(grid_x=2, grid_y=2, fanout=60, pct_ring=(40, 30, 20, 10), seed=1102),
            workloads.custom(grid_x=3, grid_y=2, fanout=40, pct_ring=(40, 30, 20, 10), seed=1103)]
    nets = [_net(eng, c, 1020) for c in cfgs]
    try:
        with eng.Batch(nets, graph_steps=10) as b:
            b.run(1020)
        for c, n in zip(cfgs, nets):
            o = orc.Oracle(c)
            o.run(1020)
            ot, og = o.raster()
            gt, gg = n.raster()
            assert np.array_equal(ot, gt) and np.array_equal(og, gg)
            s = o.synapses()
            w, sd = n.weights()
            assert np.array_equal(s["w"], w) and np.array_equal(s["sd"], sd)
    finally:
        for n in nets:
            n.close()


def test_batch_of_nets_at_different_steps(eng):
    # continuous batching: nets join at different times; each keeps its own
    # clock, long-term updates happen at its own period boundaries
    cfgs = _small_mix()[:3]
    starts = [0, 3, 517]
    T = 1000
    alone = []
    for c, s0 in zip(cfgs, starts):
        with _net(eng, c, s0 + T) as n:
            n.run(s0 + T)
            alone.append(_state(n))
    nets = [_net(eng, c, s0 + T) for c, s0 in zip(cfgs, starts)]
    try:
        for n, s0 in zip(nets, starts):
            n.run(s0)
        with eng.Batch(nets, graph_steps=10) as b:
            b.run(T)
        for n, s0, ref in zip(nets, starts, alone):
            assert n.counters()["t"] == s0 + T
            _same(_state(n), ref)
        with pytest.raises(eng.SnnError):
            eng.Batch([nets[0], nets[0]])
    finally:
        for n in nets:
            n.close()


def test_batch_recaptures_after_a_net_changes(eng):
    cfgs = _small_mix()[:3]
    alone = []
    for c in cfgs:
        with _net(eng, c, 400) as n:
            n.run(200)
            n.set_launch(dense_permille=1)
            n.run(200)
            alone.append(_state(n))
    nets = [_net(eng, c, 400) for c in cfgs]
    try:
        with eng.Batch(nets, graph_steps=10) as b:
            b.run(200)
            for n in nets:
                n.set_launch(dense_permille=1)
            b.run(200)
        for n, ref in zip(nets, alone):
            _same(_state(n), ref)
    finally:
        for n in nets:
            n.close()


def test_autotune_keeps_results(eng):
    cfg = workloads.custom(grid_x=3, grid_y=2, fanout=400, pct_ring=(40, 30, 20, 10), seed=91)
    with _net(eng, cfg, 1100) as ref:
        ref.run(1010)
        r = _state(ref)
    with _net(eng, cfg, 1100) as n:
        n.run(37)
        shape = n.autotune(probe_ms=20)
        assert n.counters()["t"] == 0 and shape["graph_steps"] in (10, 50)
        n.run(1010)
        _same(_state(n), r)


def test_batch_autotune_and_shapes_keep_results(eng):
    # the batch's own launch shapes (threads per column, resident blocks,
    # chunk length) and its autotuner change nothing in the results
    cfgs = _small_mix()[:4]
    T = 1010
    alone = []
    for c in cfgs:
        with _net(eng, c, T) as n:
            n.run(T)
            alone.append(_state(n))
    nets = [_net(eng, c, T) for c in cfgs]
    try:
        with eng.Batch(nets, graph_steps=10) as b:
            b.set_launch(deliver_block=64, deliver_blocks_per_sm=1, ltp_blocks_per_sm=1, neuron_block=32,
                         graph_steps=4)
            assert b.get_launch()["graph_steps"] == 4
            b.run(T)
            for n, ref in zip(nets, alone):
                _same(_state(n), ref)
            shape = b.autotune(probe_ms=20)
            assert shape["deliver_block"] in (128, 256) and shape["graph_steps"] in (10, 50)
            assert all(n.counters()["t"] == 0 for n in nets)
            b.run(T)
        for n, ref in zip(nets, alone):
            _same(_state(n), ref)
    finally:
        for n in nets:
            n.close()


def _digest_state(n, T):
    import hashlib
    h = hashlib.sha256()
    t, g = n.raster(0, T)
    h.update(np.stack([t, g], axis=1).astype("<i4").tobytes())
    nn = n.neurons()
    h.update(nn["v"].view(np.int32).tobytes())
    h.update(nn["u"].view(np.int32).tobytes())
    c = n.counters()
    h.update(np.array([c["spikes"], c["e_all"], c["e_exc"], c["l_exc"]], np.int64).tobytes())
    # the synapses of the first and last source rows (weights and derivatives)
    for p in (0, workloads.n_neurons(n.cfg) - 1):
        syn = n.synapses(p, 1)
        h.update(syn["w"].astype("<i4").tobytes())
        h.update(syn["sd"].astype("<i4").tobytes())
    return h.hexdigest()


def test_batch_of_256_uneven_nets_equals_nets_run_alone(eng):
    # the batched workload's 256 nets (grid side 1..16, M in {100, 400,
    # 1125}, seeds 1000..1255) in waves that fit the device: every net's
    # raster, neuron state, counters and sampled synapses after 30 steps are
    # identical batched and alone
    import torch
    cfgs = workloads.batch_workloads()
    assert len(cfgs) == 256
    T = 30
    budget = int(min(100e9, 0.6 * torch.cuda.mem_get_info()[0]))
    i = 0
    while i < len(cfgs):
        wave, used = [], 0
        while i < len(cfgs):
            n = eng.Network(cfgs[i], raster_capacity=workloads.n_neurons(cfgs[i]) * T + 1024)
            if wave and used + n.device_bytes > budget:
                n.close()
                break
            wave.append(n)
            used += n.device_bytes
            i += 1
        try:
            alone = []
            for n in wave:
                n.run(T)
                alone.append(_digest_state(n, T))
                n.reset()
            with eng.Batch(wave, graph_steps=10) as b:
                b.run(T)
            for n, ref in zip(wave, alone):
                assert _digest_state(n, T) == ref, n.cfg["name"]
        finally:
            for n in wave:
                n.close()
